"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/sar.h declares; the Python structs match the C layout.  No GPU
needed (no compute calls)."""
import ctypes
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sar.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sar_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2306_09784_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("sar_plan_create", "sar_range_compress", "sar_backproject", "sar_plan_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_binding_lists_every_declared_symbol():
    import paper_2306_09784_gb300 as sar
    assert sorted(sar.EXPORTS) == declared_functions()


def test_status_strings(lib):
    lib.sar_status_string.restype = ctypes.c_char_p
    assert lib.sar_status_string(0) == b"ok"
    assert lib.sar_status_string(2).startswith(b"out of device memory")
    lib.sar_version.restype = ctypes.c_int
    assert lib.sar_version() >= 100


def test_null_arguments_rejected_without_gpu(lib):
    """Argument checks run on the host before any CUDA call."""
    lib.sar_plan_create.restype = ctypes.c_int
    assert lib.sar_plan_create(None, None, 0, None) == 1
    out = ctypes.c_void_p()
    assert lib.sar_plan_create(None, None, 0, ctypes.byref(out)) == 1
    for fn in ("sar_range_compress", "sar_backproject", "sar_profile_bytes",
               "sar_plan_get_info", "sar_plan_check_errors"):
        getattr(lib, fn).restype = ctypes.c_int
    assert lib.sar_range_compress(None, None, 1, None, None, None) == 1
    assert lib.sar_backproject(None, None, 1, None, None, None, None, 0, None) == 1
    assert lib.sar_plan_check_errors(None) == 1
    lib.sar_alu_peaks.restype = ctypes.c_int
    assert lib.sar_alu_peaks(None, None, None) == 1


def test_plan_parameters_rejected_without_gpu(lib):
    """Radar parameters are validated on the host before any CUDA call:
    each bad value below gives SAR_EINVAL (1)."""
    import paper_2306_09784_gb300 as sar
    lib.sar_plan_create.restype = ctypes.c_int

    def params(**kw):
        p = dict(f0=77e9, slope=1e9 / 102.4e-6, fs=128 / 102.4e-6, c=299792458.0, n_samples=128,
                 os=4, n_rx=4, max_pulses=64, range_window=1, precision=0, kaiser_beta=0.0,
                 phase_sign=1, crop_lo=0, crop_hi=0, time_origin=0, max_doppler_bins=0.0)
        p.update(kw)
        return sar.RadarParams(**p)

    grid = sar.Grid(x0=-1.0, y0=2.0, dx=0.05, dy=0.05, nx=8, ny=8, pixels_xy=None, n_pixels=0)
    bad = [dict(f0=0.0), dict(f0=float("nan")), dict(slope=0.0), dict(fs=-1.0), dict(c=0.0),
           dict(n_samples=0), dict(os=3), dict(n_rx=0), dict(n_rx=65), dict(max_pulses=0),
           dict(n_samples=8, os=4), dict(n_samples=8192, os=4), dict(range_window=3),
           dict(precision=2), dict(phase_sign=0), dict(crop_lo=10, crop_hi=5),
           dict(crop_lo=0, crop_hi=512), dict(max_doppler_bins=-1.0), dict(max_doppler_bins=100.0),
           dict(range_window=2, kaiser_beta=-1.0), dict(time_origin=2), dict(time_origin=-1),
           dict(f0=1e-6),      # beta = f0 / (c a1) ~ 2.5e-15 cycles per bin
           dict(f0=1e19),      # beta ~ 2.5e9
           dict(slope=-1e9 / 102.4e-6)]  # a1 < 0
    for kw in bad:
        out = ctypes.c_void_p()
        p = params(**kw)
        assert lib.sar_plan_create(ctypes.byref(p), ctypes.byref(grid), 0, ctypes.byref(out)) == 1, kw
        assert out.value is None


def test_empty_or_invalid_grids_rejected_without_gpu(lib):
    """An empty Cartesian grid, an empty point list, an oversized grid or a
    non-finite grid origin gives SAR_EINVAL (1) before any CUDA call."""
    import paper_2306_09784_gb300 as sar
    lib.sar_plan_create.restype = ctypes.c_int
    p = sar.RadarParams(f0=77e9, slope=1e9 / 102.4e-6, fs=128 / 102.4e-6, c=299792458.0,
                        n_samples=128, os=4, n_rx=4, max_pulses=64, range_window=1, precision=0,
                        kaiser_beta=0.0, phase_sign=1, crop_lo=0, crop_hi=0, time_origin=0,
                        max_doppler_bins=0.0)
    pts = (ctypes.c_double * 2)(0.0, 3.0)
    bad = [dict(nx=0, ny=8), dict(nx=8, ny=0), dict(nx=-1, ny=8), dict(nx=1 << 16, ny=1 << 15),
           dict(nx=8, ny=8, x0=float("nan")), dict(nx=8, ny=8, dx=float("inf")),
           dict(pixels_xy=ctypes.cast(pts, ctypes.c_void_p), n_pixels=0),
           dict(pixels_xy=ctypes.cast(pts, ctypes.c_void_p), n_pixels=-5)]
    for kw in bad:
        g = dict(x0=-1.0, y0=2.0, dx=0.05, dy=0.05, nx=8, ny=8, pixels_xy=None, n_pixels=0)
        g.update(kw)
        grid = sar.Grid(**g)
        out = ctypes.c_void_p()
        assert lib.sar_plan_create(ctypes.byref(p), ctypes.byref(grid), 0, ctypes.byref(out)) == 1, kw
        assert out.value is None
    assert lib.sar_plan_create(ctypes.byref(p), None, 0, ctypes.byref(out)) == 1


def test_struct_layouts_match_header():
    import paper_2306_09784_gb300 as sar
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "sar.h"
#define P(T, F) printf(#T "." #F " %zu\n", offsetof(T, F));
int main(void) {
  printf("sar_radar_params %zu\nsar_grid %zu\nsar_plan_info %zu\n",
         sizeof(sar_radar_params), sizeof(sar_grid), sizeof(sar_plan_info));
  P(sar_radar_params, kaiser_beta) P(sar_radar_params, phase_sign) P(sar_radar_params, time_origin)
  P(sar_radar_params, max_doppler_bins)
  P(sar_grid, pixels_xy) P(sar_grid, n_pixels)
  P(sar_plan_info, n_pixels) P(sar_plan_info, bins_per_metre) P(sar_plan_info, device_bytes)
  P(sar_plan_info, rx_group) P(sar_plan_info, regs_ctas_per_sm) P(sar_plan_info, tile_w)
  P(sar_plan_info, tile_h)
  printf("sar_batch_class %zu\n", sizeof(sar_batch_class));
  P(sar_batch_class, units) P(sar_batch_class, updates) P(sar_batch_class, tuned_ms)
  P(sar_batch_class, param_args)
  printf("sar_server_config %zu\nsar_request %zu\nsar_server_stats %zu\n",
         sizeof(sar_server_config), sizeof(sar_request), sizeof(sar_server_stats));
  P(sar_request, M) P(sar_request, w_az_host) P(sar_request, image_host)
  P(sar_server_config, chunk_pulses) P(sar_server_stats, rounds) P(sar_server_stats, pool_bytes)
  printf("sar_polar_spec %zu\n", sizeof(sar_polar_spec));
  P(sar_polar_spec, factor)
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "t.c")
        open(src, "w").write(prog)
        exe = os.path.join(td, "t")
        subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.rsplit(" ", 1) for l in lines if l)
    assert int(got["sar_radar_params"]) == ctypes.sizeof(sar.RadarParams)
    assert int(got["sar_grid"]) == ctypes.sizeof(sar.Grid)
    assert int(got["sar_plan_info"]) == ctypes.sizeof(sar.PlanInfo)
    assert int(got["sar_radar_params.kaiser_beta"]) == sar.RadarParams.kaiser_beta.offset
    assert int(got["sar_radar_params.phase_sign"]) == sar.RadarParams.phase_sign.offset
    assert int(got["sar_radar_params.time_origin"]) == sar.RadarParams.time_origin.offset
    assert int(got["sar_radar_params.max_doppler_bins"]) == sar.RadarParams.max_doppler_bins.offset
    assert int(got["sar_grid.pixels_xy"]) == sar.Grid.pixels_xy.offset
    assert int(got["sar_grid.n_pixels"]) == sar.Grid.n_pixels.offset
    assert int(got["sar_plan_info.n_pixels"]) == sar.PlanInfo.n_pixels.offset
    assert int(got["sar_plan_info.bins_per_metre"]) == sar.PlanInfo.bins_per_metre.offset
    assert int(got["sar_plan_info.device_bytes"]) == sar.PlanInfo.device_bytes.offset
    assert int(got["sar_plan_info.rx_group"]) == sar.PlanInfo.rx_group.offset
    assert int(got["sar_plan_info.regs_ctas_per_sm"]) == sar.PlanInfo.regs_ctas_per_sm.offset
    assert int(got["sar_plan_info.tile_w"]) == sar.PlanInfo.tile_w.offset
    assert int(got["sar_plan_info.tile_h"]) == sar.PlanInfo.tile_h.offset
    assert int(got["sar_batch_class"]) == ctypes.sizeof(sar.BatchClass)
    for f in ("units", "updates", "tuned_ms", "param_args"):
        assert int(got[f"sar_batch_class.{f}"]) == getattr(sar.BatchClass, f).offset
    assert int(got["sar_server_config"]) == ctypes.sizeof(sar.ServerConfig)
    assert int(got["sar_request"]) == ctypes.sizeof(sar.RequestDesc)
    assert int(got["sar_server_stats"]) == ctypes.sizeof(sar.ServerStats)
    assert int(got["sar_request.M"]) == sar.RequestDesc.M.offset
    assert int(got["sar_request.w_az_host"]) == sar.RequestDesc.w_az_host.offset
    assert int(got["sar_request.image_host"]) == sar.RequestDesc.image_host.offset
    assert int(got["sar_server_config.chunk_pulses"]) == sar.ServerConfig.chunk_pulses.offset
    assert int(got["sar_server_stats.rounds"]) == sar.ServerStats.rounds.offset
    assert int(got["sar_server_stats.pool_bytes"]) == sar.ServerStats.pool_bytes.offset
    assert int(got["sar_polar_spec"]) == ctypes.sizeof(sar.PolarSpec)
    assert int(got["sar_polar_spec.factor"]) == sar.PolarSpec.factor.offset
