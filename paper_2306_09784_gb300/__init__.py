"""GB300-native automotive FMCW SAR imaging: range compression and
time-domain backprojection (after arXiv 2306.09784, Alg. 2).

This module is a thin ctypes binding over the C ABI in include/sar.h
(paper_2306_09784_gb300/_lib/libsar.so): argument marshalling only, every
step of the imaging path runs in the library's CUDA kernels.  PyTorch tensors
provide device memory and streams.  Importing fails loudly when the library
has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsar.so")

(SAR_OK, SAR_EINVAL, SAR_ENOMEM, SAR_EAGAIN, SAR_ETIMEOUT, SAR_ECUDA, SAR_EBOUNDS, SAR_ENOTFOUND,
 SAR_ESCRATCH) = range(9)
WINDOW_RECT, WINDOW_HANN, WINDOW_KAISER = 0, 1, 2
PREC_FP32, PREC_FP16 = 0, 1
ORIGIN_FIRST_SAMPLE, ORIGIN_CHIRP_CENTRE = 0, 1

# Every symbol include/sar.h declares (checked by the tests).
EXPORTS = (
    "sar_plan_create", "sar_plan_destroy", "sar_plan_get_info", "sar_profile_bytes",
    "sar_range_compress", "sar_range_spectrum", "sar_backproject", "sar_form_image_host",
    "sar_plan_check_errors", "sar_status_string", "sar_version", "sar_backproject_noalloc",
    "sar_batch_create", "sar_batch_destroy", "sar_batch_clear", "sar_batch_add",
    "sar_batch_commit", "sar_batch_launch", "sar_batch_get_info",
    "sar_server_create", "sar_server_destroy", "sar_submit", "sar_poll", "sar_wait",
    "sar_release", "sar_server_get_stats", "sar_plan_autotune", "sar_plan_set_launch",
    "sar_alu_peaks", "sar_polar_grid", "sar_doppler_offsets", "sar_batch_autotune",
    "sar_batch_num_classes", "sar_batch_get_class", "sar_batch_check_errors", "sar_batch_add_frame",
    "sar_plan_set_tile_shape",
)
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = range(4)


class SarError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


class RadarParams(ctypes.Structure):
    _fields_ = [
        ("f0", ctypes.c_double), ("slope", ctypes.c_double), ("fs", ctypes.c_double),
        ("c", ctypes.c_double), ("n_samples", ctypes.c_int32), ("os", ctypes.c_int32),
        ("n_rx", ctypes.c_int32), ("max_pulses", ctypes.c_int32),
        ("range_window", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("kaiser_beta", ctypes.c_double), ("phase_sign", ctypes.c_int32),
        ("crop_lo", ctypes.c_int32), ("crop_hi", ctypes.c_int32),
        ("time_origin", ctypes.c_int32), ("max_doppler_bins", ctypes.c_double),
    ]


class Grid(ctypes.Structure):
    _fields_ = [
        ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("dx", ctypes.c_double),
        ("dy", ctypes.c_double), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("pixels_xy", ctypes.c_void_p), ("n_pixels", ctypes.c_int64),
    ]


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("n_fft", ctypes.c_int32), ("n_bins", ctypes.c_int32), ("crop_lo", ctypes.c_int32),
        ("crop_hi", ctypes.c_int32), ("n_pixels", ctypes.c_int64), ("n_tiles", ctypes.c_int32),
        ("window_bins", ctypes.c_int32), ("pulses_per_block", ctypes.c_int32),
        ("bp_ctas", ctypes.c_int32), ("bins_per_metre", ctypes.c_double),
        ("cycles_per_bin", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
        ("rx_group", ctypes.c_int32), ("regs_ctas_per_sm", ctypes.c_int32),
        ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
    ]


class PolarSpec(ctypes.Structure):
    _fields_ = [("x_min", ctypes.c_double), ("x_max", ctypes.c_double), ("y_min", ctypes.c_double),
                ("y_max", ctypes.c_double), ("factor", ctypes.c_double)]


class BatchClass(ctypes.Structure):
    _fields_ = [("rx_group", ctypes.c_int32), ("fp16", ctypes.c_int32), ("n_jobs", ctypes.c_int32),
                ("pulses_per_block", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("regs_ctas_per_sm", ctypes.c_int32), ("units", ctypes.c_int64),
                ("updates", ctypes.c_double), ("tuned_ms", ctypes.c_double),
                ("param_args", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32), ("chunk_pulses", ctypes.c_int32),
                ("quantum_mupdates", ctypes.c_int32)]


class RequestDesc(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("beat_host", ctypes.c_void_p), ("M", ctypes.c_int32),
                ("w_az_host", ctypes.c_void_p), ("q_tx_host", ctypes.c_void_p),
                ("q_rx_host", ctypes.c_void_p), ("image_host", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int32), ("active", ctypes.c_int32), ("rounds", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("pool_bytes", ctypes.c_size_t)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libsar (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libsar not built ({path} missing): run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    vp, i32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
    lib.sar_plan_create.argtypes = [ctypes.POINTER(RadarParams), ctypes.POINTER(Grid), sz,
                                    ctypes.POINTER(vp)]
    lib.sar_plan_destroy.argtypes = [vp]
    lib.sar_plan_destroy.restype = None
    lib.sar_plan_get_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
    lib.sar_profile_bytes.argtypes = [vp, i32, ctypes.POINTER(sz)]
    lib.sar_range_compress.argtypes = [vp, vp, i32, vp, vp, vp]
    lib.sar_range_spectrum.argtypes = [vp, vp, i32, vp, vp]
    lib.sar_backproject.argtypes = [vp, vp, i32, vp, vp, vp, vp, i32, vp]
    lib.sar_backproject_noalloc.argtypes = [vp, vp, i32, vp, vp, vp, vp, i32, vp]
    lib.sar_form_image_host.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp]
    lib.sar_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    lib.sar_server_destroy.argtypes = [vp]
    lib.sar_server_destroy.restype = None
    lib.sar_submit.argtypes = [vp, ctypes.POINTER(RequestDesc), ctypes.POINTER(ctypes.c_uint64)]
    lib.sar_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i32), ctypes.POINTER(vp),
                             ctypes.POINTER(ctypes.c_double)]
    lib.sar_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double]
    lib.sar_release.argtypes = [vp, ctypes.c_uint64]
    lib.sar_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    lib.sar_batch_create.argtypes = [i32, ctypes.POINTER(vp)]
    lib.sar_batch_destroy.argtypes = [vp]
    lib.sar_batch_destroy.restype = None
    lib.sar_batch_clear.argtypes = [vp]
    lib.sar_batch_add.argtypes = [vp, vp, vp, i32, vp, vp, vp, i32]
    lib.sar_batch_commit.argtypes = [vp, vp]
    lib.sar_batch_launch.argtypes = [vp, vp]
    lib.sar_batch_get_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(i32)]
    lib.sar_plan_check_errors.argtypes = [vp]
    lib.sar_plan_autotune.argtypes = [vp, vp, i32, vp, vp, vp, vp]
    lib.sar_status_string.argtypes = [ctypes.c_int]
    lib.sar_status_string.restype = ctypes.c_char_p
    lib.sar_version.argtypes = []
    dptr = ctypes.POINTER(ctypes.c_double)
    lib.sar_alu_peaks.argtypes = [dptr, dptr, dptr]
    lib.sar_polar_grid.argtypes = [ctypes.POINTER(RadarParams), vp, i32, ctypes.POINTER(PolarSpec), vp,
                                   ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    lib.sar_doppler_offsets.argtypes = [vp, vp, vp, vp, i32, vp, vp]
    lib.sar_batch_autotune.argtypes = [vp, vp]
    lib.sar_batch_num_classes.argtypes = [vp, ctypes.POINTER(i32)]
    lib.sar_batch_get_class.argtypes = [vp, i32, ctypes.POINTER(BatchClass)]
    lib.sar_batch_check_errors.argtypes = [vp, ctypes.POINTER(i32)]
    lib.sar_batch_add_frame.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, vp, i32]
    lib.sar_plan_set_tile_shape.argtypes = [vp, i32]
    for name in EXPORTS:
        fn = getattr(lib, name)
        if name not in ("sar_plan_destroy", "sar_status_string", "sar_batch_destroy",
                        "sar_server_destroy"):
            fn.restype = ctypes.c_int
    _lib = lib
    return lib


def alu_peaks() -> dict:
    """Measured FP32 FMA (scalar and packed) and MUFU throughput of the
    current CUDA device (sar_alu_peaks), in lane operations per second."""
    lib = load_library()
    f, f2, m = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib.sar_alu_peaks(ctypes.byref(f), ctypes.byref(f2), ctypes.byref(m)), "sar_alu_peaks")
    return {"fma_lane_ops_per_s": f.value, "ffma2_lane_ops_per_s": f2.value,
            "mufu_ops_per_s": m.value}


def polar_grid(radar, q_tx, box, factor: float = 2.5):
    """Polar reconstruction grid of Sec. III-E (sar_polar_grid) for a
    synth.Radar-like object, the aperture's Tx positions q_tx [M, 2] (host)
    and box = (x_min, x_max, y_min, y_max); returns float64 numpy [P, 2]."""
    import numpy as np
    lib = load_library()
    p = RadarParams(f0=radar.f0, slope=radar.slope, fs=radar.fs, c=radar.c,
                    n_samples=radar.n_samples)
    q = np.ascontiguousarray(q_tx, dtype=np.float64).reshape(-1, 2)
    spec = PolarSpec(*(float(v) for v in box), float(factor))
    n = ctypes.c_int64()
    _check(lib.sar_polar_grid(ctypes.byref(p), q.ctypes.data, len(q), ctypes.byref(spec), None, 0,
                              ctypes.byref(n)), "sar_polar_grid")
    out = np.empty((n.value, 2))
    _check(lib.sar_polar_grid(ctypes.byref(p), q.ctypes.data, len(q), ctypes.byref(spec),
                              out.ctypes.data, n.value, ctypes.byref(n)), "sar_polar_grid")
    return out


def status_string(status: int) -> str:
    try:
        return load_library().sar_status_string(status).decode()
    except ImportError:
        return f"status {status}"


def _check(rc: int, what: str):
    if rc != SAR_OK:
        raise SarError(rc, what)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream=None) -> Optional[int]:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _require_cuda(t, name, dtype=None):
    import torch
    if t is None:
        return
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")


class Plan:
    """A sar_plan: radar parameters + reconstruction points on one device."""

    def __init__(self, *, f0: float, slope: float, fs: float, c: float, n_samples: int,
                 os_factor: int, n_rx: int, max_pulses: int, grid=None, pixels_xy=None,
                 range_window: int = WINDOW_HANN, precision: int = PREC_FP32,
                 kaiser_beta: float = 6.0, phase_sign: int = 1, crop=(0, 0),
                 max_doppler_bins: float = 0.0, hbm_budget: int = 0,
                 time_origin: int = ORIGIN_FIRST_SAMPLE):
        self._lib = load_library()
        self._plan = None
        p = RadarParams(f0=f0, slope=slope, fs=fs, c=c, n_samples=n_samples, os=os_factor,
                        n_rx=n_rx, max_pulses=max_pulses, range_window=range_window,
                        precision=precision, kaiser_beta=kaiser_beta, phase_sign=phase_sign,
                        crop_lo=int(crop[0]), crop_hi=int(crop[1]),
                        time_origin=int(time_origin), max_doppler_bins=max_doppler_bins)
        g = Grid()
        self._pix_keep = None
        if pixels_xy is not None:
            import numpy as np
            arr = np.ascontiguousarray(pixels_xy, dtype=np.float64).reshape(-1, 2)
            self._pix_keep = arr
            g.pixels_xy = arr.ctypes.data
            g.n_pixels = len(arr)
        else:
            g.x0, g.y0, g.dx, g.dy, g.nx, g.ny = (grid.x0, grid.y0, grid.dx, grid.dy,
                                                  grid.nx, grid.ny)
        handle = ctypes.c_void_p()
        _check(self._lib.sar_plan_create(ctypes.byref(p), ctypes.byref(g), hbm_budget,
                                         ctypes.byref(handle)), "sar_plan_create")
        self._plan = handle
        self._pix_keep = None
        self.params = p
        self.info = PlanInfo()
        _check(self._lib.sar_plan_get_info(self._plan, ctypes.byref(self.info)),
               "sar_plan_get_info")

    @classmethod
    def from_radar(cls, radar, max_pulses: int, grid=None, pixels_xy=None, **kw):
        """Build from a synth.Radar-like object (f0, slope, fs, c, n_samples, os, n_rx)."""
        return cls(f0=radar.f0, slope=radar.slope, fs=radar.fs, c=radar.c,
                   n_samples=radar.n_samples, os_factor=radar.os, n_rx=radar.n_rx,
                   max_pulses=max_pulses, grid=grid, pixels_xy=pixels_xy, **kw)

    def close(self):
        if self._plan is not None:
            self._lib.sar_plan_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._plan

    @property
    def n_pixels(self) -> int:
        return int(self.info.n_pixels)

    def profile_bytes(self, M: int) -> int:
        n = ctypes.c_size_t()
        _check(self._lib.sar_profile_bytes(self._plan, M, ctypes.byref(n)), "sar_profile_bytes")
        return int(n.value)

    def empty_profiles(self, M: int, device="cuda"):
        import torch
        return torch.empty(self.profile_bytes(M), dtype=torch.uint8, device=device)

    def range_compress(self, beat, w_az=None, out=None, stream=None):
        """beat: complex64 [M, R, N] CUDA tensor -> profile buffer (uint8)."""
        import torch
        _require_cuda(beat, "beat", torch.complex64)
        _require_cuda(w_az, "w_az", torch.float32)
        M = beat.shape[0]
        if out is None:
            out = self.empty_profiles(M, beat.device)
        _check(self._lib.sar_range_compress(self._plan, _ptr(beat), M, _ptr(w_az), _ptr(out),
                                            _stream(stream)), "sar_range_compress")
        return out

    def range_spectrum(self, beat, out=None, stream=None):
        """beat: complex64 [M, R, N] -> complex64 [M, R, N_fft]."""
        import torch
        _require_cuda(beat, "beat", torch.complex64)
        M, R, _ = beat.shape
        if out is None:
            out = torch.empty((M, R, int(self.info.n_fft)), dtype=torch.complex64,
                              device=beat.device)
        _check(self._lib.sar_range_spectrum(self._plan, _ptr(beat), M, _ptr(out),
                                            _stream(stream)), "sar_range_spectrum")
        return out

    def backproject(self, prof, M: int, q_tx, q_rx, image=None, accumulate: bool = False,
                    fdopp=None, stream=None):
        """Alg. 2 into image (complex64 [n_pixels]); q_tx float64 [M, 2], q_rx [M, R, 2]."""
        import torch
        _require_cuda(q_tx, "q_tx", torch.float64)
        _require_cuda(q_rx, "q_rx", torch.float64)
        _require_cuda(fdopp, "fdopp", torch.float32)
        if image is None:
            image = torch.zeros(self.n_pixels, dtype=torch.complex64, device=q_tx.device)
        _require_cuda(image, "image", torch.complex64)
        _check(self._lib.sar_backproject(self._plan, _ptr(prof), M, _ptr(q_tx), _ptr(q_rx),
                                         _ptr(fdopp), _ptr(image), 1 if accumulate else 0,
                                         _stream(stream)), "sar_backproject")
        return image

    def doppler_offsets(self, q_tx, q_rx, vel, out=None, stream=None):
        """Per-pixel f_doppler(p) in bins from the mean platform velocity
        (sar_doppler_offsets): q_tx [M, 2], q_rx [M, R, 2], vel [M, 2] float64
        CUDA tensors -> float32 [n_pixels] in image order."""
        import torch
        _require_cuda(q_tx, "q_tx", torch.float64)
        _require_cuda(q_rx, "q_rx", torch.float64)
        _require_cuda(vel, "vel", torch.float64)
        if out is None:
            out = torch.empty(self.n_pixels, dtype=torch.float32, device=q_tx.device)
        _require_cuda(out, "out", torch.float32)
        _check(self._lib.sar_doppler_offsets(self._plan, _ptr(q_tx), _ptr(q_rx), _ptr(vel),
                                             q_tx.shape[0], _ptr(out), _stream(stream)),
               "sar_doppler_offsets")
        return out

    def form_image_host(self, beat, q_tx, q_rx, image, w_az=None, stream=None):
        """Whole frame from host tensors (pinned for speed); blocks until done."""
        M = beat.shape[0]
        _check(self._lib.sar_form_image_host(self._plan, _ptr(beat), M, _ptr(w_az), _ptr(q_tx),
                                             _ptr(q_rx), _ptr(image), _stream(stream)),
               "sar_form_image_host")
        return image

    def autotune(self, prof, M: int, q_tx, q_rx, image, stream=None):
        """Pick the fastest backprojection launch shape on these inputs."""
        _check(self._lib.sar_plan_autotune(self._plan, _ptr(prof), M, _ptr(q_tx), _ptr(q_rx),
                                           _ptr(image), _stream(stream)), "sar_plan_autotune")
        return self.launch_shape()

    def launch_shape(self) -> dict:
        """The backprojection launch shape the plan uses now."""
        _check(self._lib.sar_plan_get_info(self._plan, ctypes.byref(self.info)),
               "sar_plan_get_info")
        return {"tile": [int(self.info.tile_w), int(self.info.tile_h)],
                "rx_group": int(self.info.rx_group),
                "regs_ctas_per_sm": int(self.info.regs_ctas_per_sm),
                "pulses_per_block": int(self.info.pulses_per_block),
                "bp_ctas": int(self.info.bp_ctas)}

    def set_tile_shape(self, tile_w: int) -> dict:
        """Cartesian plans: tiles of tile_w x (1024 // tile_w) pixels (16, 32, 64)."""
        _check(self._lib.sar_plan_set_tile_shape(self._plan, tile_w), "sar_plan_set_tile_shape")
        return self.launch_shape()

    def set_launch(self, rx_group: int, regs_ctas_per_sm: int, pulses_per_block: int) -> dict:
        """Install an explicit launch shape (e.g. one saved after autotune)."""
        _check(self._lib.sar_plan_set_launch(self._plan, rx_group, regs_ctas_per_sm,
                                             pulses_per_block), "sar_plan_set_launch")
        return self.launch_shape()

    def check_errors(self) -> int:
        return self._lib.sar_plan_check_errors(self._plan)


class Batch:
    """A sar_batch: several backprojection requests in one persistent launch."""

    def __init__(self, max_jobs: int):
        self._lib = load_library()
        self._b = None
        h = ctypes.c_void_p()
        _check(self._lib.sar_batch_create(max_jobs, ctypes.byref(h)), "sar_batch_create")
        self._b = h
        self._keep = []

    def close(self):
        if self._b is not None:
            self._lib.sar_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def clear(self):
        _check(self._lib.sar_batch_clear(self._b), "sar_batch_clear")
        self._keep = []

    def add(self, plan: "Plan", prof, M: int, q_tx, q_rx, image, accumulate: bool = False):
        import torch
        _require_cuda(q_tx, "q_tx", torch.float64)
        _require_cuda(q_rx, "q_rx", torch.float64)
        _require_cuda(image, "image", torch.complex64)
        _check(self._lib.sar_batch_add(self._b, plan.handle, _ptr(prof), M, _ptr(q_tx), _ptr(q_rx),
                                       _ptr(image), 1 if accumulate else 0), "sar_batch_add")
        self._keep.append((plan, prof, q_tx, q_rx, image))

    def add_frame(self, plan: "Plan", beat, w_az, prof, M: int, q_tx, q_rx, image,
                  accumulate: bool = False):
        """A frame whose range compression (beat -> prof) runs in the batch's
        packed launch before its backprojection."""
        import torch
        _require_cuda(beat, "beat", torch.complex64)
        _require_cuda(w_az, "w_az", torch.float32)
        _require_cuda(q_tx, "q_tx", torch.float64)
        _require_cuda(q_rx, "q_rx", torch.float64)
        _require_cuda(image, "image", torch.complex64)
        _check(self._lib.sar_batch_add_frame(self._b, plan.handle, _ptr(beat), _ptr(w_az), _ptr(prof), M,
                                             _ptr(q_tx), _ptr(q_rx), _ptr(image),
                                             1 if accumulate else 0), "sar_batch_add_frame")
        self._keep.append((plan, beat, w_az, prof, q_tx, q_rx, image))

    def commit(self, stream=None):
        _check(self._lib.sar_batch_commit(self._b, _stream(stream)), "sar_batch_commit")

    def launch(self, stream=None):
        _check(self._lib.sar_batch_launch(self._b, _stream(stream)), "sar_batch_launch")

    def autotune(self, stream=None):
        """Pick the launch shape (per-class block sizes, register variant, CTA
        shares) by timing; the requests' images are overwritten."""
        _check(self._lib.sar_batch_autotune(self._b, _stream(stream)), "sar_batch_autotune")
        return self.classes()

    def check_errors(self):
        """(status, [code, v1, v2, v3]) of the batched kernels' checks."""
        d = (ctypes.c_int32 * 4)()
        rc = self._lib.sar_batch_check_errors(self._b, d)
        return rc, list(d)

    def classes(self):
        """The committed batch's classes and their launch shapes."""
        n = ctypes.c_int32()
        _check(self._lib.sar_batch_num_classes(self._b, ctypes.byref(n)), "sar_batch_num_classes")
        out = []
        for i in range(n.value):
            c = BatchClass()
            _check(self._lib.sar_batch_get_class(self._b, i, ctypes.byref(c)), "sar_batch_get_class")
            out.append({f: getattr(c, f) for f, _ in BatchClass._fields_})
        return out

    def info(self):
        n, u, g = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
        _check(self._lib.sar_batch_get_info(self._b, ctypes.byref(n), ctypes.byref(u),
                                            ctypes.byref(g)), "sar_batch_get_info")
        return n.value, u.value, g.value


class Server:
    """A sar_server: continuous batching of frames from several radars.

    Host tensors passed to submit() (pinned for asynchronous copies) are kept
    referenced until the request is released."""

    def __init__(self, hbm_budget: int, max_inflight: int = 64, queue_capacity: int = 1024,
                 chunk_pulses: int = 2048, quantum_mupdates: int = 0):
        self._lib = load_library()
        self._s = None
        cfg = ServerConfig(hbm_budget_bytes=hbm_budget, max_inflight=max_inflight,
                           queue_capacity=queue_capacity, chunk_pulses=chunk_pulses,
                           quantum_mupdates=quantum_mupdates)
        h = ctypes.c_void_p()
        _check(self._lib.sar_server_create(ctypes.byref(cfg), ctypes.byref(h)), "sar_server_create")
        self._s = h
        self._keep = {}

    def close(self):
        if self._s is not None:
            self._lib.sar_server_destroy(self._s)
            self._s = None
            self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, plan: "Plan", beat, q_tx, q_rx, w_az=None, image=None, M=None) -> int:
        """Queue one frame; returns its ticket (raises SarError, e.g. SAR_EAGAIN)."""
        M = beat.shape[0] if M is None else M
        req = RequestDesc(plan=plan.handle.value, beat_host=_ptr(beat), M=M, w_az_host=_ptr(w_az),
                          q_tx_host=_ptr(q_tx), q_rx_host=_ptr(q_rx), image_host=_ptr(image))
        t = ctypes.c_uint64()
        _check(self._lib.sar_submit(self._s, ctypes.byref(req), ctypes.byref(t)), "sar_submit")
        self._keep[t.value] = (plan, beat, q_tx, q_rx, w_az, image)
        return t.value

    def poll(self, ticket: int):
        """(status, state, device image pointer, latency_ms)."""
        st, img, lat = ctypes.c_int32(), ctypes.c_void_p(), ctypes.c_double()
        rc = self._lib.sar_poll(self._s, ticket, ctypes.byref(st), ctypes.byref(img),
                                ctypes.byref(lat))
        return rc, st.value, img.value, lat.value

    def wait(self, ticket: int, timeout_ms: float = 60000.0) -> int:
        return self._lib.sar_wait(self._s, ticket, timeout_ms)

    def release(self, ticket: int) -> int:
        rc = self._lib.sar_release(self._s, ticket)
        self._keep.pop(ticket, None)
        return rc

    def stats(self) -> ServerStats:
        st = ServerStats()
        _check(self._lib.sar_server_get_stats(self._s, ctypes.byref(st)), "sar_server_get_stats")
        return st
