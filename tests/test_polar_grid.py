"""The library's polar reconstruction grid (sar_polar_grid, Sec. III-E) against
the oracle's, point for point.  The call is host-only, so these run without a
GPU; the oracle itself is pinned in tests/oracle_pins.py."""
import math

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def sar():
    import paper_2306_09784_gb300 as s
    s.load_library()
    return s


def table1(**kw):
    base = dict(f0=76.6e9, bandwidth=931e6, t_chirp=102.4e-6, pri=106.7e-6, n_samples=1024, os=4)
    base.update(kw)
    return synth.Radar(**base)


def rotated(q, ang, shift=(0.0, 0.0)):
    c, s = math.cos(ang), math.sin(ang)
    return q @ np.array([[c, s], [-s, c]]) + np.asarray(shift)


CASES = [
    # (name, radar, M, speed, rotation, shift, box, factor)
    ("paper region, 8 m/s", table1(), 1024, 8.0, 0.0, (0, 0), (-15.0125, 15.0125, 0.9875, 31.0125), 2.5),
    ("precision frame", synth.Radar(n_samples=1024, n_rx=4), 2048, 10.0, 0.0, (0, 0),
     (-10.24, 10.22, 2.0, 22.48), 2.5),
    ("box around the aperture centre", synth.Radar(n_samples=256), 256, 10.0, 0.0, (0, 0),
     (-2.3, 1.7, -1.9, 2.2), 2.5),
    ("box across the -u direction (angles wrap at pi)", synth.Radar(n_samples=256), 256, 10.0, 0.0,
     (0, 0), (-9.1, -3.2, -1.3, 1.7), 2.5),
    ("diagonal track, offset 1 km", synth.Radar(n_samples=512, n_rx=2), 512, 10.0, 0.7,
     (1000.0, -1000.0), (995.1, 1004.3, -999.2, -990.7), 3.0),
    ("finer factor", synth.Radar(n_samples=256), 256, 10.0, 0.0, (0, 0), (-1.0, 1.3, 3.0, 4.7), 6.0),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_polar_grid_matches_oracle(sar, case):
    _, radar, M, speed, ang, shift, box, factor = case
    q_tx, _ = synth.trajectory(radar, M, speed=speed)
    q_tx = rotated(q_tx, ang, shift)
    got = sar.polar_grid(radar, q_tx, box, factor)
    ref = oracle.polar_grid(radar, q_tx, box, factor)
    assert len(got) == len(ref) > 100
    assert np.max(np.abs(got - ref)) < 1e-9


def test_polar_grid_count_only_and_capacity(sar):
    import ctypes
    radar = synth.Radar(n_samples=256)
    q_tx, _ = synth.trajectory(radar, 256)
    lib = sar.load_library()
    p = sar.RadarParams(f0=radar.f0, slope=radar.slope, fs=radar.fs, c=radar.c,
                        n_samples=radar.n_samples)
    spec = sar.PolarSpec(-1.0, 1.0, 3.0, 5.0, 2.5)
    q = np.ascontiguousarray(q_tx)
    n = ctypes.c_int64()
    assert lib.sar_polar_grid(ctypes.byref(p), q.ctypes.data, len(q), ctypes.byref(spec), None, 0,
                              ctypes.byref(n)) == sar.SAR_OK
    full = n.value
    assert full == len(oracle.polar_grid(radar, q_tx, (-1.0, 1.0, 3.0, 5.0)))
    out = np.full((full, 2), 7.0)
    assert lib.sar_polar_grid(ctypes.byref(p), q.ctypes.data, len(q), ctypes.byref(spec),
                              out.ctypes.data, full - 1, ctypes.byref(n)) == sar.SAR_EINVAL
    assert n.value == full and np.all(out[-1] == 7.0)
    for bad in (sar.PolarSpec(-1.0, 1.0, 3.0, 5.0, 0.0), sar.PolarSpec(1.0, -1.0, 3.0, 5.0, 2.5),
                sar.PolarSpec(-1.0, 1.0, 3.0, float("nan"), 2.5)):
        assert lib.sar_polar_grid(ctypes.byref(p), q.ctypes.data, len(q), ctypes.byref(bad), None,
                                  0, ctypes.byref(n)) == sar.SAR_EINVAL
    still = np.repeat(q[:1], 4, axis=0)
    assert lib.sar_polar_grid(ctypes.byref(p), still.ctypes.data, 4, ctypes.byref(spec), None, 0,
                              ctypes.byref(n)) == sar.SAR_EINVAL
    assert lib.sar_polar_grid(ctypes.byref(p), q.ctypes.data, 1, ctypes.byref(spec), None, 0,
                              ctypes.byref(n)) == sar.SAR_EINVAL
