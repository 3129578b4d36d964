"""Python access to the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline and reference legs use it; the CUDA library never imports it.

``build()`` compiles oracle.c with gcc into oracle/_build/liboracle.so; the
other functions take and return numpy arrays (complex128 / float64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()

WINDOW_RECT, WINDOW_HANN, WINDOW_KAISER = 0, 1, 2


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH,
          extra_flags=()) -> str:
    """Compile the oracle (plain C, -O2, OpenMP) to a shared library."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
           *extra_flags, src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    i, d = ctypes.c_int, ctypes.c_double
    lib.oracle_window.argtypes = [i, i, d, dp]
    lib.oracle_dft.argtypes = [i, dp, i, i, dp]
    lib.oracle_fft.argtypes = [i, dp, i]
    lib.oracle_range_compress.argtypes = [i, i, i, i, dp, dp, i, d, dp, i]
    lib.oracle_backproject.argtypes = [d, d, d, d, i, i, i, i, i, i, dp, dp, dp,
                                       dp, dp, i, dp, dp, i]
    lib.oracle_backproject_alg1.argtypes = [d, d, d, d, i, i, i, i, i, i, dp, dp,
                                            dp, dp, dp, i, dp, dp, i]
    lib.oracle_matched_filter.argtypes = [d, d, d, d, i, i, i, i, dp, dp, dp, dp,
                                          dp, i, dp, dp, i]
    lib.oracle_polar_grid.argtypes = [d, d, d, d, i, i, dp, d, d, d, d, d, ctypes.c_longlong, dp,
                                      ctypes.POINTER(ctypes.c_longlong)]
    lib.oracle_doppler_offsets.argtypes = [d, d, d, i, i, i, dp, dp, dp, i, dp, dp]
    for name in ("oracle_window", "oracle_dft", "oracle_fft", "oracle_range_compress",
                 "oracle_backproject", "oracle_backproject_alg1",
                 "oracle_matched_filter", "oracle_threads", "oracle_version",
                 "oracle_polar_grid", "oracle_doppler_offsets"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load (building first if needed) and return the ctypes library."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"{what} failed (rc={rc})")


def window(kind: int, L: int, beta: float = 6.0, lib=None) -> np.ndarray:
    lib = lib or load()
    w = np.empty(L)
    _check(lib.oracle_window(kind, L, beta, _ptr(w)), "oracle_window")
    return w


def dft(x, n_out: int, sign: int = 1, lib=None) -> np.ndarray:
    lib = lib or load()
    x = _c128(x)
    X = np.empty(n_out, np.complex128)
    _check(lib.oracle_dft(len(x), _ptr(x.view(np.float64)), n_out, sign,
                          _ptr(X.view(np.float64))), "oracle_dft")
    return X


def fft(x, sign: int = 1, lib=None) -> np.ndarray:
    lib = lib or load()
    X = _c128(x).copy()
    _check(lib.oracle_fft(len(X), _ptr(X.view(np.float64)), sign), "oracle_fft")
    return X


def range_compress(beat, w_r, os_factor: int, sign: int = 1, threads: int = 0,
                   lib=None, t0: float = 0.0) -> np.ndarray:
    """beat [M, R, N] -> S [M, R, N * os], transform time origin t0 samples."""
    lib = lib or load()
    beat = _c128(beat)
    M, R, N = beat.shape
    S = np.empty((M, R, N * os_factor), np.complex128)
    _check(lib.oracle_range_compress(N, os_factor, M, R, _ptr(beat.view(np.float64)),
                                     _ptr(_f64(w_r)), sign, float(t0),
                                     _ptr(S.view(np.float64)), threads),
           "oracle_range_compress")
    return S


def carrier_at(radar, t0: float) -> float:
    """The frequency at time t0 / fs into the chirp, f0 + mu t0 / fs: the
    beat phase f0 tau + mu tau t of Sec. II, with its time origin moved to
    sample t0, has this as its constant-phase coefficient."""
    return radar.f0 + radar.slope * t0 / radar.fs


def backproject(radar, S, q_tx, q_rx, px, w_az=None, fd_idx=None, sign: int = 1,
                crop=None, threads: int = 0, lib=None, t0: float = 0.0) -> np.ndarray:
    """Alg. 2 on the pixel list px [P, 2]; returns complex128 [P].  S must come
    from a range transform with time origin t0 (samples); the phase then uses
    the carrier at that origin."""
    lib = lib or load()
    S = _c128(S)
    M, R, nfft = S.shape
    lo, hi = crop if crop is not None else (0, nfft - 1)
    px = _f64(px).reshape(-1, 2)
    out = np.empty(len(px), np.complex128)
    _check(lib.oracle_backproject(carrier_at(radar, t0), radar.slope, radar.fs, radar.c, nfft, sign,
                                  lo, hi, M, R, _ptr(S.view(np.float64)),
                                  _ptr(_f64(q_tx)), _ptr(_f64(q_rx)), _ptr(_f64(w_az)),
                                  _ptr(_f64(fd_idx)), len(px), _ptr(px),
                                  _ptr(out.view(np.float64)), threads),
           "oracle_backproject")
    return out


def backproject_alg1(radar, S, q_tx, q_rx, px, vel=None, w_az=None, sign: int = 1,
                     crop=None, threads: int = 0, lib=None) -> np.ndarray:
    """Alg. 1 (with optional per-chirp velocity vel [M, 2])."""
    lib = lib or load()
    S = _c128(S)
    M, R, nfft = S.shape
    lo, hi = crop if crop is not None else (0, nfft - 1)
    px = _f64(px).reshape(-1, 2)
    out = np.empty(len(px), np.complex128)
    _check(lib.oracle_backproject_alg1(radar.f0, radar.slope, radar.fs, radar.c, nfft,
                                       sign, lo, hi, M, R, _ptr(S.view(np.float64)),
                                       _ptr(_f64(q_tx)), _ptr(_f64(q_rx)), _ptr(_f64(vel)),
                                       _ptr(_f64(w_az)), len(px), _ptr(px),
                                       _ptr(out.view(np.float64)), threads),
           "oracle_backproject_alg1")
    return out


def matched_filter(radar, beat, w_r, q_tx, q_rx, px, w_az=None, sign: int = 1,
                   threads: int = 0, lib=None) -> np.ndarray:
    """Brute-force matched filter on the pixel list px [P, 2]."""
    lib = lib or load()
    beat = _c128(beat)
    M, R, N = beat.shape
    px = _f64(px).reshape(-1, 2)
    out = np.empty(len(px), np.complex128)
    _check(lib.oracle_matched_filter(radar.f0, radar.slope, radar.fs, radar.c, sign, N,
                                     M, R, _ptr(beat.view(np.float64)), _ptr(_f64(w_r)),
                                     _ptr(_f64(q_tx)), _ptr(_f64(q_rx)), _ptr(_f64(w_az)),
                                     len(px), _ptr(px), _ptr(out.view(np.float64)),
                                     threads), "oracle_matched_filter")
    return out


def polar_grid(radar, q_tx, box, factor: float = 2.5, lib=None) -> np.ndarray:
    """Polar reconstruction grid of Sec. III-E inside box = (x_min, x_max,
    y_min, y_max); returns float64 [P, 2] (rings by range, then angle)."""
    lib = lib or load()
    q = _f64(q_tx).reshape(-1, 2)
    n = ctypes.c_longlong()
    args = (radar.f0, radar.slope, radar.fs, radar.c, radar.n_samples, len(q), _ptr(q),
            float(box[0]), float(box[1]), float(box[2]), float(box[3]), float(factor))
    _check(lib.oracle_polar_grid(*args, 0, None, ctypes.byref(n)), "oracle_polar_grid")
    out = np.empty((n.value, 2))
    _check(lib.oracle_polar_grid(*args, n.value, _ptr(out), ctypes.byref(n)), "oracle_polar_grid")
    return out


def doppler_offsets(radar, q_tx, q_rx, vel, px, t0: float = 0.0, lib=None) -> np.ndarray:
    """Per-pixel f_doppler(p) in bins (Alg. 2, Sec. III-D) from the mean
    platform velocity vel [M, 2] and the mean antenna positions; the carrier
    is the one at the transform's time origin t0 (samples)."""
    lib = lib or load()
    q = _f64(q_tx).reshape(-1, 2)
    M = len(q)
    qr = _f64(q_rx).reshape(M, -1, 2)
    px = _f64(px).reshape(-1, 2)
    out = np.empty(len(px))
    _check(lib.oracle_doppler_offsets(carrier_at(radar, t0), radar.fs, radar.c, radar.n_fft, M,
                                      qr.shape[1], _ptr(q), _ptr(qr), _ptr(_f64(vel).reshape(M, 2)),
                                      len(px), _ptr(px), _ptr(out)), "oracle_doppler_offsets")
    return out


def threads(lib=None) -> int:
    return (lib or load()).oracle_threads()


def form_image(wl, beat, w_az=None, range_window: int = WINDOW_HANN, sign: int = 1,
               px=None, crop=None, threads: int = 0, t0: float = 0.0):
    """Range compression then Alg. 2 for a synth.Workload (convenience)."""
    r = wl.radar
    w_r = window(range_window, r.n_samples)
    S = range_compress(beat, w_r, r.os, sign=sign, threads=threads, t0=t0)
    if px is None:
        px = wl.grid.pixels()
    return backproject(r, S, wl.q_tx, wl.q_rx, px, w_az=w_az, sign=sign,
                       crop=crop if crop is not None else wl.crop, threads=threads, t0=t0)
