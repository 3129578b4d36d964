"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs, and compare."""
from __future__ import annotations

import math

import numpy as np

import oracle
import synth

# Tolerances from the accuracy targets: relative L2 error of the complex image
# against the FP64 oracle, and exact peak pixels.
TOL_FP32 = 1e-3
TOL_FP16 = 5e-3


def rel_l2(a, b) -> float:
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def make_plan(wl, precision=0, crop=None, pixels_xy=None, grid=True, max_pulses=None, **kw):
    import paper_2306_09784_gb300 as sar
    crop = wl.crop if crop is None else crop
    return sar.Plan.from_radar(
        wl.radar, max_pulses=max_pulses or wl.n_pulses,
        grid=wl.grid if (grid and pixels_xy is None) else None, pixels_xy=pixels_xy,
        precision=precision, crop=crop, **kw)


def to_dev(wl, beat, w_az):
    import torch
    dev = torch.device("cuda")
    b = torch.from_numpy(np.ascontiguousarray(beat)).to(dev)
    w = torch.from_numpy(np.asarray(w_az, np.float32)).to(dev) if w_az is not None else None
    qt = torch.from_numpy(np.ascontiguousarray(wl.q_tx)).to(dev)
    qr = torch.from_numpy(np.ascontiguousarray(wl.q_rx)).to(dev)
    return b, w, qt, qr


def gpu_image(plan, wl, beat, w_az, M=None, fdopp=None):
    """Range compression + backprojection on the GPU; returns complex64 numpy [P]."""
    import torch
    b, w, qt, qr = to_dev(wl, beat, w_az)
    M = M or wl.n_pulses
    prof = plan.range_compress(b[:M], w[:M] if w is not None else None)
    fd = torch.from_numpy(np.asarray(fdopp, np.float32)).cuda() if fdopp is not None else None
    img = plan.backproject(prof, M, qt[:M].contiguous(), qr[:M].contiguous(), fdopp=fd)
    torch.cuda.synchronize()
    return img.cpu().numpy()


def oracle_image(wl, beat, w_az, px=None, crop=None, sign=1, fd_idx=None, range_window=1,
                 threads=0, t0=0.0):
    r = wl.radar
    w_r = oracle.window(range_window, r.n_samples)
    S = oracle.range_compress(beat, w_r, r.os, sign=sign, threads=threads, t0=t0)
    if px is None:
        px = wl.grid.pixels()
    return oracle.backproject(r, S, wl.q_tx, wl.q_rx, px, w_az=w_az, sign=sign,
                              fd_idx=fd_idx, crop=crop if crop is not None else wl.crop,
                              threads=threads, t0=t0)


def nearest_pixel(grid, pt):
    ix = int(round((pt[0] - grid.x0) / grid.dx))
    iy = int(round((pt[1] - grid.y0) / grid.dy))
    return ix, iy


def peak_windows(wl, n_peaks=20, half=3):
    """Pixel indices of (2 half + 1)^2 windows around the strongest in-image
    scatterers (ordered by amplitude)."""
    g = wl.grid
    order = np.argsort(-np.abs(wl.amps))
    wins = []
    for k in order:
        ix, iy = nearest_pixel(g, wl.targets[k])
        if half <= ix < g.nx - half and half <= iy < g.ny - half:
            ys, xs = np.meshgrid(np.arange(iy - half, iy + half + 1),
                                 np.arange(ix - half, ix + half + 1), indexing="ij")
            wins.append((ys * g.nx + xs).ravel())
        if len(wins) >= n_peaks:
            break
    return wins


def check_peaks(img_gpu, img_ref, windows, rel_tie=1e-4):
    """The GPU argmax |P| in each window equals the oracle's; where the
    oracle's top two are within rel_tie, the GPU may pick either."""
    bad = []
    for w in windows:
        ref = np.abs(img_ref[w])
        got = np.abs(img_gpu[w])
        i_ref = int(np.argmax(ref))
        i_got = int(np.argmax(got))
        if i_ref == i_got:
            continue
        top = np.sort(ref)[-2:]
        if top[1] - top[0] <= rel_tie * top[1] and ref[i_got] >= top[0]:
            continue
        bad.append((int(w[i_ref]), int(w[i_got])))
    return bad


def sample_pixels(n_pixels, n, seed=7):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n_pixels, size=min(n, n_pixels), replace=False))


def beta_of(radar):
    a1 = radar.slope * radar.n_fft / (radar.c * radar.fs)
    return radar.f0 / (radar.c * a1)


def rotation(radar, crop, sign=1):
    """exp(sign j 2 pi frac(beta k)) for k = crop_lo .. crop_hi (FP64)."""
    k = np.arange(crop[0], crop[1] + 1, dtype=np.float64)
    b = beta_of(radar)
    return np.exp(sign * 2j * math.pi * np.mod(k * b, 1.0))
