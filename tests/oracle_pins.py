"""Pins for the FP64 oracle: checks against what the paper and the mathematics
fix, independent of the oracle's own code paths.

Each ``pin_*`` takes the loaded oracle library (so the mutation test can run
them against deliberately broken builds) and raises AssertionError on failure.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
import synth

C0 = synth.C0


def _radar(**kw):
    base = dict(n_samples=64, n_rx=2, os=4)
    base.update(kw)
    return synth.Radar(**base)


def _point_scene(radar, M, target, amp, offset=(0.0, 0.0)):
    q_tx, q_rx = synth.trajectory(radar, M, offset=offset)
    tgt = np.asarray(target, dtype=np.float64)[None, :] + np.asarray(offset)[None, :]
    beat = synth.beat_signal(radar, q_tx, q_rx, tgt, np.array([amp]))
    return q_tx, q_rx, beat


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# --------------------------------------------------------------------------
# transforms and windows
# --------------------------------------------------------------------------
def pin_fft(lib):
    """Oracle FFT = numpy's (i)fft (library routine) = direct-sum DFT."""
    rng = np.random.Generator(np.random.PCG64(11))
    for n in (1, 2, 8, 64, 1024):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        Xp = oracle.fft(x, +1, lib=lib)
        Xm = oracle.fft(x, -1, lib=lib)
        assert np.allclose(Xp, np.fft.ifft(x) * n, rtol=0, atol=1e-9 * max(1, n))
        assert np.allclose(Xm, np.fft.fft(x), rtol=0, atol=1e-9 * max(1, n))
    # textbook DFT with zero padding vs an explicit numpy matrix product
    x = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    k = np.arange(48)[:, None]
    n = np.arange(12)[None, :]
    ref = np.exp(2j * np.pi * n * k / 48) @ x
    assert np.allclose(oracle.dft(x, 48, +1, lib=lib), ref, atol=1e-10)


def pin_windows(lib):
    """Hann / Kaiser / rect against numpy's window routines."""
    for L in (1, 2, 7, 64, 255):
        assert np.allclose(oracle.window(oracle.WINDOW_HANN, L, lib=lib),
                           np.hanning(L) if L > 1 else np.ones(1), atol=1e-15)
        assert np.allclose(oracle.window(oracle.WINDOW_KAISER, L, 6.0, lib=lib),
                           np.kaiser(L, 6.0), atol=1e-12)
        assert np.all(oracle.window(oracle.WINDOW_RECT, L, lib=lib) == 1.0)


def pin_range_compress(lib):
    """Range compression = per-row textbook DFT of the windowed row."""
    rng = np.random.Generator(np.random.PCG64(5))
    M, R, N, os_ = 3, 2, 16, 4
    beat = rng.standard_normal((M, R, N)) + 1j * rng.standard_normal((M, R, N))
    w = np.hanning(N)
    S = oracle.range_compress(beat, w, os_, +1, lib=lib)
    k = np.arange(N * os_)[:, None]
    n = np.arange(N)[None, :]
    E = np.exp(2j * np.pi * n * k / (N * os_))
    ref = np.einsum("kn,mrn->mrk", E, beat * w)
    assert np.allclose(S, ref, atol=1e-10)
    Sm = oracle.range_compress(beat, w, os_, -1, lib=lib)
    assert np.allclose(Sm, np.einsum("kn,mrn->mrk", E.conj(), beat * w), atol=1e-10)
    # time origin at the chirp centre: the DFT over the centred index n - t0
    t0 = (N - 1) / 2.0
    Ec = np.exp(2j * np.pi * (n - t0) * k / (N * os_))
    for sg, Es in ((+1, Ec), (-1, Ec.conj())):
        Sc = oracle.range_compress(beat, w, os_, sg, lib=lib, t0=t0)
        assert np.allclose(Sc, np.einsum("kn,mrn->mrk", Es, beat * w), atol=1e-10)


# --------------------------------------------------------------------------
# point-target closed forms
# --------------------------------------------------------------------------
def pin_matched_filter_closed_form(lib):
    """Noiseless stop-and-hop point target on a pixel: every term of the
    matched filter is a * sum(w_r) * w_az[m], so |P_bf| = |a| R sum(w_az) sum(w_r)
    (rect windows: |a| R M N, the pulse-count-times-amplitude sum)."""
    radar = _radar()
    M = 24
    a = 0.7 * np.exp(0.4j)
    tgt = (0.3, 3.0)
    q_tx, q_rx, beat = _point_scene(radar, M, tgt, a)
    N, R = radar.n_samples, radar.n_rx
    P = oracle.matched_filter(radar, beat, np.ones(N), q_tx, q_rx,
                              np.array([tgt]), lib=lib)
    assert abs(P[0] - a * R * M * N) < 1e-9 * abs(a) * R * M * N
    w_az = np.hanning(M)
    w_r = np.hanning(N)
    P = oracle.matched_filter(radar, beat, w_r, q_tx, q_rx, np.array([tgt]), w_az=w_az,
                              lib=lib)
    ref = a * R * w_az.sum() * w_r.sum()
    assert abs(P[0] - ref) < 1e-9 * abs(ref)
    # conjugate convention: beat generated with the opposite sign convention
    # images to the conjugate
    Pm = oracle.matched_filter(radar, beat.conj(), np.ones(N), q_tx, q_rx,
                               np.array([tgt]), sign=-1, lib=lib)
    assert abs(Pm[0] - np.conj(a) * R * M * N) < 1e-9 * abs(a) * R * M * N


def pin_backproject_point_target(lib):
    """FFT + linear interpolation at the target: within the interpolation loss
    of the closed form, phase equal to arg(a), peak on the true pixel."""
    radar = _radar(os=4)
    M = 24
    a = 1.3 * np.exp(-1.1j)
    tgt = (0.3, 3.0)
    q_tx, q_rx, beat = _point_scene(radar, M, tgt, a)
    N, R = radar.n_samples, radar.n_rx
    S = oracle.range_compress(beat, np.ones(N), radar.os, lib=lib)
    P = oracle.backproject(radar, S, q_tx, q_rx, np.array([tgt]), lib=lib)[0]
    ref = a * R * M * N
    ratio = abs(P) / abs(ref)
    # linear interpolation between bins whose phases differ by ~pi/os loses at
    # most 1 - cos(pi / (2 os)) at mid-bin, plus the Dirichlet roll-off
    assert 0.85 <= ratio <= 1.0 + 1e-9, ratio
    assert abs(np.angle(P / ref)) < 0.05
    # peak on the true pixel of a local grid at a third of the range
    # resolution (finer grids resolve the interpolation ripple instead)
    g = synth.Grid(x0=tgt[0] - 0.2, y0=tgt[1] - 0.2, dx=0.05, dy=0.05, nx=9, ny=9)
    img = oracle.backproject(radar, S, q_tx, q_rx, g.pixels(), lib=lib)
    assert int(np.argmax(np.abs(img))) == 4 * 9 + 4


def pin_time_origin_mid_bin(lib):
    """One term whose index falls exactly half-way between two bins (one chirp,
    Rx at the Tx, range-window Hann).  With the transform's time origin at the
    chirp centre, the windowed tone's spectrum is real around its peak, so the
    interpolated magnitude is the window transform half a bin off,
    C = sum_n w[n] cos(pi (n - (N-1)/2) / N_fft), and the image phase is arg(a).
    With the origin at sample 0 the two neighbours differ in phase by
    pi (N-1) / N_fft, and interpolation loses cos(pi (N-1) / (2 N_fft)) more."""
    radar = _radar(n_rx=1, os=4)
    N, nfft = radar.n_samples, radar.n_fft
    w = np.hanning(N)
    a = 0.9 * np.exp(0.4j)
    d = (100.5) / radar.bins_per_metre            # two-way path on a mid-bin index
    q_tx = np.array([[0.0, 0.0]])
    q_rx = np.array([[[0.0, 0.0]]])
    tgt = np.array([[0.0, d / 2.0]])
    beat = synth.beat_signal(radar, q_tx, q_rx, tgt, np.array([a]))
    t0 = (N - 1) / 2.0
    C = abs(np.sum(w * np.cos(np.pi * (np.arange(N) - t0) / nfft)))
    for origin, expect in ((t0, C), (0.0, C * math.cos(np.pi * (N - 1) / (2.0 * nfft)))):
        S = oracle.range_compress(beat, w, radar.os, lib=lib, t0=origin)
        P = oracle.backproject(radar, S, q_tx, q_rx, tgt, lib=lib, t0=origin)[0]
        assert abs(abs(P) - abs(a) * expect) < 1e-9 * abs(a) * C, (origin, abs(P), expect)
        assert abs(np.angle(P / a)) < 1e-9


def pin_interpolation_convergence(lib):
    """FFT + lerp converges to the brute-force matched filter as the
    zero-padding factor grows: linear interpolation is second order, so the
    error falls by ~4 per doubling of os."""
    rng = np.random.Generator(np.random.PCG64(3))
    M = 16
    tg = np.stack([rng.uniform(-0.5, 0.5, 3), rng.uniform(2.5, 3.5, 3)], 1)
    am = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    g = synth.Grid(x0=-0.6, y0=2.4, dx=0.1, dy=0.1, nx=13, ny=13)
    errs, errs_c = [], []
    for os_ in (4, 8, 16):
        radar = _radar(os=os_)
        q_tx, q_rx = synth.trajectory(radar, M)
        beat = synth.beat_signal(radar, q_tx, q_rx, tg, am)
        w_r = np.hanning(radar.n_samples)
        ref = oracle.matched_filter(radar, beat, w_r, q_tx, q_rx, g.pixels(), lib=lib)
        S = oracle.range_compress(beat, w_r, os_, lib=lib)
        img = oracle.backproject(radar, S, q_tx, q_rx, g.pixels(), lib=lib)
        errs.append(rel_l2(img, ref))
        # the same limit with the transform's time origin at the chirp centre,
        # where the spectrum's phase is flat across the main lobe
        t0 = (radar.n_samples - 1) / 2.0
        S = oracle.range_compress(beat, w_r, os_, lib=lib, t0=t0)
        img = oracle.backproject(radar, S, q_tx, q_rx, g.pixels(), lib=lib, t0=t0)
        errs_c.append(rel_l2(img, ref))
    assert errs[0] < 0.1, errs
    assert errs[1] / errs[0] < 0.35 and errs[2] / errs[1] < 0.35, errs
    assert errs_c[1] / errs_c[0] < 0.35 and errs_c[2] / errs_c[1] < 0.35, errs_c
    assert all(c < 0.2 * e for c, e in zip(errs_c, errs)), (errs_c, errs)


def _minus3db_width(coord, mag):
    """Full width at half power of a sampled main lobe (linear edges)."""
    p = mag / mag.max()
    k = int(np.argmax(p))
    thr = 1 / math.sqrt(2)
    i = k
    while p[i] > thr:
        i -= 1
    left = coord[i] + (thr - p[i]) / (p[i + 1] - p[i]) * (coord[i + 1] - coord[i])
    j = k
    while p[j] > thr:
        j += 1
    right = coord[j - 1] + (p[j - 1] - thr) / (p[j - 1] - p[j]) * (coord[j] - coord[j - 1])
    return right - left


def pin_resolution(lib):
    """-3 dB widths of a point target: range 0.886 c / 2B with rect and
    1.44 c / 2B with Hann range windows (textbook DFT main lobes); azimuth
    0.886 lambda y / 2L for a rect aperture of length L."""
    radar = _radar(n_samples=128, n_rx=1, os=4)
    M = 256
    tgt = (0.0, 4.0)
    q_tx, q_rx, beat = _point_scene(radar, M, tgt, 1.0)
    N = radar.n_samples
    ys = np.arange(-0.3, 0.3, 0.002) + tgt[1]
    line = np.stack([np.zeros_like(ys), ys], 1)
    res = C0 / (2 * radar.bandwidth)
    for w_r, k_w in ((np.ones(N), 0.886), (np.hanning(N), 1.44)):
        P = oracle.matched_filter(radar, beat, w_r, q_tx, q_rx, line, lib=lib)
        width = _minus3db_width(ys, np.abs(P))
        assert abs(width / (k_w * res) - 1) < 0.10, (width, k_w * res)
    xs = np.arange(-0.08, 0.08, 0.0005)
    line = np.stack([xs, np.full_like(xs, tgt[1])], 1)
    P = oracle.matched_filter(radar, beat, np.ones(N), q_tx, q_rx, line, lib=lib)
    L = (M - 1) * 10.0 * radar.pri
    az = 0.886 * radar.wavelength * tgt[1] / (2 * L)
    width = _minus3db_width(xs, np.abs(P))
    assert abs(width / az - 1) < 0.10, (width, az)


# --------------------------------------------------------------------------
# invariants of the backprojection
# --------------------------------------------------------------------------
def _small_case(lib, R=2, M=20, seed=1, offset=(0.0, 0.0)):
    radar = _radar(n_rx=R)
    rng = np.random.Generator(np.random.PCG64(seed))
    q_tx, q_rx = synth.trajectory(radar, M, jitter=0.01, rng=rng, offset=offset)
    tg = np.stack([rng.uniform(-0.8, 0.8, 4), rng.uniform(2.0, 4.0, 4)], 1)
    tg = tg + np.asarray(offset)
    am = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    g = synth.Grid(x0=-1.0 + offset[0], y0=1.8 + offset[1], dx=0.07, dy=0.07,
                   nx=30, ny=33)
    return radar, q_tx, q_rx, tg, am, g


def pin_linearity(lib):
    """P(s1 + s2) = P(s1) + P(s2) (range compression and BP are linear)."""
    radar, q_tx, q_rx, tg, am, g = _small_case(lib)
    b1 = synth.beat_signal(radar, q_tx, q_rx, tg[:2], am[:2])
    b2 = synth.beat_signal(radar, q_tx, q_rx, tg[2:], am[2:])
    w = np.hanning(radar.n_samples)
    wa = np.hanning(len(q_tx))

    def img(b):
        S = oracle.range_compress(b, w, radar.os, lib=lib)
        return oracle.backproject(radar, S, q_tx, q_rx, g.pixels(), w_az=wa, lib=lib)

    assert rel_l2(img(b1) + img(b2), img(b1 + b2)) < 1e-12


def pin_alg1_equals_alg2(lib):
    """Alg. 1 without velocity (vector window) and Alg. 2 without Doppler give
    the same image: the paper's mathematical optimisation changes nothing
    (Table II row 3, Delta SNR 0)."""
    radar, q_tx, q_rx, tg, am, g = _small_case(lib)
    b = synth.beat_signal(radar, q_tx, q_rx, tg, am)
    S = oracle.range_compress(b, np.hanning(radar.n_samples), radar.os, lib=lib)
    wa = np.hanning(len(q_tx))
    i1 = oracle.backproject_alg1(radar, S, q_tx, q_rx, g.pixels(), w_az=wa, lib=lib)
    i2 = oracle.backproject(radar, S, q_tx, q_rx, g.pixels(), w_az=wa, lib=lib)
    assert rel_l2(i1, i2) < 1e-10


def pin_alg1_doppler_sign(lib):
    """Alg. 1's velocity term against a simulator with intra-chirp motion.

    The antennas move at v_p during each chirp, so the delay to a target ahead
    of the track shrinks within the chirp and the beat tone is shifted by the
    Doppler frequency f0 d(tau)/dt (about one native range bin here).  Alg. 1
    with v(m) = -v_p (the scene's velocity relative to the radar) puts every
    term back on its range bin: over a scan of v = -s v_p the focus at the true
    target is sharpest at s = 1, where it equals the stop-and-hop focus of the
    same scene without motion, and its phase is arg(a).  With the opposite
    sign the term lands two bins off, near the Hann main-lobe null."""
    radar = _radar(n_rx=2, os=4)
    M, speed = 32, 20.0
    q_tx, q_rx = synth.trajectory(radar, M, speed=speed)
    v_p = np.array([speed, 0.0])
    tgt = np.array([[6.0, 2.0]])
    a = np.array([1.3 * np.exp(-1.1j)])
    w_r = oracle.window(oracle.WINDOW_HANN, radar.n_samples, lib=lib)
    moving = synth.beat_signal(radar, q_tx, q_rx, tgt, a, intra_chirp_velocity=v_p)
    still = synth.beat_signal(radar, q_tx, q_rx, tgt, a)
    S = oracle.range_compress(moving, w_r, radar.os, lib=lib)
    S0 = oracle.range_compress(still, w_r, radar.os, lib=lib)
    scale = np.linspace(-2.0, 2.0, 41)
    P = np.array([oracle.backproject_alg1(radar, S, q_tx, q_rx, tgt,
                                          vel=np.tile(-s * v_p, (M, 1)), lib=lib)[0]
                  for s in scale])
    P0 = oracle.backproject_alg1(radar, S0, q_tx, q_rx, tgt, lib=lib)[0]
    best = int(np.argmax(np.abs(P)))
    assert abs(scale[best] - 1.0) < 1e-9, scale[best]
    i0, i1, im1 = (int(np.argmin(np.abs(scale - v))) for v in (0.0, 1.0, -1.0))
    assert abs(abs(P[i1]) / abs(P0) - 1.0) < 2e-3, (abs(P[i1]), abs(P0))
    assert abs(np.angle(P[i1] / a[0])) < 0.05
    assert abs(P[i0]) < 0.7 * abs(P[i1])
    assert abs(P[im1]) < 0.1 * abs(P[i1])


def pin_rx_halving(lib):
    """Halving the Rx count halves a calibrated point target's peak
    (-6.02 dB, Sec. III-F)."""
    radar = _radar(n_rx=4)
    M = 24
    tgt = (0.2, 3.3)
    q_tx, q_rx, beat = _point_scene(radar, M, tgt, 1.0)
    N = radar.n_samples
    p4 = oracle.matched_filter(radar, beat, np.ones(N), q_tx, q_rx, np.array([tgt]),
                               lib=lib)[0]
    p2 = oracle.matched_filter(radar, beat[:, :2], np.ones(N), q_tx, q_rx[:, :2],
                               np.array([tgt]), lib=lib)[0]
    assert abs(abs(p2) / abs(p4) - 0.5) < 1e-9
    S = oracle.range_compress(beat, np.ones(N), radar.os, lib=lib)
    b4 = oracle.backproject(radar, S, q_tx, q_rx, np.array([tgt]), lib=lib)[0]
    b2 = oracle.backproject(radar, S[:, :2], q_tx, q_rx[:, :2], np.array([tgt]),
                            lib=lib)[0]
    assert abs(abs(b2) / abs(b4) - 0.5) < 0.02


def pin_single_term(lib):
    """One pixel, one chirp, one Rx, hand-computed.

    c = 4, f0 = 1/6, slope / fs = 0.4375, N_fft = 16:
      a1 = slope N_fft / (c fs) = 0.4375 * 16 / 4 = 1.75 bins per metre.
    Tx and Rx at the origin, pixel at (0, 3): d_hyp = 6 m, f_ind = 10.5,
    i0 = 10, f = 0.5, v = (S[10] + S[11]) / 2 = ((2+1j) + (4-1j)) / 2 = 3;
    s_hyp = exp(j 2 pi f0 d / c) = exp(j pi / 2) = j;  w_sar = 0.5
      => P = 1.5 j  (conjugate convention: -1.5 j).
    Base bin outside the crop range contributes nothing.
    """
    radar = synth.Radar(f0=1.0 / 6.0, bandwidth=0.4375 * 8.0, t_chirp=1.0,
                        n_samples=8, n_rx=1, os=2, c=4.0)
    assert abs(radar.slope / radar.fs - 0.4375) < 1e-15
    S = np.zeros((1, 1, 16), np.complex128)
    S[0, 0, 10] = 2 + 1j
    S[0, 0, 11] = 4 - 1j
    q = np.zeros((1, 2))
    qr = np.zeros((1, 1, 2))
    px = np.array([[0.0, 3.0]])
    P = oracle.backproject(radar, S, q, qr, px, w_az=np.array([0.5]), lib=lib)[0]
    assert abs(P - 1.5j) < 1e-12, P
    Pm = oracle.backproject(radar, S, q, qr, px, w_az=np.array([0.5]), sign=-1,
                            lib=lib)[0]
    assert abs(Pm + 1.5j) < 1e-12, Pm
    P1 = oracle.backproject_alg1(radar, S, q, qr, px, w_az=np.array([0.5]), lib=lib)[0]
    assert abs(P1 - 1.5j) < 1e-12, P1
    for crop in ((0, 10), (11, 15)):
        Pc = oracle.backproject(radar, S, q, qr, px, crop=crop, lib=lib)[0]
        assert Pc == 0, (crop, Pc)
    Pc = oracle.backproject(radar, S, q, qr, px, crop=(10, 11), lib=lib)[0]
    assert abs(Pc - 3j) < 1e-12


def pin_subaperture_additivity(lib):
    """BP over [0, M) = BP over [0, k) + BP over [k, M)."""
    radar, q_tx, q_rx, tg, am, g = _small_case(lib, M=21)
    b = synth.beat_signal(radar, q_tx, q_rx, tg, am)
    S = oracle.range_compress(b, np.hanning(radar.n_samples), radar.os, lib=lib)
    wa = np.hanning(len(q_tx))
    full = oracle.backproject(radar, S, q_tx, q_rx, g.pixels(), w_az=wa, lib=lib)
    k = 8
    a = oracle.backproject(radar, S[:k], q_tx[:k], q_rx[:k], g.pixels(), w_az=wa[:k],
                           lib=lib)
    b_ = oracle.backproject(radar, S[k:], q_tx[k:], q_rx[k:], g.pixels(), w_az=wa[k:],
                            lib=lib)
    assert rel_l2(a + b_, full) < 1e-12


def pin_translation_invariance(lib):
    """Moving scene and trajectory by (1000 m, 1000 m) leaves the image
    unchanged (FP64 positions keep the 77 GHz phase)."""
    imgs = []
    for off in ((0.0, 0.0), (1000.0, 1000.0)):
        radar, q_tx, q_rx, tg, am, g = _small_case(lib, offset=off)
        b = synth.beat_signal(radar, q_tx, q_rx, tg, am)
        S = oracle.range_compress(b, np.hanning(radar.n_samples), radar.os, lib=lib)
        imgs.append(oracle.backproject(radar, S, q_tx, q_rx, g.pixels(), lib=lib))
    assert rel_l2(imgs[1], imgs[0]) < 1e-6


def pin_bp_matches_matched_filter(lib):
    """On a multi-target scene the oracle image is within the os = 16
    interpolation error of the brute-force matched filter."""
    radar, q_tx, q_rx, tg, am, g = _small_case(lib)
    radar = _radar(n_rx=2, os=16)
    b = synth.beat_signal(radar, q_tx, q_rx, tg, am)
    w = np.hanning(radar.n_samples)
    wa = np.hanning(len(q_tx))
    ref = oracle.matched_filter(radar, b, w, q_tx, q_rx, g.pixels(), w_az=wa, lib=lib)
    S = oracle.range_compress(b, w, radar.os, lib=lib)
    img = oracle.backproject(radar, S, q_tx, q_rx, g.pixels(), w_az=wa, lib=lib)
    assert rel_l2(img, ref) < 5e-3


# --------------------------------------------------------------------------
# polar reconstruction grid (Sec. III-E) and Doppler offsets (Sec. III-D)
# --------------------------------------------------------------------------
def _table1_radar(**kw):
    """Table I: f0 76.6 GHz, B 931 MHz, T_P 102.4 us, PRI 106.7 us; fs 10 MHz."""
    base = dict(f0=76.6e9, bandwidth=931e6, t_chirp=102.4e-6, pri=106.7e-6,
                n_samples=1024, n_rx=1, os=4)
    base.update(kw)
    return synth.Radar(**base)


def _ring_counts(o, r, box, dphi):
    """Points of the angular lattice j dphi in [-pi, pi) on the circle of
    radius r about o that lie in the box, counted from the circle-box
    intersection (crossing angles of the four border lines), not by
    enumerating the lattice."""
    x0, x1, y0, y1 = box
    cuts = [-math.pi, math.pi]
    for xb in (x0, x1):
        c = (xb - o[0]) / r
        if abs(c) <= 1:
            a = math.acos(c)
            cuts += [a, -a]
    for yb in (y0, y1):
        sn = (yb - o[1]) / r
        if abs(sn) <= 1:
            a = math.asin(sn)
            cuts += [a, math.pi - a if a > 0 else -math.pi - a]
    cuts = sorted(min(max(c, -math.pi), math.pi) for c in cuts)
    n = 0
    for a, b in zip(cuts[:-1], cuts[1:]):
        if b - a < 1e-15:
            continue
        m = 0.5 * (a + b)
        x, y = o[0] + r * math.cos(m), o[1] + r * math.sin(m)
        if x0 <= x <= x1 and y0 <= y <= y1:
            jlo = max(math.ceil(a / dphi), math.ceil(-math.pi / dphi))
            jhi = min(math.floor(b / dphi), math.ceil(math.pi / dphi) - 1)
            n += max(0, jhi - jlo + 1)
    return n


def _polar_setup(speed=8.0, M=1024):
    radar = _table1_radar()
    q_tx, _ = synth.trajectory(radar, M, speed=speed)
    o = 0.5 * (q_tx[0] + q_tx[-1])
    L = float(np.hypot(*(q_tx[-1] - q_tx[0])))
    lam = C0 / (radar.f0 + radar.bandwidth / 2.0)
    dr = C0 / (2.0 * radar.bandwidth) / 2.5
    dphi = lam / (2.0 * L) / 2.5
    return radar, q_tx, o, L, dr, dphi


def pin_polar_grid_lattice(lib):
    """Every point sits on the lattice (k dr, j dphi) about the aperture centre
    with dr = c / (2 B) / 2.5 and dphi = lambda / (2 L) / 2.5 (Table I: 6.44 cm),
    inside the box, once, ring by ring with ascending angle; and per ring the
    count equals the number of lattice angles inside the circle-box
    intersection computed from the crossing angles."""
    radar, q_tx, o, L, dr, dphi = _polar_setup()
    assert abs(dr - 0.0644022) < 1e-7
    box = (-3.31, 2.93, 1.07, 6.13)
    g = oracle.polar_grid(radar, q_tx, box, 2.5, lib=lib)
    assert len(g) > 1000
    assert np.all((g[:, 0] >= box[0]) & (g[:, 0] <= box[1]) & (g[:, 1] >= box[2]) & (g[:, 1] <= box[3]))
    e = g - o
    k = np.hypot(e[:, 0], e[:, 1]) / dr
    j = np.arctan2(e[:, 1], e[:, 0]) / dphi
    assert np.max(np.abs(k - np.rint(k))) < 1e-9
    assert np.max(np.abs(j - np.rint(j))) < 1e-6
    ki, ji = np.rint(k).astype(np.int64), np.rint(j).astype(np.int64)
    assert ki.min() >= 1
    key = ki * 10 ** 7 + ji
    assert np.all(np.diff(key) > 0)  # unique, rings ascending, angles ascending
    for kk in range(1, int(ki.max()) + 2):
        assert int(np.sum(ki == kk)) == _ring_counts(o, kk * dr, box, dphi), kk


def pin_polar_grid_spacing(lib):
    """Neighbours on a ring are lambda r / (2 L) / 2.5 apart (chord 2 r sin(dphi/2))
    and neighbouring rings dr apart: the textbook range and azimuth
    resolutions divided by the factor; a factor of 5 doubles the density
    along both axes (4x the points)."""
    radar, q_tx, o, L, dr, dphi = _polar_setup(speed=9.0)
    box = (-1.5, 1.5, 4.0, 7.0)
    g = oracle.polar_grid(radar, q_tx, box, 2.5, lib=lib)
    e = g - o
    r = np.hypot(e[:, 0], e[:, 1])
    ring = np.rint(r / dr).astype(np.int64)
    kk = int(np.median(ring))
    pts = g[ring == kk]
    d = np.hypot(*np.diff(pts, axis=0).T)
    lam = C0 / (radar.f0 + radar.bandwidth / 2.0)
    az = lam * (kk * dr) / (2.0 * L) / 2.5
    assert np.allclose(d, 2 * kk * dr * math.sin(dphi / 2), rtol=1e-9)
    assert abs(np.median(d) / az - 1.0) < 1e-4
    g5 = oracle.polar_grid(radar, q_tx, box, 5.0, lib=lib)
    assert abs(len(g5) / len(g) - 4.0) < 0.05


def pin_polar_grid_point_target(lib):
    """A point target on a grid point images to its peak exactly there; one
    between grid points peaks at one of the four lattice points around it."""
    radar = _radar(n_samples=128, n_rx=2, os=4)
    M = 96
    q_tx, q_rx = synth.trajectory(radar, M)
    box = (-0.45, 0.52, 3.61, 4.33)
    g = oracle.polar_grid(radar, q_tx, box, 2.5, lib=lib)
    o = 0.5 * (q_tx[0] + q_tx[-1])
    L = float(np.hypot(*(q_tx[-1] - q_tx[0])))
    dr = C0 / (2.0 * radar.bandwidth) / 2.5
    dphi = C0 / (radar.f0 + radar.bandwidth / 2.0) / (2.0 * L) / 2.5
    w_r = oracle.window(oracle.WINDOW_HANN, radar.n_samples, lib=lib)
    wa = np.hanning(M)
    on = g[int(np.argmin(np.hypot(g[:, 0] - 0.03, g[:, 1] - 3.97)))]
    r0, p0 = math.hypot(*(on - o)), math.atan2(*(on - o)[::-1])
    off = o + (r0 + 0.43 * dr) * np.array([math.cos(p0 + 0.61 * dphi), math.sin(p0 + 0.61 * dphi)])
    for tgt, on_grid in ((on, True), (off, False)):
        beat = synth.beat_signal(radar, q_tx, q_rx, tgt[None, :], np.array([1.0 + 0.2j]))
        S = oracle.range_compress(beat, w_r, radar.os, lib=lib)
        img = oracle.backproject(radar, S, q_tx, q_rx, g, w_az=wa, lib=lib)
        best = g[int(np.argmax(np.abs(img)))]
        if on_grid:
            assert np.allclose(best, tgt, atol=1e-12)
        else:
            e = best - o
            kb, jb = math.hypot(*e) / dr, math.atan2(e[1], e[0]) / dphi
            kt, jt = (r0 + 0.43 * dr) / dr, (p0 + 0.61 * dphi) / dphi
            assert round(kb) in (math.floor(kt), math.ceil(kt)), (kb, kt)
            assert round(jb) in (math.floor(jt), math.ceil(jt)), (jb, jt)


def pin_doppler_offsets_closed_form(lib):
    """Track along +x at speed v: a pixel ahead on the track axis closes at
    2 v, f_doppler = -2 f0 v / c * N_fft / fs bins; one behind opens at 2 v;
    one abeam of the mean Tx position sees only the Rx offset's share,
    f0 v dx / (c r) * N_fft / fs with dx the mean Rx offset along x."""
    radar = _radar(n_samples=256, n_rx=3, os=4)
    M, v = 65, 12.0
    q_tx, q_rx = synth.trajectory(radar, M, speed=v)
    vel = np.tile([v, 0.0], (M, 1))
    px = np.array([[40.0, 0.0], [-40.0, 0.0], [0.0, 7.0]])
    fd = oracle.doppler_offsets(radar, q_tx, q_rx, vel, px, lib=lib)
    scale = radar.f0 / C0 * radar.n_fft / radar.fs
    assert abs(fd[0] - (-2 * v * scale)) < 1e-9 * abs(fd[0])
    assert abs(fd[1] - (2 * v * scale)) < 1e-9 * abs(fd[1])
    dx = float(np.mean(q_rx[..., 0]) - np.mean(q_tx[:, 0]))
    gx = -dx
    ref = -(v * gx / math.hypot(gx, 7.0)) * scale
    assert abs(fd[2] - ref) < 1e-9 * abs(ref)


def pin_doppler_offsets_finite_difference(lib):
    """The offset equals f0 / c times the rate of change of the two-way path
    to the aperture's middle chirp, taken as a central difference of the
    per-chirp distances (positions only, no velocity input) over one PRI, for
    a straight constant-velocity track with an odd chirp count."""
    radar = _radar(n_samples=128, n_rx=4, os=4)
    M, v = 81, 9.5
    q_tx, q_rx = synth.trajectory(radar, M, speed=v)
    vel = np.tile([v, 0.0], (M, 1))
    rng = np.random.Generator(np.random.PCG64(21))
    px = np.stack([rng.uniform(-6, 6, 50), rng.uniform(1, 12, 50)], 1)
    fd = oracle.doppler_offsets(radar, q_tx, q_rx, vel, px, lib=lib)
    mc = M // 2
    qr_mean = q_rx.mean(axis=1)

    def path(m):
        return np.hypot(*(px - q_tx[m]).T) + np.hypot(*(px - qr_mean[m]).T)

    ddot = (path(mc + 1) - path(mc - 1)) / (2 * radar.pri)
    ref = radar.f0 * ddot / C0 * radar.n_fft / radar.fs
    assert np.max(np.abs(fd - ref)) < 1e-6 * np.max(np.abs(ref))


def pin_doppler_offsets_refocus(lib):
    """With the antennas moving during each chirp (intra-chirp motion, 20 m/s),
    Alg. 2 with these per-pixel offsets focuses each target as the same scene
    without motion does (|P| within 0.5 %); without offsets the focus drops
    below 70 %, with reversed offsets below 15 %."""
    radar = _radar(n_samples=128, n_rx=2, os=4)
    M, v_p = 96, np.array([20.0, 0.0])
    q_tx, q_rx = synth.trajectory(radar, M, speed=float(v_p[0]))
    tg = np.array([[2.6, 1.5], [4.0, 2.5], [5.0, 3.75]])
    am = np.array([1.0, 0.7 * np.exp(1j), 1.2j])
    w_r = oracle.window(oracle.WINDOW_HANN, radar.n_samples, lib=lib)
    wa = np.hanning(M)
    moving = synth.beat_signal(radar, q_tx, q_rx, tg, am, intra_chirp_velocity=v_p)
    still = synth.beat_signal(radar, q_tx, q_rx, tg, am)
    S = oracle.range_compress(moving, w_r, radar.os, lib=lib)
    S0 = oracle.range_compress(still, w_r, radar.os, lib=lib)
    fd = oracle.doppler_offsets(radar, q_tx, q_rx, np.tile(v_p, (M, 1)), tg, lib=lib)
    assert np.all(np.abs(fd) > 1.0)
    focus = np.abs(oracle.backproject(radar, S0, q_tx, q_rx, tg, w_az=wa, lib=lib))
    for f, lo, hi in ((fd, 0.995, 1.005), (None, 0.0, 0.7), (-fd, 0.0, 0.15)):
        got = np.abs(oracle.backproject(radar, S, q_tx, q_rx, tg, w_az=wa, fd_idx=f, lib=lib))
        assert np.all((got / focus >= lo) & (got / focus <= hi)), (got / focus, lo, hi)


def pin_doppler_velocity_variation_below_100hz(lib):
    """Sec. III-D: the velocity may be taken as constant over a chirp sequence
    because its variation moves the Doppler frequency by well under 100 Hz.
    Table I sequence (1024 chirps, 109.3 ms) of a car at 10 m/s accelerating
    at 1 m/s^2: each chirp's own velocity moves every pixel's Doppler
    frequency by at most 2 f0 max|v(m) - vbar| / c = 28 Hz, attained for a
    pixel along the track."""
    radar = _table1_radar(n_rx=2)
    M = 1024
    q_tx, q_rx = synth.trajectory(radar, M, speed=10.0)
    t = (np.arange(M) - (M - 1) / 2) * radar.pri
    vel = np.stack([10.0 + 1.0 * t, np.zeros(M)], 1)
    rng = np.random.Generator(np.random.PCG64(4))
    px = np.concatenate([[[60.0, 0.0]], np.stack([rng.uniform(-15, 15, 40), rng.uniform(1, 31, 40)], 1)])
    hz = radar.fs / radar.n_fft
    mean = oracle.doppler_offsets(radar, q_tx, q_rx, vel, px, lib=lib)
    dev = 0.0
    for m in (0, M // 3, M - 1):
        per = oracle.doppler_offsets(radar, q_tx, q_rx, np.tile(vel[m], (M, 1)), px, lib=lib)
        dev = max(dev, float(np.max(np.abs(per - mean))) * hz)
    bound = 2 * radar.f0 * float(np.max(np.abs(vel[:, 0] - vel[:, 0].mean()))) / C0
    assert abs(bound - 28.0) < 0.5, bound
    assert abs(dev - bound) < 1e-6 * bound, (dev, bound)
    assert dev < 100.0


ALL_PINS = [
    pin_fft, pin_windows, pin_range_compress, pin_matched_filter_closed_form,
    pin_backproject_point_target, pin_time_origin_mid_bin, pin_interpolation_convergence,
    pin_resolution,
    pin_linearity, pin_alg1_equals_alg2, pin_alg1_doppler_sign, pin_rx_halving, pin_single_term,
    pin_subaperture_additivity, pin_translation_invariance,
    pin_bp_matches_matched_filter,
    pin_polar_grid_lattice, pin_polar_grid_spacing, pin_polar_grid_point_target,
    pin_doppler_offsets_closed_form, pin_doppler_offsets_finite_difference,
    pin_doppler_offsets_refocus, pin_doppler_velocity_variation_below_100hz,
]
