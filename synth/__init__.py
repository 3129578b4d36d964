"""Seeded synthetic inputs for automotive FMCW SAR imaging.

This module is the measurement side only: radar parameters, antenna
trajectories, point-scatterer scenes and the FMCW beat signal such a scene
produces.  It holds none of the imaging arithmetic (no range window, no range
transform, no interpolation, no backprojection).  The FP64 oracle and the CUDA
library both consume the arrays made here, so that parity tests compare the
two on identical inputs.

Radar model (paper Table I and Sec. II, plus readings where the paper is silent):

* FMCW chirp of slope ``mu = B / T_P`` starting at ``f0`` at sample 0;
  ``fs = N / T_P``.
* IQ beat signal taken as Rx times conj(Tx), stop-and-hop:
  ``s[m, r, n] = sum_k a_k exp(-j 2 pi (f0 tau + mu tau n / fs - rvp mu tau^2 / 2))``
  with ``tau = (|p_k - q_tx(m)| + |p_k - q_rx(m, r)|) / c``.
* One Tx, ``R`` Rx antennas on a line along the driving direction,
  Rx ``r`` at ``q_tx + (r + 1) lambda / 2`` (the paper gives no layout).
* 2-D geometry (the paper's distances are 2-D).

Everything random is drawn from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

C0 = 299_792_458.0


@dataclasses.dataclass(frozen=True)
class Radar:
    """FMCW radar and processing parameters (SI units)."""

    f0: float = 77e9          # frequency at sample 0 of each chirp (Hz)
    bandwidth: float = 1e9    # B (Hz)
    t_chirp: float = 102.4e-6  # T_P (s)
    pri: float = 106.7e-6     # T_P0 (s)
    n_samples: int = 256      # N
    n_rx: int = 1             # R
    os: int = 4               # zero-padding factor of the range transform
    c: float = C0

    @property
    def slope(self) -> float:
        return self.bandwidth / self.t_chirp

    @property
    def fs(self) -> float:
        return self.n_samples / self.t_chirp

    @property
    def n_fft(self) -> int:
        return self.n_samples * self.os

    @property
    def wavelength(self) -> float:
        return self.c / self.f0

    @property
    def bins_per_metre(self) -> float:
        """Range-transform bins per metre of two-way path."""
        return self.slope * self.n_fft / (self.c * self.fs)


@dataclasses.dataclass(frozen=True)
class Grid:
    """Cartesian image grid; pixel (ix, iy) sits at (x0 + ix dx, y0 + iy dy)."""

    x0: float
    y0: float
    dx: float
    dy: float
    nx: int
    ny: int

    def pixels(self) -> np.ndarray:
        """[ny*nx, 2] FP64 pixel centres, x fastest."""
        xs = self.x0 + self.dx * np.arange(self.nx)
        ys = self.y0 + self.dy * np.arange(self.ny)
        gx, gy = np.meshgrid(xs, ys)
        return np.stack([gx.ravel(), gy.ravel()], axis=1)


@dataclasses.dataclass
class Workload:
    name: str
    radar: Radar
    n_pulses: int
    grid: Grid
    q_tx: np.ndarray          # [M, 2] float64
    q_rx: np.ndarray          # [M, R, 2] float64
    targets: np.ndarray       # [K, 2] float64
    amps: np.ndarray          # [K] complex128
    snr_db: Optional[float]
    seed: int
    crop: tuple               # (crop_lo, crop_hi) entry range of the range profiles


def centred_grid(nx: int, ny: int, spacing: float, y_start: float) -> Grid:
    x0 = -spacing * (nx - 1) / 2.0
    return Grid(x0=x0, y0=y_start, dx=spacing, dy=spacing, nx=nx, ny=ny)


def trajectory(radar: Radar, n_pulses: int, speed: float = 10.0,
               jitter: float = 0.0, jitter_periods: float = 3.0,
               rng: Optional[np.random.Generator] = None,
               offset=(0.0, 0.0)):
    """Linear track along +x, centred on x = 0, at the chirp starts m * PRI.

    ``jitter`` adds a sinusoidal lateral (y) deviation of that amplitude with
    ``jitter_periods`` periods over the aperture and a seeded phase.
    Returns (q_tx [M, 2], q_rx [M, R, 2]) in FP64.
    """
    m = np.arange(n_pulses, dtype=np.float64)
    step = speed * radar.pri
    x = (m - (n_pulses - 1) / 2.0) * step
    y = np.zeros_like(x)
    if jitter:
        phase = (rng.uniform(0.0, 2 * np.pi) if rng is not None else 0.0)
        y = jitter * np.sin(2 * np.pi * jitter_periods * m / n_pulses + phase)
    q_tx = np.stack([x + offset[0], y + offset[1]], axis=1)
    spacing = radar.wavelength / 2.0
    rx_off = (np.arange(radar.n_rx, dtype=np.float64) + 1.0) * spacing
    q_rx = np.empty((n_pulses, radar.n_rx, 2))
    q_rx[:, :, 0] = q_tx[:, None, 0] + rx_off[None, :]
    q_rx[:, :, 1] = q_tx[:, None, 1]
    return q_tx, q_rx


def _spread_points(rng, n, lo, hi, min_sep, max_tries=100000):
    pts = []
    tries = 0
    while len(pts) < n and tries < max_tries:
        tries += 1
        p = rng.uniform(lo, hi)
        if all(np.hypot(*(p - q)) >= min_sep for q in pts):
            pts.append(p)
    if len(pts) < n:
        raise RuntimeError("could not place scatterers")
    return np.array(pts)


def crop_for(radar: Radar, grid: Grid, q_tx: np.ndarray, q_rx: np.ndarray,
             margin_bins: int = 8):
    """Entry range [lo, hi) of the range profiles that covers every
    (pixel, pulse, Rx) of this geometry, plus a margin.  Bounded by the
    valid entry range [0, N_fft - 1)."""
    xs = np.array([grid.x0, grid.x0 + grid.dx * (grid.nx - 1)])
    ys = np.array([grid.y0, grid.y0 + grid.dy * (grid.ny - 1)])
    ants = np.concatenate([q_tx[:, None, :], q_rx], axis=1).reshape(-1, 2)
    ax_lo, ax_hi = ants[:, 0].min(), ants[:, 0].max()
    ay_lo, ay_hi = ants[:, 1].min(), ants[:, 1].max()
    # distance bounds between the pixel box and the antenna box
    gapx = max(0.0, max(xs.min() - ax_hi, ax_lo - xs.max()))
    gapy = max(0.0, max(ys.min() - ay_hi, ay_lo - ys.max()))
    dmin = math.hypot(gapx, gapy)
    farx = max(abs(xs.max() - ax_lo), abs(ax_hi - xs.min()))
    fary = max(abs(ys.max() - ay_lo), abs(ay_hi - ys.min()))
    dmax = math.hypot(farx, fary)
    a1 = radar.bins_per_metre
    lo = max(0, int(math.floor(a1 * 2 * dmin)) - margin_bins)
    hi = min(radar.n_fft - 1, int(math.ceil(a1 * 2 * dmax)) + margin_bins)
    return lo, hi


def make_workload(name: str, seed: int = 0) -> Workload:
    """The named synthetic workloads.

    tiny      : 1 Rx, 256 chirps x 256 samples, 128^2 px at 5 cm, 5 scatterers
                (CN(0,1) amplitudes, at pixel centres, >= 10 range cells apart),
                20 dB AWGN, Hann windows.
    full      : 4 Rx, 1024 chirps x 512 samples, +-2 cm sinusoidal lateral
                jitter, 512^2 px at 2.5 cm, 200 Rayleigh scatterers plus 20000
                clutter scatterers at -30 dB.
    precision : 4 Rx, 2048 chirps x 1024 samples, 1024^2 px at 2 cm,
                1000 scatterers at ranges 2-50 m.
    small     : a quick multi-tile case (2 Rx, 96 chirps x 128 samples,
                80 x 72 px) used by fast tests.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if name == "tiny":
        radar = Radar(n_samples=256, n_rx=1, os=4)
        M = 256
        grid = centred_grid(128, 128, 0.05, 2.0)
        q_tx, q_rx = trajectory(radar, M)
        pix = grid.pixels()
        res = C0 / (2 * radar.bandwidth)
        inner = np.array([[grid.x0 + 10 * grid.dx, grid.y0 + 10 * grid.dy]])
        outer = np.array([[grid.x0 + (grid.nx - 11) * grid.dx,
                           grid.y0 + (grid.ny - 11) * grid.dy]])
        pts = _spread_points(rng, 5, inner[0], outer[0], 10 * res)
        ix = np.rint((pts[:, 0] - grid.x0) / grid.dx)
        iy = np.rint((pts[:, 1] - grid.y0) / grid.dy)
        targets = np.stack([grid.x0 + ix * grid.dx, grid.y0 + iy * grid.dy], 1)
        amps = (rng.standard_normal(5) + 1j * rng.standard_normal(5)) / np.sqrt(2)
        snr = 20.0
        del pix
    elif name == "full":
        radar = Radar(n_samples=512, n_rx=4, os=4)
        M = 1024
        grid = centred_grid(512, 512, 0.025, 2.0)
        q_tx, q_rx = trajectory(radar, M, jitter=0.02, rng=rng)
        xlo, xhi = grid.x0, grid.x0 + grid.dx * (grid.nx - 1)
        ylo, yhi = grid.y0, grid.y0 + grid.dy * (grid.ny - 1)
        n_t, n_c = 200, 20000
        tp = np.stack([rng.uniform(xlo, xhi, n_t), rng.uniform(ylo, yhi, n_t)], 1)
        ta = rng.rayleigh(1.0, n_t) * np.exp(1j * rng.uniform(0, 2 * np.pi, n_t))
        cp = np.stack([rng.uniform(xlo, xhi, n_c), rng.uniform(ylo, yhi, n_c)], 1)
        ca = (10 ** (-30 / 20)) * (rng.standard_normal(n_c)
                                   + 1j * rng.standard_normal(n_c)) / np.sqrt(2)
        targets = np.concatenate([tp, cp])
        amps = np.concatenate([ta, ca])
        snr = 20.0
    elif name == "precision":
        radar = Radar(n_samples=1024, n_rx=4, os=4)
        M = 2048
        grid = centred_grid(1024, 1024, 0.02, 2.0)
        q_tx, q_rx = trajectory(radar, M, jitter=0.02, rng=rng)
        n_t = 1000
        rr = rng.uniform(2.0, 50.0, n_t)
        th = rng.uniform(np.deg2rad(-60), np.deg2rad(60), n_t)
        targets = np.stack([rr * np.sin(th), rr * np.cos(th)], 1)
        amps = rng.rayleigh(1.0, n_t) * np.exp(1j * rng.uniform(0, 2 * np.pi, n_t))
        snr = 20.0
    elif name == "small":
        radar = Radar(n_samples=128, n_rx=2, os=4)
        M = 96
        grid = Grid(x0=-1.8, y0=1.5, dx=0.05, dy=0.05, nx=80, ny=72)
        q_tx, q_rx = trajectory(radar, M, jitter=0.01, rng=rng)
        n_t = 12
        targets = np.stack([rng.uniform(-1.6, 1.9, n_t), rng.uniform(1.7, 4.9, n_t)], 1)
        amps = (rng.standard_normal(n_t) + 1j * rng.standard_normal(n_t)) / np.sqrt(2)
        snr = 20.0
    else:
        raise KeyError(name)
    crop = crop_for(radar, grid, q_tx, q_rx)
    return Workload(name=name, radar=radar, n_pulses=M, grid=grid, q_tx=q_tx,
                    q_rx=q_rx, targets=targets, amps=amps, snr_db=snr, seed=seed,
                    crop=crop)


def beat_signal(radar: Radar, q_tx: np.ndarray, q_rx: np.ndarray,
                targets: np.ndarray, amps: np.ndarray, rvp: bool = False,
                snr_db: Optional[float] = None, seed: int = 0,
                device: Optional[str] = None, chunk: int = 64,
                intra_chirp_velocity: Optional[np.ndarray] = None) -> np.ndarray:
    """Stop-and-hop FMCW beat cube [M, R, N] (complex128, numpy).

    ``device`` = None computes with numpy on the CPU; a torch device string
    ("cuda") computes the same FP64 formula with torch (for large scenes).
    AWGN (if ``snr_db``) is per-sample, relative to the mean power of the
    noiseless cube, drawn from PCG64(seed + 1).

    ``intra_chirp_velocity`` ([2] or [M, 2], m/s; numpy path only) drops the
    stop-and-hop assumption: during chirp m every antenna moves from its
    chirp-start position at that velocity, so the delay is re-evaluated at
    every sample, ``tau(t) = (|p - q_tx - v t| + |p - q_rx - v t|) / c``, and
    the phase is ``f0 tau(t) + mu tau(t) t``.  Its rate of change is the
    Doppler shift that Alg. 1's velocity term compensates.
    """
    M = q_tx.shape[0]
    R = q_rx.shape[1]
    N = radar.n_samples
    t = np.arange(N, dtype=np.float64) / radar.fs
    if intra_chirp_velocity is not None:
        if device is not None:
            raise ValueError("intra_chirp_velocity is computed on the numpy path only")
        v = np.broadcast_to(np.asarray(intra_chirp_velocity, dtype=np.float64), (M, 2))
        out = np.zeros((M, R, N), dtype=np.complex128)
        for k, (p, a) in enumerate(zip(targets, amps)):
            # antenna positions at every sample: [M, N, 2] and [M, R, N, 2]
            tx = q_tx[:, None, :] + v[:, None, :] * t[None, :, None]
            rx = q_rx[:, :, None, :] + v[:, None, None, :] * t[None, None, :, None]
            dtx = np.hypot(p[0] - tx[..., 0], p[1] - tx[..., 1])             # [M, N]
            drx = np.hypot(p[0] - rx[..., 0], p[1] - rx[..., 1])             # [M, R, N]
            tau = (dtx[:, None, :] + drx) / radar.c                          # [M, R, N]
            ph = radar.f0 * tau
            if rvp:
                ph = ph - 0.5 * radar.slope * tau * tau
            ph = ph - np.floor(ph) + radar.slope * tau * t
            out += a * np.exp(-2j * np.pi * ph)
    elif device is None:
        out = np.zeros((M, R, N), dtype=np.complex128)
        for k0 in range(0, len(targets), chunk):
            tk = targets[k0:k0 + chunk]
            ak = amps[k0:k0 + chunk]
            dtx = np.hypot(tk[None, :, 0] - q_tx[:, None, 0],
                           tk[None, :, 1] - q_tx[:, None, 1])          # [M, K]
            drx = np.hypot(tk[None, None, :, 0] - q_rx[:, :, None, 0],
                           tk[None, None, :, 1] - q_rx[:, :, None, 1])  # [M, R, K]
            tau = (dtx[:, None, :] + drx) / radar.c                   # [M, R, K]
            ph0 = radar.f0 * tau
            if rvp:
                ph0 = ph0 - 0.5 * radar.slope * tau * tau
            # cycles of the constant part reduced before the exponential
            ph0 = ph0 - np.floor(ph0)
            for n0 in range(0, N, 256):
                tn = t[n0:n0 + 256]
                ph = ph0[..., None] + radar.slope * tau[..., None] * tn  # [M,R,K,n]
                out[:, :, n0:n0 + 256] += np.einsum(
                    "k,mrkn->mrn", ak, np.exp(-2j * np.pi * ph))
    else:
        import torch
        dev = torch.device(device)
        f64 = torch.float64
        qt = torch.as_tensor(q_tx, dtype=f64, device=dev)
        qr = torch.as_tensor(q_rx, dtype=f64, device=dev)
        tt = torch.as_tensor(t, dtype=f64, device=dev)
        acc = torch.zeros((M, R, N), dtype=torch.complex128, device=dev)
        chunk = max(1, min(256, int(4e8 // (M * R * N))))
        for k0 in range(0, len(targets), chunk):
            tk = torch.as_tensor(targets[k0:k0 + chunk], dtype=f64, device=dev)
            ak = torch.as_tensor(amps[k0:k0 + chunk], dtype=torch.complex128, device=dev)
            dtx = torch.hypot(tk[None, :, 0] - qt[:, None, 0], tk[None, :, 1] - qt[:, None, 1])
            drx = torch.hypot(tk[None, None, :, 0] - qr[:, :, None, 0],
                              tk[None, None, :, 1] - qr[:, :, None, 1])
            tau = (dtx[:, None, :] + drx) / radar.c
            ph0 = radar.f0 * tau
            if rvp:
                ph0 = ph0 - 0.5 * radar.slope * tau * tau
            ph0 = ph0 - torch.floor(ph0)
            ph = ph0[..., None] + radar.slope * tau[..., None] * tt   # [M,R,K,N]
            ang = -2.0 * math.pi * ph
            z = torch.polar(torch.ones_like(ang), ang)
            acc += torch.einsum("k,mrkn->mrn", ak, z)
        out = acc.cpu().numpy()
    if snr_db is not None:
        p_sig = float(np.mean(np.abs(out) ** 2))
        if p_sig > 0:
            rng = np.random.Generator(np.random.PCG64(seed + 1))
            sigma = math.sqrt(p_sig * 10 ** (-snr_db / 10) / 2)
            out = out + sigma * (rng.standard_normal(out.shape)
                                 + 1j * rng.standard_normal(out.shape))
    return out


def workload_beat(wl: Workload, device: Optional[str] = None) -> np.ndarray:
    """The workload's beat cube rounded to complex64 (the library's input type)."""
    b = beat_signal(wl.radar, wl.q_tx, wl.q_rx, wl.targets, wl.amps,
                    snr_db=wl.snr_db, seed=wl.seed, device=device)
    return b.astype(np.complex64)


def azimuth_weights(n_pulses: int, kind: str = "hann") -> np.ndarray:
    """Per-chirp weights w_sar[m] (an input of the backprojection, paper
    Sec. III-B): numpy's symmetric Hann window, or all ones ("rect")."""
    if kind == "rect":
        return np.ones(n_pulses)
    return np.hanning(n_pulses) if n_pulses > 1 else np.ones(1)


def make_batched_requests(n: int = 64, seed: int = 0, n_targets: int = 20,
                          m_range=(128, 1024), side_range=(128, 768), rx_range=(1, 4),
                          n_samples: int = 512):
    """Uneven sub-aperture requests for the batched form: seeded pulse counts,
    square image sides (multiples of 16 px at 2.5 cm from y = 2 m), Rx counts,
    trajectories (+-2 cm jitter) and point-scatterer scenes (Rayleigh
    amplitudes, 20 dB AWGN).  Returns a list of Workload."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        side = int(rng.integers(side_range[0] // 16, side_range[1] // 16 + 1)) * 16
        R = int(rng.integers(rx_range[0], rx_range[1] + 1))
        radar = Radar(n_samples=n_samples, n_rx=R, os=4)
        grid = centred_grid(side, side, 0.025, 2.0)
        q_tx, q_rx = trajectory(radar, M, jitter=0.02, rng=rng)
        xlo, xhi = grid.x0, grid.x0 + grid.dx * (grid.nx - 1)
        ylo, yhi = grid.y0, grid.y0 + grid.dy * (grid.ny - 1)
        tg = np.stack([rng.uniform(xlo, xhi, n_targets), rng.uniform(ylo, yhi, n_targets)], 1)
        am = rng.rayleigh(1.0, n_targets) * np.exp(1j * rng.uniform(0, 2 * np.pi, n_targets))
        out.append(Workload(name=f"batch{i}", radar=radar, n_pulses=M, grid=grid, q_tx=q_tx,
                            q_rx=q_rx, targets=tg, amps=am, snr_db=20.0, seed=seed * 1000 + i,
                            crop=crop_for(radar, grid, q_tx, q_rx)))
    return out
