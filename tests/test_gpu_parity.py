"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs."""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.gpu_helpers import (TOL_FP16, TOL_FP32, beta_of, check_peaks, gpu_image, make_plan,
                               nearest_pixel, oracle_image, peak_windows, rel_l2, rotation,
                               to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    import paper_2306_09784_gb300 as sar
    sar.load_library()  # fails loudly when the library is missing
    return t


@pytest.fixture(scope="module")
def small():
    wl = synth.make_workload("small")
    return wl, synth.workload_beat(wl), np.hanning(wl.n_pulses)


@pytest.fixture(scope="module")
def tiny():
    wl = synth.make_workload("tiny")
    return wl, synth.workload_beat(wl), np.hanning(wl.n_pulses)


# ----------------------------------------------------------------------------
# range compression
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("os_factor,N", [(4, 128), (1, 64), (16, 64), (4, 4096), (2, 64)])
def test_range_spectrum_vs_oracle(torch, os_factor, N):
    radar = synth.Radar(n_samples=N, n_rx=3, os=os_factor)
    rng = np.random.Generator(np.random.PCG64(N + os_factor))
    M = 5
    beat = (rng.standard_normal((M, 3, N)) + 1j * rng.standard_normal((M, 3, N))).astype(np.complex64)
    grid = synth.Grid(0.0, 2.0, 0.05, 0.05, 4, 4)
    import paper_2306_09784_gb300 as sar
    plan = sar.Plan.from_radar(radar, max_pulses=M, grid=grid)
    spec = plan.range_spectrum(torch.from_numpy(beat).cuda()).cpu().numpy()
    ref = oracle.range_compress(beat, oracle.window(1, N), os_factor)
    err = np.abs(spec - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err


def test_range_spectrum_vs_cufft(torch, small):
    """Cross-check against cuFFT (torch.fft.ifft, library call) of the
    windowed, zero-padded rows."""
    wl, beat, _ = small
    plan = make_plan(wl)
    b = torch.from_numpy(beat).cuda()
    spec = plan.range_spectrum(b)
    r = wl.radar
    w = torch.from_numpy(np.hanning(r.n_samples).astype(np.float32)).cuda()
    x = torch.zeros((wl.n_pulses, r.n_rx, r.n_fft), dtype=torch.complex64, device="cuda")
    x[:, :, :r.n_samples] = b * w
    ref = torch.fft.ifft(x, dim=-1) * r.n_fft
    err = ((spec - ref).abs().max() / ref.abs().max()).item()
    assert err < 2e-6, err


@pytest.mark.parametrize("precision", [0, 1])
def test_profile_vs_oracle(torch, small, precision):
    """Stored profile = w_sar[m] rot[k] S[m][r][k] over the crop, FP32 or FP16
    with a per-(chirp, Rx) scale."""
    wl, beat, w_az = small
    plan = make_plan(wl, precision=precision)
    b, w, _, _ = to_dev(wl, beat, w_az)
    prof = plan.range_compress(b, w).cpu().numpy()
    M, R = wl.n_pulses, wl.radar.n_rx
    lo, hi = wl.crop
    nb = hi - lo + 1
    S = oracle.range_compress(beat, oracle.window(1, wl.radar.n_samples), wl.radar.os)
    ref = w_az[:, None, None] * rotation(wl.radar, wl.crop)[None, None, :] * S[:, :, lo:hi + 1]
    if precision == 0:
        got = prof.view(np.complex64).reshape(M, R, nb)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 2e-6, err
    else:
        pad = (M * R * 4 + 255) // 256 * 256
        scale = prof[:M * R * 4].view(np.float32).reshape(M, R)
        h = prof[pad:pad + M * R * nb * 4].view(np.float16).reshape(M, R, nb, 2).astype(np.float64)
        got = (h[..., 0] + 1j * h[..., 1]) * scale[..., None]
        rowmax = np.abs(ref).max(axis=-1)
        nz = rowmax > 0  # Hann w_sar is exactly zero at both ends of the aperture
        assert np.all(got[~nz] == 0)
        err = (np.abs(got - ref)[nz] / rowmax[nz][:, None]).max()
        assert err < 2e-3, err


SPLIT_CASES = [
    # (N, os, precision, sign, M, R, crop (None = full valid range))
    (1024, 4, 1, 1, 9, 4, (1207, 1833)),     # the precision frame's shape, odd crop start
    (1024, 4, 0, -1, 5, 3, (0, 4094)),       # conjugate convention, whole valid range
    (1024, 2, 1, 1, 11, 2, (301, 1500)),     # two sub-transforms per row, four rows per CTA
    (1024, 8, 0, 1, 3, 4, (2000, 6100)),     # eight sub-transforms per row (256 threads)
    (1024, 1, 1, 1, 10, 3, (5, 1000)),       # no zero padding
    (512, 4, 0, 1, 7, 3, (512, 1101)),       # the full frame's shape, ragged rows
    (512, 16, 1, 1, 4, 2, (17, 8190)),       # sixteen sub-transforms of 16 threads
    (256, 8, 1, -1, 13, 1, (33, 2046)),      # 8-thread sub-transforms
    (256, 16, 0, 1, 6, 2, (3, 4093)),
]


@pytest.mark.parametrize("case", SPLIT_CASES, ids=lambda c: f"N{c[0]}-os{c[1]}-p{c[2]}-s{c[3]}")
def test_profile_split_kernel_vs_oracle(torch, case):
    """The split-transform range compression (N = 256, 512, 1024, os sub-
    transforms of N points) against the oracle: stored profile =
    w_sar[m] rot[k] S[m][r][k] over the crop, FP32 or FP16 with a
    per-(chirp, Rx) scale."""
    N, os_factor, precision, sign, M, R, crop = case
    radar = synth.Radar(n_samples=N, n_rx=R, os=os_factor)
    rng = np.random.Generator(np.random.PCG64(N * os_factor + M))
    beat = (rng.standard_normal((M, R, N)) + 1j * rng.standard_normal((M, R, N))).astype(np.complex64)
    w_az = rng.uniform(0.2, 1.0, M)
    grid = synth.Grid(0.0, 2.0, 0.05, 0.05, 4, 4)
    import paper_2306_09784_gb300 as sar
    plan = sar.Plan.from_radar(radar, max_pulses=M, grid=grid, precision=precision, crop=crop,
                               phase_sign=sign)
    b = torch.from_numpy(beat).cuda()
    w = torch.from_numpy(w_az.astype(np.float32)).cuda()
    prof = plan.range_compress(b, w).cpu().numpy()
    lo, hi = crop
    nb = hi - lo + 1
    S = oracle.range_compress(beat, oracle.window(1, N), os_factor, sign=sign)
    ref = w_az.astype(np.float32).astype(np.float64)[:, None, None] * \
        rotation(radar, crop, sign)[None, None, :] * S[:, :, lo:hi + 1]
    if precision == 0:
        got = prof.view(np.complex64).reshape(M, R, nb)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 2e-6, err
    else:
        pad = (M * R * 4 + 255) // 256 * 256
        scale = prof[:M * R * 4].view(np.float32).reshape(M, R)
        h = prof[pad:pad + M * R * nb * 4].view(np.float16).reshape(M, R, nb, 2).astype(np.float64)
        got = (h[..., 0] + 1j * h[..., 1]) * scale[..., None]
        rowmax = np.abs(ref).max(axis=-1)
        err = (np.abs(got - ref) / rowmax[..., None]).max()
        assert err < 2e-3, err
        # the scale maps each row's largest component to 2^14
        comp = np.maximum(np.abs(h[..., 0]), np.abs(h[..., 1])).max(axis=-1)
        assert np.all(np.abs(comp - 16384.0) <= 16.0), comp


def test_profile_from_8_byte_aligned_beat(torch, small):
    """A beat cube that starts 8 bytes past a 16-byte boundary takes the
    8-byte staging copies and gives the same profiles bit for bit."""
    wl, beat, w_az = small
    plan = make_plan(wl, precision=1)
    b, w, _, _ = to_dev(wl, beat, w_az)
    big = torch.empty(b.numel() + 1, dtype=torch.complex64, device="cuda")
    shifted = big[1:].view(b.shape)
    shifted.copy_(b)
    assert shifted.data_ptr() % 16 == 8
    ref = plan.range_compress(b, w)
    got = plan.range_compress(shifted, w)
    torch.cuda.synchronize()
    assert torch.equal(ref, got)


# ----------------------------------------------------------------------------
# backprojection
# ----------------------------------------------------------------------------
def test_tiny_fp32(torch, tiny):
    """Config 'tiny': full image vs oracle, rel L2 <= 1e-3, exact peak pixels."""
    wl, beat, w_az = tiny
    plan = make_plan(wl)
    img = gpu_image(plan, wl, beat, w_az)
    ref = oracle_image(wl, beat, w_az)
    err = rel_l2(img, ref)
    print(f"tiny fp32 rel L2 = {err:.3e}")
    assert err <= TOL_FP32, err
    assert check_peaks(img, ref, peak_windows(wl, n_peaks=5)) == []
    assert plan.check_errors() == 0


def test_tiny_fp16(torch, tiny):
    wl, beat, w_az = tiny
    plan = make_plan(wl, precision=1)
    img = gpu_image(plan, wl, beat, w_az)
    ref = oracle_image(wl, beat, w_az)
    err = rel_l2(img, ref)
    print(f"tiny fp16 rel L2 = {err:.3e}")
    assert err <= TOL_FP16, err
    assert check_peaks(img, ref, peak_windows(wl, n_peaks=5)) == []


@pytest.mark.parametrize("precision", [0, 1])
def test_small_multitile_ragged(torch, small, precision):
    """80 x 72 pixels: several 32 x 32 tiles with ragged edges, 2 Rx."""
    wl, beat, w_az = small
    plan = make_plan(wl, precision=precision)
    img = gpu_image(plan, wl, beat, w_az)
    ref = oracle_image(wl, beat, w_az)
    err = rel_l2(img, ref)
    assert err <= (TOL_FP32 if precision == 0 else TOL_FP16), err


def test_subaperture_accumulate(torch, small):
    """BP over [0, M) = BP over [0, k) accumulated with BP over [k, M)."""
    wl, beat, w_az = small
    plan = make_plan(wl)
    b, w, qt, qr = to_dev(wl, beat, w_az)
    M, k = wl.n_pulses, 37
    full = plan.backproject(plan.range_compress(b, w), M, qt, qr)
    img = plan.backproject(plan.range_compress(b[:k].contiguous(), w[:k].contiguous()), k,
                           qt[:k].contiguous(), qr[:k].contiguous())
    plan.backproject(plan.range_compress(b[k:].contiguous(), w[k:].contiguous()), M - k,
                     qt[k:].contiguous(), qr[k:].contiguous(), image=img, accumulate=True)
    e = ((img - full).abs().norm() / full.abs().norm()).item()
    assert e < 1e-5, e


def test_linearity(torch, small):
    wl, beat, w_az = small
    rng = np.random.Generator(np.random.PCG64(99))
    beat2 = (rng.standard_normal(beat.shape) + 1j * rng.standard_normal(beat.shape)).astype(np.complex64)
    plan = make_plan(wl)
    a = gpu_image(plan, wl, beat, w_az)
    b = gpu_image(plan, wl, beat2, w_az)
    s = gpu_image(plan, wl, (beat + beat2).astype(np.complex64), w_az)
    assert rel_l2(a + b, s) < 1e-5


def test_deterministic(torch, small):
    wl, beat, w_az = small
    plan = make_plan(wl)
    a = gpu_image(plan, wl, beat, w_az)
    b = gpu_image(plan, wl, beat, w_az)
    assert np.array_equal(a, b)


def test_translation_invariance(torch):
    """Scene and trajectory offset by (1000 m, 1000 m): the FP64 per-tile
    reference keeps the GPU image within tolerance of the oracle (a plain FP32
    distance would lose the 77 GHz phase)."""
    wl0 = synth.make_workload("small")
    off = np.array([1000.0, 1000.0])
    wl = synth.Workload(name="small+1km", radar=wl0.radar, n_pulses=wl0.n_pulses,
                        grid=synth.Grid(wl0.grid.x0 + off[0], wl0.grid.y0 + off[1], wl0.grid.dx,
                                        wl0.grid.dy, wl0.grid.nx, wl0.grid.ny),
                        q_tx=wl0.q_tx + off, q_rx=wl0.q_rx + off, targets=wl0.targets + off,
                        amps=wl0.amps, snr_db=wl0.snr_db, seed=wl0.seed, crop=wl0.crop)
    beat = synth.workload_beat(wl)
    w_az = np.hanning(wl.n_pulses)
    plan = make_plan(wl)
    img = gpu_image(plan, wl, beat, w_az)
    ref = oracle_image(wl, beat, w_az)
    assert rel_l2(img, ref) <= TOL_FP32


@pytest.mark.parametrize("n_rx", [1, 2, 3, 4, 8, 64])
def test_rx_counts(torch, n_rx):
    """Inner-loop Rx grouping (1, 2, 3, 4), ragged pulse blocks (M = 45) and
    the largest Rx count a plan accepts (64: one chirp per pipeline block)."""
    radar = synth.Radar(n_samples=128, n_rx=n_rx, os=4)
    M = 45
    rng = np.random.Generator(np.random.PCG64(n_rx))
    q_tx, q_rx = synth.trajectory(radar, M, jitter=0.01, rng=rng)
    grid = synth.Grid(-0.8, 2.0, 0.04, 0.04, 40, 33)
    tg = np.stack([rng.uniform(-0.7, 0.7, 6), rng.uniform(2.1, 3.2, 6)], 1)
    am = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    wl = synth.Workload("rx", radar, M, grid, q_tx, q_rx, tg, am, None, 0,
                        synth.crop_for(radar, grid, q_tx, q_rx))
    beat = synth.workload_beat(wl)
    w_az = np.hanning(M)
    img = gpu_image(make_plan(wl), wl, beat, w_az)
    ref = oracle_image(wl, beat, w_az)
    assert rel_l2(img, ref) <= TOL_FP32


@pytest.mark.parametrize("os_factor", [1, 2, 8, 16])
def test_zero_padding_factors(torch, os_factor):
    radar = synth.Radar(n_samples=128 if os_factor < 16 else 256, n_rx=2, os=os_factor)
    M = 40
    q_tx, q_rx = synth.trajectory(radar, M)
    grid = synth.Grid(-0.6, 2.5, 0.05, 0.05, 24, 24)
    rng = np.random.Generator(np.random.PCG64(os_factor))
    tg = np.stack([rng.uniform(-0.5, 0.5, 4), rng.uniform(2.6, 3.6, 4)], 1)
    am = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    wl = synth.Workload("os", radar, M, grid, q_tx, q_rx, tg, am, 20.0, 1,
                        synth.crop_for(radar, grid, q_tx, q_rx))
    beat = synth.workload_beat(wl)
    w_az = np.hanning(M)
    img = gpu_image(make_plan(wl), wl, beat, w_az)
    ref = oracle_image(wl, beat, w_az)
    assert rel_l2(img, ref) <= TOL_FP32


def test_full_crop_default(torch, small):
    """crop (0, 0) = full valid range [0, N_fft - 1)."""
    wl, beat, w_az = small
    plan = make_plan(wl, crop=(0, 0))
    img = gpu_image(plan, wl, beat, w_az)
    ref = oracle_image(wl, beat, w_az, crop=(0, wl.radar.n_fft - 1))
    assert rel_l2(img, ref) <= TOL_FP32


def test_crop_cuts_geometry(torch, small):
    """A crop narrower than the geometry: terms outside contribute nothing,
    exactly as in the oracle."""
    wl, beat, w_az = small
    lo, hi = wl.crop
    crop = (lo + (hi - lo) // 3, lo + 2 * (hi - lo) // 3)
    plan = make_plan(wl, crop=crop)
    img = gpu_image(plan, wl, beat, w_az)
    ref = oracle_image(wl, beat, w_az, crop=crop)
    assert rel_l2(img, ref) <= TOL_FP32


def test_conjugate_convention(torch, small):
    wl, beat, w_az = small
    plan = make_plan(wl, phase_sign=-1)
    bc = np.conj(beat).astype(np.complex64)
    img = gpu_image(plan, wl, bc, w_az)
    ref = oracle_image(wl, bc, w_az, sign=-1)
    assert rel_l2(img, ref) <= TOL_FP32
    ref_plus = oracle_image(wl, beat, w_az)
    assert rel_l2(img, np.conj(ref_plus)) <= TOL_FP32


def test_pixel_list_polar(torch, small):
    """Explicit reconstruction points (a polar grid centred on the aperture,
    Sec. III-E) in the caller's order."""
    wl, beat, w_az = small
    rr = np.arange(1.6, 4.8, 0.03)
    th = np.deg2rad(np.arange(-35, 35, 0.6))
    R_, T_ = np.meshgrid(rr, th, indexing="ij")
    px = np.stack([R_.ravel() * np.sin(T_.ravel()), R_.ravel() * np.cos(T_.ravel())], 1)
    perm = np.random.Generator(np.random.PCG64(3)).permutation(len(px))
    px = px[perm]
    plan = make_plan(wl, pixels_xy=px)
    img = gpu_image(plan, wl, beat, w_az)
    ref = oracle_image(wl, beat, w_az, px=px)
    assert rel_l2(img, ref) <= TOL_FP32


def test_near_field_clamped_path(torch):
    """Pixels 0.3-1.5 m from the track: antennas come within twice the tile
    radius of tile references, so those pulse blocks run the clamped loop; the
    staged windows still cover every pixel and the result matches the oracle."""
    radar = synth.Radar(n_samples=128, n_rx=2, os=4)
    M = 60
    q_tx, q_rx = synth.trajectory(radar, M)
    grid = synth.Grid(-0.8, 0.3, 0.04, 0.04, 41, 31)
    rng = np.random.Generator(np.random.PCG64(17))
    tg = np.stack([rng.uniform(-0.7, 0.7, 5), rng.uniform(0.4, 1.4, 5)], 1)
    am = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    wl = synth.Workload("near", radar, M, grid, q_tx, q_rx, tg, am, 20.0, 2,
                        synth.crop_for(radar, grid, q_tx, q_rx))
    beat = synth.workload_beat(wl)
    w_az = np.hanning(M)
    img = gpu_image(make_plan(wl), wl, beat, w_az)
    ref = oracle_image(wl, beat, w_az)
    assert np.isfinite(img).all()
    assert rel_l2(img, ref) <= TOL_FP32


def test_single_pixel_single_pulse(torch):
    radar = synth.Radar(n_samples=64, n_rx=1, os=4)
    q_tx, q_rx = synth.trajectory(radar, 1)
    grid = synth.Grid(0.1, 3.0, 0.05, 0.05, 1, 1)
    wl = synth.Workload("one", radar, 1, grid, q_tx, q_rx, np.array([[0.1, 3.0]]),
                        np.array([1.0 + 0.5j]), None, 0, synth.crop_for(radar, grid, q_tx, q_rx))
    beat = synth.workload_beat(wl)
    img = gpu_image(make_plan(wl), wl, beat, np.ones(1))
    ref = oracle_image(wl, beat, np.ones(1))
    assert abs(img[0] - ref[0]) <= 1e-4 * abs(ref[0])


def test_doppler_offsets(torch, small):
    """Per-pixel f_doppler(p) index offsets of Alg. 2 (phase from d_hyp)."""
    wl, beat, w_az = small
    rng = np.random.Generator(np.random.PCG64(5))
    fd = rng.uniform(-1.5, 1.5, wl.grid.nx * wl.grid.ny)
    plan = make_plan(wl, max_doppler_bins=2.0)
    img = gpu_image(plan, wl, beat, w_az, fdopp=fd)
    ref = oracle_image(wl, beat, w_az, fd_idx=fd.astype(np.float32).astype(np.float64))
    assert rel_l2(img, ref) <= TOL_FP32


def test_doppler_offsets_at_the_largest_bound(torch, small):
    """max_doppler_bins at its limit (64 bins): the staged windows widen by
    128 bins.  Offsets up to +-70 bins: the oracle gets the caller's offsets
    as they are; pixels within the bound match it, pixels beyond it (and a
    non-finite one) get no contribution (0, or their old value when
    accumulating) and the call is flagged SAR_EBOUNDS."""
    import paper_2306_09784_gb300 as sar
    import torch as t
    wl, beat, w_az = small
    rng = np.random.Generator(np.random.PCG64(6))
    fd = rng.uniform(-70.0, 70.0, wl.grid.nx * wl.grid.ny).astype(np.float32)
    fd[17] = np.nan
    plan = make_plan(wl, max_doppler_bins=64.0)
    img = gpu_image(plan, wl, beat, w_az, fdopp=fd)
    assert plan.check_errors() == sar.SAR_EBOUNDS
    assert plan.check_errors() == sar.SAR_OK
    inb = np.abs(fd) <= 64.0
    assert 0.05 < 1.0 - inb.mean() < 0.2
    ref = oracle_image(wl, beat, w_az, fd_idx=fd.astype(np.float64))
    assert rel_l2(img[inb], ref[inb]) <= TOL_FP32
    assert np.all(img[~inb] == 0)
    # accumulating: the excluded pixels keep their old value
    b, w, qt, qr = to_dev(wl, beat, w_az)
    prof = plan.range_compress(b, w)
    base = rng.standard_normal(plan.n_pixels) + 1j * rng.standard_normal(plan.n_pixels)
    image = t.from_numpy(base.astype(np.complex64)).cuda()
    plan.backproject(prof, wl.n_pulses, qt, qr, image=image, accumulate=True,
                     fdopp=t.from_numpy(fd).cuda())
    acc = image.cpu().numpy()
    assert plan.check_errors() == sar.SAR_EBOUNDS
    assert np.array_equal(acc[~inb], base.astype(np.complex64)[~inb])
    assert rel_l2(acc[inb] - base.astype(np.complex64)[inb], ref[inb]) <= TOL_FP32


@pytest.mark.parametrize("precision", [0, 1])
def test_time_origin_chirp_centre(torch, small, precision):
    """Transform time origin at the chirp centre: the CUDA image equals the
    oracle's centred-transform image (carrier at the centre instant), with and
    without Doppler offsets; it differs from the first-sample image by the
    interpolation error that the centring removes."""
    import paper_2306_09784_gb300 as sar
    wl, beat, w_az = small
    t0 = (wl.radar.n_samples - 1) / 2.0
    tol = TOL_FP32 if precision == 0 else TOL_FP16
    plan = make_plan(wl, precision=precision, time_origin=sar.ORIGIN_CHIRP_CENTRE,
                     max_doppler_bins=2.0)
    img = gpu_image(plan, wl, beat, w_az)
    ref = oracle_image(wl, beat, w_az, t0=t0)
    assert rel_l2(img, ref) <= tol
    assert check_peaks(img, ref, peak_windows(wl)) == []
    rng = np.random.Generator(np.random.PCG64(8))
    fd = rng.uniform(-1.5, 1.5, wl.grid.nx * wl.grid.ny).astype(np.float32)
    img_fd = gpu_image(plan, wl, beat, w_az, fdopp=fd)
    assert rel_l2(img_fd, oracle_image(wl, beat, w_az, t0=t0, fd_idx=fd.astype(np.float64))) <= tol
    first = oracle_image(wl, beat, w_az)
    assert rel_l2(img, first) > 5 * tol


def test_time_origin_chirp_centre_conjugate(torch, small):
    """Chirp-centre time origin under the conjugate convention: the image is
    the conjugate of the +1 convention's centred image, and equals the
    oracle's centred transform with sign -1."""
    import paper_2306_09784_gb300 as sar
    wl, beat, w_az = small
    t0 = (wl.radar.n_samples - 1) / 2.0
    plan = make_plan(wl, phase_sign=-1, time_origin=sar.ORIGIN_CHIRP_CENTRE)
    bc = np.conj(beat).astype(np.complex64)
    img = gpu_image(plan, wl, bc, w_az)
    assert rel_l2(img, oracle_image(wl, bc, w_az, sign=-1, t0=t0)) <= TOL_FP32
    assert rel_l2(img, np.conj(oracle_image(wl, beat, w_az, t0=t0))) <= TOL_FP32


def _moving_platform(radar, M, v_p):
    q_tx, q_rx = synth.trajectory(radar, M, speed=float(v_p[0]))
    return q_tx, q_rx, np.tile(v_p, (M, 1))


def _library_doppler(plan, q_tx, q_rx, vel):
    import torch as t
    fd = plan.doppler_offsets(t.from_numpy(q_tx).cuda(), t.from_numpy(np.ascontiguousarray(q_rx)).cuda(),
                              t.from_numpy(vel).cuda())
    t.cuda.synchronize()
    return fd.cpu().numpy()


def test_doppler_offsets_vs_oracle(torch):
    """sar_doppler_offsets (Sec. III-D, mean velocity, a CUDA kernel over the
    plan's pixels) against the oracle's, pixel by pixel, on the 1024 x 1024
    precision grid with a jittered, accelerating track, and on a point list;
    also under the chirp-centre time origin (carrier at the centre)."""
    import paper_2306_09784_gb300 as sar
    wl = synth.make_workload("precision")
    M = wl.n_pulses
    t = (np.arange(M) - (M - 1) / 2) * wl.radar.pri
    vel = np.stack([10.0 + 0.8 * t, 0.3 * np.sin(t * 20.0)], 1)
    px = wl.grid.pixels()
    for origin, t0 in ((sar.ORIGIN_FIRST_SAMPLE, 0.0),
                       (sar.ORIGIN_CHIRP_CENTRE, (wl.radar.n_samples - 1) / 2.0)):
        plan = make_plan(wl, precision=1, max_doppler_bins=8.0, time_origin=origin)
        got = _library_doppler(plan, wl.q_tx, wl.q_rx, vel)
        ref = oracle.doppler_offsets(wl.radar, wl.q_tx, wl.q_rx, vel, px, t0=t0)
        assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref)), np.max(np.abs(got - ref))
    rng = np.random.Generator(np.random.PCG64(3))
    pts = np.stack([rng.uniform(-10, 10, 5000), rng.uniform(0.5, 25, 5000)], 1)
    plan = make_plan(wl, precision=1, max_doppler_bins=8.0, pixels_xy=pts)
    got = _library_doppler(plan, wl.q_tx, wl.q_rx, vel)
    ref = oracle.doppler_offsets(wl.radar, wl.q_tx, wl.q_rx, vel, pts)
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_doppler_offsets_refocus_a_moving_platform(torch):
    """Alg. 2's per-pixel f_doppler(p) on a scene recorded with the antennas
    moving during each chirp (20 m/s, targets ahead of the track, offsets of
    2 to 4 bins).  With f_doppler(p) from sar_doppler_offsets (mean velocity),
    the CUDA image matches the oracle given the oracle's own offsets, and each
    target focuses as the same scene without motion does; without offsets, or
    with their sign reversed, the focus collapses."""
    radar = synth.Radar(n_samples=128, n_rx=2, os=4)
    M, v_p = 96, np.array([20.0, 0.0])
    q_tx, q_rx, vel = _moving_platform(radar, M, v_p)
    grid = synth.Grid(x0=2.0, y0=1.0, dx=0.05, dy=0.05, nx=72, ny=64)
    cells = np.array([[12, 10], [40, 30], [60, 55]])
    targets = np.stack([grid.x0 + cells[:, 0] * grid.dx, grid.y0 + cells[:, 1] * grid.dy], 1)
    amps = np.array([1.0, 0.7 * np.exp(1j), 1.2j])
    wl = synth.Workload("moving", radar, M, grid, q_tx, q_rx, targets, amps, None, 0,
                        synth.crop_for(radar, grid, q_tx, q_rx))
    moving = synth.beat_signal(radar, q_tx, q_rx, targets, amps,
                               intra_chirp_velocity=v_p).astype(np.complex64)
    still = synth.beat_signal(radar, q_tx, q_rx, targets, amps).astype(np.complex64)
    w_az = np.hanning(M)
    plan = make_plan(wl, max_doppler_bins=8.0)
    fd = _library_doppler(plan, q_tx, q_rx, vel)
    fd_ref = oracle.doppler_offsets(radar, q_tx, q_rx, vel, grid.pixels())
    assert np.max(np.abs(fd - fd_ref)) <= 2e-6 * np.max(np.abs(fd_ref))
    img = gpu_image(plan, wl, moving, w_az, fdopp=fd)
    img_none = gpu_image(plan, wl, moving, w_az)
    img_neg = gpu_image(plan, wl, moving, w_az, fdopp=-fd)
    assert plan.check_errors() == 0
    assert rel_l2(img, oracle_image(wl, moving, w_az, fd_idx=fd_ref)) <= TOL_FP32
    focus = oracle_image(wl, still, w_az)
    for tg in targets:
        ix, iy = nearest_pixel(grid, tg)
        i = iy * grid.nx + ix
        assert abs(abs(img[i]) / abs(focus[i]) - 1.0) < 5e-3
        assert abs(img_none[i]) < 0.7 * abs(focus[i])
        assert abs(img_neg[i]) < 0.15 * abs(focus[i])


@pytest.mark.parametrize("precision", [0, 1])
def test_moving_platform_on_polar_grid(torch, precision):
    """Sec. III-D and III-E together: a moving-platform scene (intra-chirp
    motion at 20 m/s) imaged on the polar grid from sar_polar_grid with
    offsets from sar_doppler_offsets.  The library's grid equals the oracle's,
    the CUDA image equals the oracle's (oracle grid, oracle offsets) and every
    target, placed on a grid point, peaks exactly there."""
    import paper_2306_09784_gb300 as sar
    radar = synth.Radar(n_samples=128, n_rx=2, os=4)
    M, v_p = 96, np.array([20.0, 0.0])
    q_tx, q_rx, vel = _moving_platform(radar, M, v_p)
    box = (2.03, 5.61, 0.97, 4.22)
    grid_lib = sar.polar_grid(radar, q_tx, box)
    grid_ref = oracle.polar_grid(radar, q_tx, box)
    assert len(grid_lib) == len(grid_ref) > 5000
    assert np.max(np.abs(grid_lib - grid_ref)) < 1e-9
    want = np.array([[2.6, 1.5], [4.0, 2.5], [5.0, 3.75], [3.3, 3.9]])
    k = [int(np.argmin(np.hypot(*(grid_ref - w).T))) for w in want]
    targets = grid_ref[k]
    amps = np.array([1.0, 0.7 * np.exp(1j), 1.2j, 0.8 - 0.3j])
    moving = synth.beat_signal(radar, q_tx, q_rx, targets, amps,
                               intra_chirp_velocity=v_p).astype(np.complex64)
    w_az = np.hanning(M)
    cart = synth.Grid(2.0, 0.95, 0.05, 0.05, 74, 67)  # covers the box: sets the crop only
    wl = synth.Workload("polar", radar, M, cart, q_tx, q_rx, targets, amps, None, 0,
                        synth.crop_for(radar, cart, q_tx, q_rx))
    plan = make_plan(wl, precision=precision, pixels_xy=grid_lib, max_doppler_bins=8.0)
    fd = _library_doppler(plan, q_tx, q_rx, vel)
    fd_ref = oracle.doppler_offsets(radar, q_tx, q_rx, vel, grid_ref)
    assert np.max(np.abs(fd - fd_ref)) <= 2e-6 * np.max(np.abs(fd_ref))
    img = gpu_image(plan, wl, moving, w_az, fdopp=fd)
    assert plan.check_errors() == 0
    ref = oracle_image(wl, moving, w_az, px=grid_ref, fd_idx=fd_ref)
    assert rel_l2(img, ref) <= (TOL_FP32 if precision == 0 else TOL_FP16)
    e = grid_ref - 0.5 * (q_tx[0] + q_tx[-1])
    r, ph = np.hypot(e[:, 0], e[:, 1]), np.arctan2(e[:, 1], e[:, 0])
    for kk in k:  # the neighbourhood of each target: +-3 rings, +-6 angles
        win = np.nonzero((np.abs(r - r[kk]) < 0.2) & (np.abs(ph - ph[kk]) < 0.03))[0]
        assert win[np.argmax(np.abs(img[win]))] == kk
        assert win[np.argmax(np.abs(ref[win]))] == kk


def test_invalid_geometry_is_flagged(torch, small):
    """A non-finite antenna position is skipped (no contribution) and
    reported by sar_plan_check_errors; the rest of the image is unaffected."""
    import paper_2306_09784_gb300 as sar
    wl, beat, w_az = small
    plan = make_plan(wl)
    b, w, qt, qr = to_dev(wl, beat, w_az)
    qt_bad = qt.clone()
    qt_bad[5, 0] = float("nan")
    img = plan.backproject(plan.range_compress(b, w), wl.n_pulses, qt_bad, qr)
    assert plan.check_errors() == sar.SAR_EBOUNDS
    assert plan.check_errors() == sar.SAR_OK
    keep = np.ones(wl.n_pulses, bool)
    keep[5] = False
    wk = w_az.copy()
    wk[5] = 0.0
    ref = oracle_image(wl, beat, wk)
    assert np.isfinite(img.cpu().numpy()).all()
    assert rel_l2(img.cpu().numpy(), ref) <= TOL_FP32


def test_host_entry_point(torch, small):
    """sar_form_image_host (host buffers, copies inside) = the device path."""
    wl, beat, w_az = small
    plan = make_plan(wl)
    dev = gpu_image(plan, wl, beat, w_az)
    import torch as t
    hb = t.from_numpy(beat).pin_memory()
    hw = t.from_numpy(w_az.astype(np.float32)).pin_memory()
    hq = t.from_numpy(wl.q_tx).pin_memory()
    hr = t.from_numpy(np.ascontiguousarray(wl.q_rx)).pin_memory()
    out = t.empty(plan.n_pixels, dtype=t.complex64).pin_memory()
    plan.form_image_host(hb, hq, hr, out, w_az=hw)
    assert np.array_equal(out.numpy(), dev)
    # a pageable destination takes the copy path instead of the kernels' own writes
    out_pageable = t.empty(plan.n_pixels, dtype=t.complex64)
    plan.form_image_host(hb, hq, hr, out_pageable, w_az=hw)
    assert np.array_equal(out_pageable.numpy(), dev)


def test_host_entry_point_two_chunks(torch):
    """A frame large enough for sar_form_image_host to upload in two chunks
    (512^2 px, 1024 chirps x 4 Rx x 512 samples, FP16): the image equals the
    device path up to FP32 summation order (the second chunk accumulates onto
    the first) and the oracle within tolerance on the whole image."""
    import torch as t
    wl, beat, w_az, ref = _oracle_frame("full")
    plan = make_plan(wl, precision=1)
    dev = gpu_image(plan, wl, beat, w_az)
    hb = t.from_numpy(beat).pin_memory()
    hw = t.from_numpy(w_az.astype(np.float32)).pin_memory()
    hq = t.from_numpy(wl.q_tx).pin_memory()
    hr = t.from_numpy(np.ascontiguousarray(wl.q_rx)).pin_memory()
    out = t.empty(plan.n_pixels, dtype=t.complex64).pin_memory()
    plan.form_image_host(hb, hq, hr, out, w_az=hw)
    img = out.numpy()
    assert rel_l2(img, dev) < 1e-5
    out_pageable = t.empty(plan.n_pixels, dtype=t.complex64)
    plan.form_image_host(hb, hq, hr, out_pageable, w_az=hw)
    assert np.array_equal(out_pageable.numpy(), img)
    check_whole_image(wl, img, ref, TOL_FP16)


def test_invalid_arguments(torch, small):
    import paper_2306_09784_gb300 as sar
    wl, beat, w_az = small
    plan = make_plan(wl)
    b, w, qt, qr = to_dev(wl, beat, w_az)
    lib = sar.load_library()
    prof = plan.range_compress(b, w)
    img = t_img = __import__("torch").zeros(plan.n_pixels, dtype=__import__("torch").complex64,
                                            device="cuda")
    assert lib.sar_backproject(plan.handle, prof.data_ptr(), wl.n_pulses + 1, qt.data_ptr(),
                               qr.data_ptr(), None, img.data_ptr(), 0, None) == sar.SAR_EINVAL
    assert lib.sar_backproject(plan.handle, None, wl.n_pulses, qt.data_ptr(), qr.data_ptr(),
                               None, img.data_ptr(), 0, None) == sar.SAR_EINVAL
    assert lib.sar_range_compress(plan.handle, b.data_ptr(), 0, None, prof.data_ptr(),
                                  None) == sar.SAR_EINVAL
    # Doppler offsets need a plan with a Doppler bound
    fd = __import__("torch").zeros(plan.n_pixels, device="cuda")
    assert lib.sar_backproject(plan.handle, prof.data_ptr(), wl.n_pulses, qt.data_ptr(),
                               qr.data_ptr(), fd.data_ptr(), t_img.data_ptr(), 0,
                               None) == sar.SAR_EINVAL
    with pytest.raises(sar.SarError):
        sar.Plan.from_radar(synth.Radar(n_samples=100, os=3), max_pulses=4, grid=wl.grid)
    with pytest.raises(sar.SarError):
        make_plan(wl, crop=(50, 40))


def test_hbm_budget(torch, small):
    import paper_2306_09784_gb300 as sar
    wl, _, _ = small
    with pytest.raises(sar.SarError) as e:
        make_plan(wl, hbm_budget=1024)
    assert e.value.status == sar.SAR_ENOMEM


# ----------------------------------------------------------------------------
# full-size configurations, whole images
# ----------------------------------------------------------------------------
_ORACLE_FRAMES = {}


def _oracle_frame(name):
    """Seeded workload and its whole FP64 oracle image (all host cores), kept
    for both profile storages."""
    if name not in _ORACLE_FRAMES:
        wl = synth.make_workload(name)
        beat = synth.workload_beat(wl, device="cuda")
        w_az = np.hanning(wl.n_pulses)
        _ORACLE_FRAMES.clear()
        _ORACLE_FRAMES[name] = (wl, beat, w_az, oracle_image(wl, beat, w_az))
    return _ORACLE_FRAMES[name]


def _whole_frame(name, precision):
    import torch as t
    wl, beat, w_az, ref = _oracle_frame(name)
    plan = make_plan(wl, precision=precision)
    # the launch shape the benchmark uses: autotuned on these inputs
    b, w, qt, qr = to_dev(wl, beat, w_az)
    prof = plan.range_compress(b, w)
    plan.autotune(prof, wl.n_pulses, qt, qr, t.zeros(plan.n_pixels, dtype=t.complex64, device="cuda"))
    del b, w, qt, qr, prof
    img = gpu_image(plan, wl, beat, w_az)
    assert plan.check_errors() == 0
    return wl, img, ref


def check_whole_image(wl, img, ref, tol, n_peaks=20):
    """Element-by-element comparison of a whole Cartesian image: global
    relative L2 error, the error of every 32 x 32 block against the larger of
    the block's and the image's RMS (a defect confined to one tile, a split
    tile's fix-up slot or a ragged edge shows there), and exact peak pixels."""
    err = rel_l2(img, ref)
    assert err <= tol, err
    g = wl.grid
    e2 = np.abs(img - ref).reshape(g.ny, g.nx) ** 2
    r2 = np.abs(ref).reshape(g.ny, g.nx) ** 2
    rms2 = r2.mean()
    worst = 0.0
    for y0 in range(0, g.ny, 32):
        for x0 in range(0, g.nx, 32):
            eb = e2[y0:y0 + 32, x0:x0 + 32]
            rb = r2[y0:y0 + 32, x0:x0 + 32]
            worst = max(worst, math.sqrt(eb.sum() / max(rb.sum(), rms2 * eb.size)))
    assert worst <= tol, worst
    assert np.isfinite(img).all()
    assert check_peaks(img, ref, peak_windows(wl, n_peaks=n_peaks)) == []
    return err, worst


@pytest.mark.parametrize("precision", [0, 1])
def test_full_config_whole_image(torch, precision):
    """Config 'full' (512^2 px, 1024 chirps x 4 Rx, jitter, clutter): every
    pixel against the oracle."""
    wl, img, ref = _whole_frame("full", precision)
    err, worst = check_whole_image(wl, img, ref, TOL_FP32 if precision == 0 else TOL_FP16)
    print(f"full precision={precision} rel L2 = {err:.3e}, worst block {worst:.3e}")


def test_full_config_whole_image_wide_tiles(torch):
    """Config 'full' on 64 x 16 pixel tiles (FP16 profiles): every pixel
    against the oracle."""
    import paper_2306_09784_gb300 as sar
    wl, beat, w_az, ref = _oracle_frame("full")
    plan = make_plan(wl, precision=1)
    assert plan.set_tile_shape(64)["tile"] == [64, 16]
    img = gpu_image(plan, wl, beat, w_az)
    assert plan.check_errors() == sar.SAR_OK
    err, worst = check_whole_image(wl, img, ref, TOL_FP16)
    print(f"full, 64 x 16 tiles: rel L2 = {err:.3e}, worst block {worst:.3e}")


@pytest.mark.parametrize("precision", [0, 1])
def test_precision_config_whole_image(torch, precision):
    """Config 'precision' (1024^2 px at 2 cm, 2048 chirps x 1024 samples x 4 Rx),
    the benchmark workload in the bench's launch configuration: every pixel
    against the oracle."""
    wl, img, ref = _whole_frame("precision", precision)
    err, worst = check_whole_image(wl, img, ref, TOL_FP32 if precision == 0 else TOL_FP16)
    print(f"precision-config precision={precision} rel L2 = {err:.3e}, worst block {worst:.3e}")


def test_autotune_keeps_results(torch, small):
    """The autotuner changes only the launch shape: within tolerance of the
    oracle with exact peaks, and within FP32 summation order of the default
    shape when it keeps the default tiling (another tiling measures each
    pixel from another tile reference, a different FP32 rounding)."""
    wl, beat, w_az = small
    plan = make_plan(wl, precision=1)
    before = gpu_image(plan, wl, beat, w_az)
    b, w, qt, qr = to_dev(wl, beat, w_az)
    prof = plan.range_compress(b, w)
    scratch = torch.zeros(plan.n_pixels, dtype=torch.complex64, device="cuda")
    shape = plan.autotune(prof, wl.n_pulses, qt, qr, scratch)
    assert shape["pulses_per_block"] >= 1 and shape["bp_ctas"] >= 1
    assert shape["tile"] in ([32, 32], [64, 16], [16, 64])
    after = gpu_image(plan, wl, beat, w_az)
    if shape["tile"] == [32, 32]:
        assert rel_l2(after, before) < 1e-5
    ref = oracle_image(wl, beat, w_az)
    assert rel_l2(after, ref) <= TOL_FP16
    assert check_peaks(after, ref, peak_windows(wl)) == []


def test_tile_shapes(torch, small):
    """Cartesian tiles of 64 x 16, 16 x 64 and 32 x 32 pixels (ragged on the
    80 x 72 grid), FP32 and FP16 profiles: each image against the oracle with
    exact peaks; switching back to a tiling reuses it (the same image bit for
    bit); other widths and point-list plans are rejected, the plan unchanged."""
    import paper_2306_09784_gb300 as sar
    wl, beat, w_az = small
    ref = oracle_image(wl, beat, w_az)
    wins = peak_windows(wl)
    g = wl.grid
    for precision, tol in ((0, TOL_FP32), (1, TOL_FP16)):
        plan = make_plan(wl, precision=precision)
        shape0 = plan.launch_shape()
        assert shape0["tile"] == [32, 32]
        first = gpu_image(plan, wl, beat, w_az)
        imgs = {}
        for tw in (64, 16, 32):
            shape = plan.set_tile_shape(tw)
            th = 1024 // tw
            assert shape["tile"] == [tw, th]
            assert plan.info.n_tiles == -(-g.nx // tw) * -(-g.ny // th)
            img = gpu_image(plan, wl, beat, w_az)
            assert plan.check_errors() == sar.SAR_OK
            err = rel_l2(img, ref)
            assert err <= tol, (tw, err)
            assert check_peaks(img, ref, wins) == [], tw
            imgs[tw] = img
        # back on 32 x 32 tiles and the first launch shape: the same image
        plan.set_launch(shape0["rx_group"], shape0["regs_ctas_per_sm"], shape0["pulses_per_block"])
        assert plan.launch_shape() == shape0
        assert np.array_equal(gpu_image(plan, wl, beat, w_az), first)
        before = plan.launch_shape()
        for bad in (0, 8, 24, 128, -32):
            with pytest.raises(sar.SarError) as e:
                plan.set_tile_shape(bad)
            assert e.value.status == sar.SAR_EINVAL
            assert plan.launch_shape() == before
    plist = make_plan(wl, pixels_xy=g.pixels())
    assert plist.launch_shape()["tile"] == [0, 0]
    with pytest.raises(sar.SarError) as e:
        plist.set_tile_shape(32)
    assert e.value.status == sar.SAR_EINVAL


def test_autotuned_shape_is_remembered(torch, small):
    """A plan created after sar_plan_autotune with the same key (device, Rx
    count, window, storage, size buckets) starts from the tuned shape."""
    wl, beat, w_az = small
    plan = make_plan(wl, precision=1)
    b, w, qt, qr = to_dev(wl, beat, w_az)
    prof = plan.range_compress(b, w)
    scratch = torch.zeros(plan.n_pixels, dtype=torch.complex64, device="cuda")
    tuned = plan.autotune(prof, wl.n_pulses, qt, qr, scratch)
    again = make_plan(wl, precision=1)
    assert again.launch_shape() == tuned
    img = gpu_image(again, wl, beat, w_az)
    assert rel_l2(img, gpu_image(plan, wl, beat, w_az)) < 1e-6


def test_set_launch_shapes(torch):
    """Every valid launch shape gives the same image within FP32 summation
    order; shapes out of range are rejected and leave the plan unchanged."""
    import paper_2306_09784_gb300 as sar
    radar = synth.Radar(n_samples=128, n_rx=4, os=4)
    M = 40
    rng = np.random.Generator(np.random.PCG64(77))
    q_tx, q_rx = synth.trajectory(radar, M, jitter=0.01, rng=rng)
    grid = synth.Grid(-1.0, 2.0, 0.04, 0.04, 50, 41)
    tg = np.stack([rng.uniform(-0.9, 0.9, 5), rng.uniform(2.1, 3.5, 5)], 1)
    am = rng.standard_normal(5) + 1j * rng.standard_normal(5)
    wl = synth.Workload("shapes", radar, M, grid, q_tx, q_rx, tg, am, 20.0, 3,
                        synth.crop_for(radar, grid, q_tx, q_rx))
    beat = synth.workload_beat(wl)
    w_az = np.hanning(M)
    plan = make_plan(wl, precision=0)
    ref = gpu_image(plan, wl, beat, w_az)
    assert rel_l2(ref, oracle_image(wl, beat, w_az)) <= TOL_FP32
    default = plan.launch_shape()
    assert default["rx_group"] == 4
    for rg in (1, 2, 4):
        for minb in (2, 3):
            for mb in (1, 7, 16):
                shape = plan.set_launch(rg, minb, mb)
                assert (shape["rx_group"], shape["regs_ctas_per_sm"], shape["pulses_per_block"]) == \
                    (rg, minb, mb)
                img = gpu_image(plan, wl, beat, w_az)
                assert rel_l2(img, ref) < 1e-5, shape
    before = plan.launch_shape()
    for bad in ((3, 2, 8), (0, 2, 8), (5, 2, 8), (4, 1, 8), (4, 4, 8), (4, 2, 0), (4, 2, 33)):
        with pytest.raises(sar.SarError) as e:
            plan.set_launch(*bad)
        assert e.value.status == sar.SAR_EINVAL
        assert plan.launch_shape() == before
    assert plan.check_errors() == sar.SAR_OK


def test_off_axis_rx_array(torch):
    """Rx array tilted 30 degrees off the driving direction: the expansion
    loop takes its general (x and y offset) form."""
    radar = synth.Radar(n_samples=128, n_rx=4, os=4)
    M = 64
    rng = np.random.Generator(np.random.PCG64(31))
    q_tx, _ = synth.trajectory(radar, M, jitter=0.01, rng=rng)
    ang = np.deg2rad(30.0)
    step = radar.wavelength / 2 * np.array([np.cos(ang), np.sin(ang)])
    q_rx = q_tx[:, None, :] + (np.arange(4) + 1.0)[None, :, None] * step[None, None, :]
    grid = synth.Grid(-0.9, 2.2, 0.04, 0.04, 45, 38)
    tg = np.stack([rng.uniform(-0.8, 0.8, 6), rng.uniform(2.3, 3.6, 6)], 1)
    am = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    wl = synth.Workload("offaxis", radar, M, grid, q_tx, q_rx, tg, am, 20.0, 3,
                        synth.crop_for(radar, grid, q_tx, q_rx))
    beat = synth.workload_beat(wl)
    w_az = np.hanning(M)
    img = gpu_image(make_plan(wl), wl, beat, w_az)
    ref = oracle_image(wl, beat, w_az)
    assert rel_l2(img, ref) <= TOL_FP32


@pytest.mark.parametrize("precision", [0, 1])
def test_kaiser_range_window(torch, small, precision):
    """Kaiser range window (beta 6) instead of Hann (Sec. III-B)."""
    import paper_2306_09784_gb300 as sar
    wl, beat, w_az = small
    plan = make_plan(wl, precision=precision, range_window=sar.WINDOW_KAISER, kaiser_beta=6.0)
    img = gpu_image(plan, wl, beat, w_az)
    ref = oracle_image(wl, beat, w_az, range_window=oracle.WINDOW_KAISER)
    assert rel_l2(img, ref) <= (TOL_FP32 if precision == 0 else TOL_FP16)


def test_fp16_doppler_conjugate(torch, small):
    """FP16 profiles with Doppler offsets under the conjugate convention."""
    wl, beat, w_az = small
    rng = np.random.Generator(np.random.PCG64(8))
    fd = rng.uniform(-1.0, 1.0, wl.grid.nx * wl.grid.ny)
    bc = np.conj(beat).astype(np.complex64)
    plan = make_plan(wl, precision=1, phase_sign=-1, max_doppler_bins=1.5)
    img = gpu_image(plan, wl, bc, w_az, fdopp=fd)
    ref = oracle_image(wl, bc, w_az, sign=-1, fd_idx=fd.astype(np.float32).astype(np.float64))
    assert rel_l2(img, ref) <= TOL_FP16
