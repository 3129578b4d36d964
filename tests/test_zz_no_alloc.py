"""sar_backproject_noalloc: the backprojection entry point that allocates no
device memory.

It exists for callers that cannot allocate device memory while they image
frames: embedded or safety-certified automotive processes that allocate only
at start-up, and hosts whose device memory is reserved in advance by another
allocator.  Its only scratch (partial sums of pixel tiles shared by several
CTAs) is one static 16 MiB device array that every call on a device shares.

Through the C ABI these tests check that its image equals sar_backproject's,
within the parity tolerance, on two calls in a row (the second call finds the
first call's scratch contents) -- plain, accumulating onto a filled image and
with per-pixel Doppler offsets -- that a call leaves the device's free memory
unchanged, and that work beyond the static scratch is rejected with
SAR_ESCRATCH.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth
from tests.gpu_helpers import TOL_FP32, make_plan, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _run_both(wl, beat, w_az, precision):
    import torch
    import paper_2306_09784_gb300 as sar
    lib = sar.load_library()
    plan = make_plan(wl, precision=precision)
    b, w, qt, qr = to_dev(wl, beat, w_az)
    M = wl.n_pulses
    prof = plan.range_compress(b, w)
    ref = plan.backproject(prof, M, qt, qr)
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(2):  # two calls in a row share the static scratch
        img = torch.full((plan.n_pixels,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
        rc = lib.sar_backproject_noalloc(plan.handle, prof.data_ptr(), M, qt.data_ptr(),
                                         qr.data_ptr(), None, img.data_ptr(), 0, stream)
        assert rc == sar.SAR_OK, sar.status_string(rc)
        torch.cuda.synchronize()
        outs.append(img.cpu().numpy())
    assert plan.check_errors() == sar.SAR_OK
    return ref.cpu().numpy(), outs


@pytest.mark.parametrize("name,precision", [("small", 0), ("small", 1), ("tiny", 0)])
def test_noalloc_matches_backproject_twice(name, precision):
    """Every tile of these small frames is split across CTAs, so every output
    pixel passes through the static scratch."""
    wl = synth.make_workload(name)
    beat = synth.workload_beat(wl)
    ref, outs = _run_both(wl, beat, np.hanning(wl.n_pulses), precision)
    for out in outs:
        assert rel_l2(out, ref) <= TOL_FP32


def test_noalloc_accumulate_twice():
    """accumulate = 1 onto a filled image: the fix-up's read-add-write path
    through the static scratch equals sar_backproject's on the same image."""
    import torch
    import paper_2306_09784_gb300 as sar
    lib = sar.load_library()
    wl = synth.make_workload("small")
    beat = synth.workload_beat(wl)
    plan = make_plan(wl, precision=1)
    b, w, qt, qr = to_dev(wl, beat, np.hanning(wl.n_pulses))
    M = wl.n_pulses
    prof = plan.range_compress(b, w)
    g = torch.Generator(device="cuda").manual_seed(3)
    base = torch.randn(plan.n_pixels, dtype=torch.complex64, device="cuda", generator=g)
    ref = plan.backproject(prof, M, qt, qr, image=base.clone(), accumulate=True).cpu().numpy()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        img = base.clone()
        rc = lib.sar_backproject_noalloc(plan.handle, prof.data_ptr(), M, qt.data_ptr(),
                                         qr.data_ptr(), None, img.data_ptr(), 1, stream)
        assert rc == sar.SAR_OK, sar.status_string(rc)
        torch.cuda.synchronize()
        assert rel_l2(img.cpu().numpy(), ref) <= TOL_FP32
    assert plan.check_errors() == sar.SAR_OK


def test_noalloc_doppler_offsets_twice():
    """Per-pixel Doppler index offsets (a plan with max_doppler_bins > 0)
    through the static scratch equal sar_backproject's."""
    import torch
    import paper_2306_09784_gb300 as sar
    lib = sar.load_library()
    wl = synth.make_workload("small")
    beat = synth.workload_beat(wl)
    plan = make_plan(wl, max_doppler_bins=2.0)
    b, w, qt, qr = to_dev(wl, beat, np.hanning(wl.n_pulses))
    M = wl.n_pulses
    prof = plan.range_compress(b, w)
    rng = np.random.Generator(np.random.PCG64(11))
    fd = torch.from_numpy(rng.uniform(-1.5, 1.5, plan.n_pixels).astype(np.float32)).cuda()
    ref = plan.backproject(prof, M, qt, qr, fdopp=fd).cpu().numpy()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        img = torch.full((plan.n_pixels,), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
        rc = lib.sar_backproject_noalloc(plan.handle, prof.data_ptr(), M, qt.data_ptr(),
                                         qr.data_ptr(), fd.data_ptr(), img.data_ptr(), 0, stream)
        assert rc == sar.SAR_OK, sar.status_string(rc)
        torch.cuda.synchronize()
        assert rel_l2(img.cpu().numpy(), ref) <= TOL_FP32
    assert plan.check_errors() == sar.SAR_OK


def test_noalloc_call_leaves_free_memory_unchanged():
    """The property in the name: on a freshly created plan (whose creation set
    the static scratch up), a call changes the device's free memory by
    nothing.  sar_backproject runs first so that its kernels are loaded."""
    import torch
    import paper_2306_09784_gb300 as sar
    lib = sar.load_library()
    wl = synth.make_workload("small")
    beat = synth.workload_beat(wl)
    plan = make_plan(wl)
    b, w, qt, qr = to_dev(wl, beat, np.hanning(wl.n_pulses))
    M = wl.n_pulses
    prof = plan.range_compress(b, w)
    ref = plan.backproject(prof, M, qt, qr)
    img = torch.zeros(plan.n_pixels, dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    torch.cuda.mem_get_info()
    free0, _ = torch.cuda.mem_get_info()
    rc = lib.sar_backproject_noalloc(plan.handle, prof.data_ptr(), M, qt.data_ptr(),
                                     qr.data_ptr(), None, img.data_ptr(), 0, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert rc == sar.SAR_OK, sar.status_string(rc)
    assert free1 == free0, (free0, free1)
    assert rel_l2(img.cpu().numpy(), ref.cpu().numpy()) <= TOL_FP32


def test_noalloc_full_config_twice():
    """512 x 512 pixels, 1024 chirps x 4 Rx: most tiles span two CTAs."""
    wl = synth.make_workload("full")
    beat = synth.workload_beat(wl, device="cuda")
    ref, outs = _run_both(wl, beat, np.hanning(wl.n_pulses), 1)
    for out in outs:
        assert rel_l2(out, ref) <= TOL_FP32


def test_noalloc_rejects_work_beyond_static_scratch():
    """A 4096 x 2048 image (8192 tiles) needs ~70 MB of partial sums: the call
    returns SAR_ESCRATCH and leaves the image untouched."""
    import torch
    import paper_2306_09784_gb300 as sar
    lib = sar.load_library()
    radar = synth.Radar(n_samples=128, n_rx=1, os=4)
    M = 32
    grid = synth.Grid(-40.96, 2.0, 0.02, 0.02, 4096, 2048)
    plan = sar.Plan.from_radar(radar, max_pulses=M, grid=grid)
    prof = torch.zeros(plan.profile_bytes(M), dtype=torch.uint8, device="cuda")
    q_tx, q_rx = synth.trajectory(radar, M)
    qt = torch.from_numpy(q_tx).cuda()
    qr = torch.from_numpy(np.ascontiguousarray(q_rx)).cuda()
    img = torch.full((plan.n_pixels,), complex(1.0, 2.0), dtype=torch.complex64, device="cuda")
    rc = lib.sar_backproject_noalloc(plan.handle, prof.data_ptr(), M, qt.data_ptr(), qr.data_ptr(),
                                     None, img.data_ptr(), 0,
                                     torch.cuda.current_stream().cuda_stream)
    assert rc == sar.SAR_ESCRATCH
    assert "static scratch" in sar.status_string(rc)
    torch.cuda.synchronize()
    assert bool((img == complex(1.0, 2.0)).all())
