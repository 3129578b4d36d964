"""Batched form: several uneven requests, each with its own plan, in one
persistent backprojection launch (and under a CUDA graph)."""
import numpy as np
import pytest

import synth
from tests.gpu_helpers import TOL_FP32, make_plan, oracle_image, rel_l2, sample_pixels, to_dev

pytestmark = pytest.mark.gpu


def _prepare(wl, precision=0, device_beat=False, **kw):
    import torch
    beat = synth.workload_beat(wl, device="cuda" if device_beat else None)
    w_az = np.hanning(wl.n_pulses)
    plan = make_plan(wl, precision=precision, **kw)
    b, w, qt, qr = to_dev(wl, beat, w_az)
    prof = plan.range_compress(b, w)
    return dict(wl=wl, beat=beat, w_az=w_az, plan=plan, prof=prof, qt=qt, qr=qr)


def _single(r):
    img = r["plan"].backproject(r["prof"], r["wl"].n_pulses, r["qt"], r["qr"])
    return img


def test_mixed_batch_equals_single_requests():
    """Requests with different plans, Rx counts, storages, sizes, tile shapes
    and point lists: each batched image equals its own sar_backproject image
    (same sum up to FP32 ordering) and the oracle."""
    import torch
    import paper_2306_09784_gb300 as sar
    reqs = []
    reqs.append(_prepare(synth.make_workload("small"), 0))
    reqs.append(_prepare(synth.make_workload("small", seed=3), 1))
    reqs.append(_prepare(synth.make_workload("tiny"), 0))
    for wl in synth.make_batched_requests(5, seed=11, m_range=(40, 200), side_range=(32, 160),
                                          n_samples=128):
        reqs.append(_prepare(wl, precision=int(wl.radar.n_rx % 2)))
    # plans on other tile shapes mix with the default ones
    reqs[0]["plan"].set_tile_shape(64)
    reqs[3]["plan"].set_tile_shape(16)
    batch = sar.Batch(len(reqs))
    images = []
    for r in reqs:
        img = torch.zeros(r["plan"].n_pixels, dtype=torch.complex64, device="cuda")
        batch.add(r["plan"], r["prof"], r["wl"].n_pulses, r["qt"], r["qr"], img)
        images.append(img)
    batch.commit()
    batch.launch()
    torch.cuda.synchronize()
    assert batch.check_errors() == (sar.SAR_OK, [0, 0, 0, 0])
    n, units, ctas = batch.info()
    assert n == len(reqs) and units > 0 and ctas > 0
    assert len(batch.classes()) >= 3
    for r, img in zip(reqs, images):
        single = _single(r)
        torch.cuda.synchronize()
        e = rel_l2(img.cpu().numpy(), single.cpu().numpy())
        assert e < 1e-5, (r["wl"].name, e)
    for r, img in zip(reqs[:3], images[:3]):
        ref = oracle_image(r["wl"], r["beat"], r["w_az"])
        tol = TOL_FP32 if r["plan"].params.precision == 0 else 5e-3
        assert rel_l2(img.cpu().numpy(), ref) <= tol


def test_batch_accumulate_subapertures():
    """Two batched sub-apertures accumulated into one image = one full pass."""
    import torch
    import paper_2306_09784_gb300 as sar
    wl = synth.make_workload("small")
    r = _prepare(wl)
    full = _single(r)
    M, k = wl.n_pulses, 50
    b, w, qt, qr = to_dev(wl, r["beat"], r["w_az"])
    p1 = r["plan"].range_compress(b[:k].contiguous(), w[:k].contiguous())
    p2 = r["plan"].range_compress(b[k:].contiguous(), w[k:].contiguous())
    img = torch.zeros(r["plan"].n_pixels, dtype=torch.complex64, device="cuda")
    batch = sar.Batch(2)
    batch.add(r["plan"], p1, k, qt[:k].contiguous(), qr[:k].contiguous(), img)
    batch.commit()
    batch.launch()
    batch.clear()
    batch.add(r["plan"], p2, M - k, qt[k:].contiguous(), qr[k:].contiguous(), img, accumulate=True)
    batch.commit()
    batch.launch()
    torch.cuda.synchronize()
    assert ((img - full).abs().norm() / full.abs().norm()).item() < 1e-5


def test_batched_config_64_requests_graph():
    """The batched configuration: 64 requests of 128-1024 pulses, 128^2-768^2
    pixels, 1-4 Rx, FP16 profiles, autotuned, one persistent launch captured
    in a CUDA graph and replayed; every request matches its single-request
    image and sampled pixels match the oracle."""
    import torch
    import paper_2306_09784_gb300 as sar
    wls = synth.make_batched_requests(64, seed=5)
    reqs = [_prepare(wl, precision=1, device_beat=True) for wl in wls]
    batch = sar.Batch(64)
    images = []
    for r in reqs:
        img = torch.zeros(r["plan"].n_pixels, dtype=torch.complex64, device="cuda")
        batch.add(r["plan"], r["prof"], r["wl"].n_pulses, r["qt"], r["qr"], img)
        images.append(img)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.commit(stream)
        classes = batch.autotune(stream)
    stream.synchronize()
    assert batch.check_errors() == (sar.SAR_OK, [0, 0, 0, 0])
    # the autotuned launch: one class per Rx count (all FP16), each on the
    # whole grid with its own pulse block
    n, units, ctas = batch.info()
    assert n == 64 and sorted(c["rx_group"] for c in classes) == [1, 2, 3, 4]
    assert max(c["ctas"] for c in classes) == ctas
    assert sum(c["units"] for c in classes) == units
    assert len({c["regs_ctas_per_sm"] for c in classes}) == 1
    assert all(c["fp16"] == 1 and c["ctas"] >= 1 and 0 <= c["pulses_per_block"] <= 32 for c in classes)
    assert all(c["tuned_ms"] > 0 and c["param_args"] in (0, 1) for c in classes)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        batch.launch(stream)
    for img in images:
        img.zero_()
    g.replay()
    g.replay()  # replays overwrite (accumulate = 0): same result
    torch.cuda.synchronize()
    assert batch.check_errors() == (sar.SAR_OK, [0, 0, 0, 0])
    for r, img in zip(reqs, images):
        single = _single(r)
        torch.cuda.synchronize()
        assert rel_l2(img.cpu().numpy(), single.cpu().numpy()) < 1e-5, r["wl"].name
    for r, img in list(zip(reqs, images))[::16]:
        wl = r["wl"]
        idx = sample_pixels(r["plan"].n_pixels, 300, seed=1)
        ref = oracle_image(wl, r["beat"], r["w_az"], px=wl.grid.pixels()[idx])
        assert rel_l2(img.cpu().numpy()[idx], ref) <= 5e-3


def test_batch_mixes_time_origins():
    """Plans with the transform's time origin at the first sample and at the
    chirp centre in one batch: each image equals its own single call and the
    oracle with that origin."""
    import torch
    import paper_2306_09784_gb300 as sar
    wl = synth.make_workload("small", seed=5)
    reqs = [_prepare(wl, p, time_origin=o)
            for p in (0, 1) for o in (sar.ORIGIN_FIRST_SAMPLE, sar.ORIGIN_CHIRP_CENTRE)]
    batch = sar.Batch(len(reqs))
    images = []
    for r in reqs:
        img = torch.zeros(r["plan"].n_pixels, dtype=torch.complex64, device="cuda")
        batch.add(r["plan"], r["prof"], wl.n_pulses, r["qt"], r["qr"], img)
        images.append(img)
    batch.commit()
    batch.launch()
    torch.cuda.synchronize()
    t0 = (wl.radar.n_samples - 1) / 2.0
    for r, img in zip(reqs, images):
        got = img.cpu().numpy()
        assert rel_l2(got, _single(r).cpu().numpy()) < 1e-5
        centre = r["plan"].params.time_origin == sar.ORIGIN_CHIRP_CENTRE
        ref = oracle_image(wl, r["beat"], r["w_az"], t0=t0 if centre else 0.0)
        tol = TOL_FP32 if r["plan"].params.precision == 0 else 5e-3
        assert rel_l2(got, ref) <= tol


def test_batch_frames_range_compressed_in_packed_launches():
    """sar_batch_add_frame: frames of three transform shapes (two packed
    split-kernel classes and one shape for the general kernel) are range-
    compressed inside sar_batch_launch; each frame's profiles equal its own
    sar_range_compress bit for bit and each image equals its single
    backprojection."""
    import torch
    import paper_2306_09784_gb300 as sar
    shapes = [(512, 4, 1), (512, 4, 1), (256, 8, 0), (512, 4, 1), (128, 4, 1), (256, 8, 0)]
    frames = []
    for i, (N, os_f, prec) in enumerate(shapes):
        radar = synth.Radar(n_samples=N, n_rx=1 + i % 3, os=os_f)
        M = 40 + 17 * i
        rng = np.random.Generator(np.random.PCG64(70 + i))
        q_tx, q_rx = synth.trajectory(radar, M, jitter=0.01, rng=rng)
        grid = synth.centred_grid(48 + 16 * i, 40 + 8 * i, 0.03, 2.0)
        tg = np.stack([rng.uniform(-0.5, 0.5, 4), rng.uniform(2.2, 3.0, 4)], 1)
        am = rng.standard_normal(4) + 1j * rng.standard_normal(4)
        wl = synth.Workload(f"f{i}", radar, M, grid, q_tx, q_rx, tg, am, 20.0, i,
                            synth.crop_for(radar, grid, q_tx, q_rx))
        r = _prepare(wl, precision=prec)
        r["b"], r["w"], _, _ = to_dev(wl, r["beat"], r["w_az"])
        frames.append(r)
    batch = sar.Batch(len(frames))
    outs = []
    for r in frames:
        # zeroed: FP16 profiles leave the padding after the scale table unwritten
        prof = torch.zeros_like(r["prof"])
        r["prof"] = r["plan"].range_compress(r["b"], r["w"], out=torch.zeros_like(r["prof"]))
        img = torch.zeros(r["plan"].n_pixels, dtype=torch.complex64, device="cuda")
        batch.add_frame(r["plan"], r["b"], r["w"], prof, r["wl"].n_pulses, r["qt"], r["qr"], img)
        outs.append((prof, img))
    batch.commit()
    batch.launch()
    torch.cuda.synchronize()
    assert batch.check_errors() == (sar.SAR_OK, [0, 0, 0, 0])
    for r, (prof, img) in zip(frames, outs):
        assert torch.equal(prof, r["prof"]), r["wl"].name
        single = _single(r)
        torch.cuda.synchronize()
        assert rel_l2(img.cpu().numpy(), single.cpu().numpy()) < 1e-5, r["wl"].name


def test_batch_class_beyond_parameter_table():
    """130 requests in one class (more than the 128 whose arguments travel as
    launch parameters): the class kernel reads the device table; every image
    equals the single request's, and a 2-request batch of the same plan takes
    the parameter path with the same images."""
    import torch
    import paper_2306_09784_gb300 as sar
    r = _prepare(synth.make_workload("small"), 0)
    single = _single(r)
    torch.cuda.synchronize()
    for n, param in ((130, 0), (2, 1)):
        batch = sar.Batch(n)
        images = []
        for _ in range(n):
            img = torch.full((r["plan"].n_pixels,), float("nan"), dtype=torch.complex64, device="cuda")
            batch.add(r["plan"], r["prof"], r["wl"].n_pulses, r["qt"], r["qr"], img)
            images.append(img)
        batch.commit()
        batch.launch()
        torch.cuda.synchronize()
        assert batch.check_errors() == (sar.SAR_OK, [0, 0, 0, 0])
        cls = batch.classes()
        assert len(cls) == 1 and cls[0]["n_jobs"] == n and cls[0]["param_args"] == param
        ref = single.cpu().numpy()
        for img in images:
            e = rel_l2(img.cpu().numpy(), ref)
            assert e < 1e-5, (n, e)

