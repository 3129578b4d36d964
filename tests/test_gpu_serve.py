"""Served form: continuous batching of frames from several radars.

Failures are made on the host (malformed or oversized requests, a full
queue, timeouts, cancelled tickets, a radar thread that stops); nothing
faults, traps or hangs the GPU."""
import threading
import time

import numpy as np
import pytest

import synth
from tests.gpu_helpers import TOL_FP32, make_plan, oracle_image, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _frame(wl, precision=0, tile_w=None):
    """Host (pinned) inputs of one frame, its plan (on tiles tile_w pixels wide
    if given) and its stand-alone image."""
    import torch
    beat = synth.workload_beat(wl)
    w_az = np.hanning(wl.n_pulses).astype(np.float32)
    plan = make_plan(wl, precision=precision)
    if tile_w:
        plan.set_tile_shape(tile_w)
    b, w, qt, qr = to_dev(wl, beat, w_az)
    alone = plan.backproject(plan.range_compress(b, w), wl.n_pulses, qt, qr)
    torch.cuda.synchronize()
    host = dict(beat=torch.from_numpy(beat).pin_memory(),
                w_az=torch.from_numpy(w_az).pin_memory(),
                q_tx=torch.from_numpy(np.ascontiguousarray(wl.q_tx)).pin_memory(),
                q_rx=torch.from_numpy(np.ascontiguousarray(wl.q_rx)).pin_memory(),
                image=torch.empty(plan.n_pixels, dtype=torch.complex64).pin_memory())
    return dict(wl=wl, beat=beat, w_az=w_az, plan=plan, alone=alone.cpu().numpy(), host=host)


class _DeviceArray:
    """A float32 view of device memory the library owns (CUDA array interface)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False),
                                         "version": 2}


def _submit(srv, f):
    h = f["host"]
    return srv.submit(f["plan"], h["beat"], h["q_tx"], h["q_rx"], w_az=h["w_az"], image=h["image"])


def _frames(n, seed=21):
    out = []
    for i, wl in enumerate(synth.make_batched_requests(n, seed=seed, m_range=(60, 300),
                                                       side_range=(48, 224), n_samples=128)):
        out.append(_frame(wl, precision=i % 2, tile_w=(None, 16, 64)[i % 3]))
    return out


def test_served_frame_equals_standalone_and_oracle():
    import paper_2306_09784_gb300 as sar
    f = _frame(synth.make_workload("small"))
    srv = sar.Server(hbm_budget=256 << 20, chunk_pulses=32)
    t = _submit(srv, f)
    assert srv.wait(t, 60000) == sar.SAR_OK
    rc, state, img_dev, lat = srv.poll(t)
    assert rc == sar.SAR_OK and state == sar.REQ_DONE and img_dev and lat > 0
    img = f["host"]["image"].numpy()
    assert rel_l2(img, f["alone"]) < 1e-5
    assert rel_l2(img, oracle_image(f["wl"], f["beat"], f["w_az"])) <= TOL_FP32
    assert srv.release(t) == sar.SAR_OK
    assert srv.poll(t)[0] == sar.SAR_ENOTFOUND
    srv.close()


def test_host_image_mapped_and_pageable_match_the_device_image():
    """A pinned (mapped) destination is written by the final round's kernels,
    a pageable one by a copy: both equal the device image sar_poll returns,
    bit for bit."""
    import torch
    import paper_2306_09784_gb300 as sar
    f = _frame(synth.make_workload("small"))
    h = f["host"]
    srv = sar.Server(hbm_budget=256 << 20, chunk_pulses=40)
    for image in (torch.empty(f["plan"].n_pixels, dtype=torch.complex64).pin_memory(),
                  torch.empty(f["plan"].n_pixels, dtype=torch.complex64)):
        t = srv.submit(f["plan"], h["beat"], h["q_tx"], h["q_rx"], w_az=h["w_az"], image=image)
        assert srv.wait(t, 60000) == sar.SAR_OK
        rc, state, img_dev, _ = srv.poll(t)
        assert rc == sar.SAR_OK and img_dev
        dev = torch.as_tensor(_DeviceArray(img_dev, 2 * f["plan"].n_pixels), device="cuda")
        assert np.array_equal(image.numpy().view(np.float32), dev.cpu().numpy())
        assert rel_l2(image.numpy(), f["alone"]) < 1e-5
        srv.release(t)
    srv.close()


@pytest.mark.parametrize("chunk,quantum", [(48, 0), (4096, 2)], ids=["chunk48", "quantum2M"])
def test_each_result_same_alone_and_in_the_mix(chunk, quantum):
    """Twelve frames of different radars (plans, Rx counts, storages, sizes,
    tile shapes) submitted together and while others run: every image equals the same
    frame imaged alone, within the FP32 summation-order tolerance; with
    fixed chunks and with a work quantum per request and round."""
    import paper_2306_09784_gb300 as sar
    frames = _frames(12)
    srv = sar.Server(hbm_budget=1 << 30, chunk_pulses=chunk, quantum_mupdates=quantum)
    tickets = [_submit(srv, f) for f in frames[:6]]
    time.sleep(0.002)  # the rest arrive while the first rounds run
    tickets += [_submit(srv, f) for f in frames[6:]]
    for t in tickets:
        assert srv.wait(t, 60000) == sar.SAR_OK
    for f in frames:
        assert rel_l2(f["host"]["image"].numpy(), f["alone"]) < 1e-5, f["wl"].name
    st = srv.stats()
    assert st.completed == 12 and st.rounds >= 2
    for t in tickets:
        srv.release(t)
    srv.close()


def test_admission_by_hbm_budget():
    """A budget that holds one frame at a time: frames are admitted one after
    another and all complete."""
    import paper_2306_09784_gb300 as sar
    frames = _frames(4, seed=3)
    need = max(f["plan"].profile_bytes(f["wl"].n_pulses) + f["beat"].nbytes + f["plan"].n_pixels * 8
               + f["wl"].n_pulses * (4 + 16 + 16 * f["wl"].radar.n_rx) for f in frames)
    srv = sar.Server(hbm_budget=max(int(need * 1.05) + (64 << 10), 1 << 20), chunk_pulses=64)
    tickets = [_submit(srv, f) for f in frames]
    max_active = 0
    deadline = time.time() + 60
    while srv.stats().completed < 4 and time.time() < deadline:
        max_active = max(max_active, srv.stats().active)
        time.sleep(0.0005)
    assert srv.stats().completed == 4
    assert max_active <= 1
    for f, t in zip(frames, tickets):
        assert rel_l2(f["host"]["image"].numpy(), f["alone"]) < 1e-5
        srv.release(t)
    srv.close()


def test_rejections_on_the_host():
    import torch
    import paper_2306_09784_gb300 as sar
    f = _frame(synth.make_workload("small"))
    h = f["host"]
    # never fits the budget: a 768 x 768 frame (4.7 MB image) against 1 MiB
    big = _frame(synth.make_batched_requests(1, seed=2, m_range=(40, 40), side_range=(768, 768),
                                             n_samples=128)[0])
    small = sar.Server(hbm_budget=1 << 20)
    with pytest.raises(sar.SarError) as e:
        _submit(small, big)
    assert e.value.status == sar.SAR_ENOMEM
    small.close()
    srv = sar.Server(hbm_budget=64 << 20, queue_capacity=2, chunk_pulses=16)
    # malformed requests
    with pytest.raises(sar.SarError) as e:
        srv.submit(f["plan"], h["beat"], h["q_tx"], h["q_rx"], M=0)
    assert e.value.status == sar.SAR_EINVAL
    with pytest.raises(sar.SarError) as e:
        srv.submit(f["plan"], h["beat"], h["q_tx"], h["q_rx"], M=f["wl"].n_pulses + 1)
    assert e.value.status == sar.SAR_EINVAL
    # unknown tickets
    assert srv.poll(987654)[0] == sar.SAR_ENOTFOUND
    assert srv.release(987654) == sar.SAR_ENOTFOUND
    assert srv.wait(987654, 1.0) == sar.SAR_ENOTFOUND
    # a full queue answers EAGAIN
    outs = [torch.empty_like(h["image"]).pin_memory() for _ in range(12)]
    tickets, again = [], 0
    for o in outs:
        try:
            tickets.append(srv.submit(f["plan"], h["beat"], h["q_tx"], h["q_rx"], w_az=h["w_az"],
                                      image=o))
        except sar.SarError as err:
            assert err.status == sar.SAR_EAGAIN
            again += 1
    assert again > 0
    for t in tickets:
        assert srv.wait(t, 60000) == sar.SAR_OK
        srv.release(t)
    srv.close()


def test_wait_timeout_and_cancellation():
    import paper_2306_09784_gb300 as sar
    f = _frame(synth.make_workload("small"))
    g = _frame(synth.make_workload("small", seed=4))
    srv = sar.Server(hbm_budget=512 << 20, max_inflight=1, chunk_pulses=8)
    t1 = _submit(srv, f)
    t2 = _submit(srv, g)  # queued behind t1 (one slot)
    assert srv.wait(t2, 0.0) == sar.SAR_ETIMEOUT
    assert srv.release(t2) == sar.SAR_OK          # dropped while queued
    assert srv.poll(t2)[0] == sar.SAR_ENOTFOUND
    t3 = _submit(srv, g)
    assert srv.release(t1) == sar.SAR_OK          # cancelled while running
    assert srv.wait(t3, 60000) == sar.SAR_OK      # the server carries on
    assert rel_l2(g["host"]["image"].numpy(), g["alone"]) < 1e-5
    srv.release(t3)
    srv.close()


def test_radar_thread_that_stops():
    """Three radar threads submit frames at seeded Poisson times; one stops
    after its first frame.  Every submitted frame completes correctly."""
    import paper_2306_09784_gb300 as sar
    frames = _frames(3, seed=9)
    srv = sar.Server(hbm_budget=1 << 30, chunk_pulses=64)
    done, lock = [], threading.Lock()

    def radar(k, n_frames, rate_hz):
        rng = np.random.Generator(np.random.PCG64(100 + k))
        f = frames[k]
        h = f["host"]
        import torch
        for i in range(n_frames):
            time.sleep(rng.exponential(1.0 / rate_hz))
            out = torch.empty_like(h["image"]).pin_memory()
            t = srv.submit(f["plan"], h["beat"], h["q_tx"], h["q_rx"], w_az=h["w_az"], image=out)
            with lock:
                done.append((k, t, out))

    threads = [threading.Thread(target=radar, args=(k, n, 200.0))
               for k, n in ((0, 4), (1, 1), (2, 4))]  # radar 1 stops after one frame
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert len(done) == 9
    for k, t, out in done:
        assert srv.wait(t, 60000) == sar.SAR_OK
        assert rel_l2(out.numpy(), frames[k]["alone"]) < 1e-5
        srv.release(t)
    srv.close()
