"""Serving loop (continuous batching of frames from many drones), through the C ABI.

Each frame's decisions from the server must be identical to the same frame
run alone (bit-exact: a frame's results do not depend on the rest of its
batch), and one frame is checked against the FP64 oracle as in the chain
tests (decisions exact outside the 1e-5 tie margin).
"""
import time

import numpy as np
import pytest

import oracle
from oracle import cfar as ocfar
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MARGIN = 1e-5


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_11077_gb300 import build as b
    b.build()
    import paper_2012_11077_gb300 as pkg
    pkg.lib()
    return pkg


def params_of(rc):
    return rc.make_pre_params(synth.FS_HZ, mean_len=5, halo_c=-1)


def band_cols(rc, N, w):
    return rc.rcfar_band_plan(N, rc.make_pre_params(synth.FS_HZ, mean_len=5, halo_c=w.train_c + w.guard_c)).cols


def win_of(rc, w):
    return rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)


def run_stream(rc, srv, arrivals, drones, variants, pool, C_of, rate_scale=1.0, memory="host"):
    """Submit the stream at its arrival times (scaled); returns completions and det buffers.
    memory: "host" (pinned host frames and decisions), "device" (frames already in device
    memory, decisions written there) or "mixed" (alternating)."""
    dets, done = {}, {}
    dev_bufs, on_dev = {}, {}  # device frames and decision buffers, made (and complete) before the stream starts
    for i, (d, v) in enumerate(zip(drones, variants)):
        if memory == "device" or (memory == "mixed" and i % 2 == 1):
            x, w = pool[(int(d), int(v))]
            if (int(d), int(v)) not in on_dev:
                on_dev[(int(d), int(v))] = x.cuda()
            dev_bufs[i] = (on_dev[(int(d), int(v))],
                           torch.full((x.shape[0], C_of[int(d)]), 7, dtype=torch.uint8, device="cuda"))
    torch.cuda.synchronize()
    t0 = rc.rcfar_server_now_ns()
    for i, (ta, d, v) in enumerate(zip(arrivals, drones, variants)):
        x, w = pool[(int(d), int(v))]
        dev = memory == "device" or (memory == "mixed" and i % 2 == 1)
        if dev:
            x, det = dev_bufs[i]
        else:
            det = torch.full((x.shape[0], C_of[int(d)]), 7, dtype=torch.uint8).pin_memory()
        dets[i] = det
        t_arr = t0 + int(ta * rate_scale * 1e9)
        while rc.rcfar_server_now_ns() < t_arr:
            time.sleep(0.0002)
        rc.rcfar_server_submit(srv, x, win_of(rc, w), det, tag=i, arrival_ns=t_arr)
        for c in rc.rcfar_server_poll(srv, 64, 0):
            done[c.tag] = c
    deadline = time.time() + 120
    while len(done) < len(arrivals) and time.time() < deadline:
        for c in rc.rcfar_server_poll(srv, 256, 100):
            done[c.tag] = c
    return done, {i: d.cpu() for i, d in dets.items()}


@pytest.mark.parametrize("memory", ["host", "device", "mixed"])
def test_serving_each_result_equals_alone(rc, memory):
    arrivals, drones, variants, cases = synth.serving_stream(
        n_requests=60, n_drones=5, rate_hz=50000.0, seed=11, m_range=(64, 256), n_range=(256, 1024), n_variants=2)
    srv = rc.rcfar_server_create(device=0, budget_bytes=256 << 20, slots=2, max_batch_frames=6, max_rows=256,
                                 max_n=1024, max_window=20, params=params_of(rc))
    pool, C_of = {}, {}
    for d, vs in enumerate(cases):
        C_of[d] = band_cols(rc, vs[0].spec.N, vs[0].window)
        for v, c in enumerate(vs):
            pool[(d, v)] = (torch.from_numpy(synth.radar_frame(c.spec)).pin_memory(), c.window)
    try:
        done, dets = run_stream(rc, srv, arrivals, drones, variants, pool, C_of, memory=memory)
        stats = rc.rcfar_server_get_stats(srv)
    finally:
        rc.rcfar_server_destroy(srv)
    assert len(done) == len(arrivals)
    slots = set()
    for i, c in done.items():
        assert c.status == rc.RCFAR_OK
        assert c.arrival_ns <= c.admit_ns <= c.done_ns
        assert 1 <= c.batch_frames <= 6
        slots.add(c.slot)
    assert stats["completed"] == len(arrivals) and stats["batches"] >= len(arrivals) // 6
    assert stats["max_batch_frames_seen"] <= 6
    if memory == "host":
        assert slots == {0, 1}  # both slots carried batches (copies of one overlap the other's chain)
    # each frame alone: one-frame rcfar_run_batch on a separate handle
    h = rc.rcfar_create(device=0, max_rows=256, max_cols=520, max_n=1024, max_window=20, max_frames=1,
                        batch_bytes=64 << 20)
    try:
        alone = {}
        for (d, v), (x, w) in pool.items():
            det1 = torch.empty((x.shape[0], C_of[d]), dtype=torch.uint8, device="cuda")
            rc.rcfar_run_batch(h, [rc.frame_desc(x.cuda(), win_of(rc, w), det1)], params_of(rc))
            alone[(d, v)] = det1.cpu()
        assert rc.rcfar_get_error(h) == rc.RCFAR_OK
    finally:
        rc.rcfar_destroy(h)
    for i in range(len(arrivals)):
        assert torch.equal(dets[i], alone[(int(drones[i]), int(variants[i]))]), i
    # one drone's frame against the FP64 oracle
    d, v = int(drones[0]), int(variants[0])
    c = cases[d][v]
    X = synth.radar_frame(c.spec)
    P_o, band_o = oracle.preprocess_frame(X, synth.FS_HZ, 5, halo=c.halo_c)
    w = c.window
    res = oracle.cfar_chain(P_o, band_o, w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
    cmp = ocfar.compare_decisions(dets[0].numpy(), res.det, P_o, res.thr, res.cut, margin=MARGIN)
    assert cmp.mismatches == 0, cmp


def test_serving_rejects_device_pointers_of_no_device_and_mixed_kinds(rc):
    srv = rc.rcfar_server_create(device=0, budget_bytes=64 << 20, slots=1, max_batch_frames=4, max_rows=64,
                                 max_n=512, max_window=8, params=params_of(rc))
    try:
        w = rc.make_window(4, 4, 1, 1, 1e-3)
        x = torch.zeros((64, 512), dtype=torch.float32).pin_memory()
        C = band_cols(rc, 512, w)
        det = torch.zeros((64, C), dtype=torch.uint8).pin_memory()
        # a host buffer declared as device memory is refused by the library itself
        req = rc.rcfar_request(x.data_ptr(), 64, 512, 512, w, det.data_ptr(), C, 1, 0, rc.RCFAR_MEM_DEVICE, 0)
        assert rc.lib().rcfar_server_submit(srv, rc.ctypes.byref(req)) == rc.RCFAR_ERR_INVALID_ARG
        req.memory = 5
        assert rc.lib().rcfar_server_submit(srv, rc.ctypes.byref(req)) == rc.RCFAR_ERR_INVALID_ARG
        # a device frame with host decisions is refused by the binding
        with pytest.raises(ValueError):
            rc.rcfar_server_submit(srv, x.cuda(), w, det, tag=2)
    finally:
        rc.rcfar_server_destroy(srv)


def test_serving_admission_limits(rc):
    p = params_of(rc)
    with pytest.raises(rc.RcfarError) as e:
        rc.rcfar_server_create(device=0, budget_bytes=64 << 20, slots=1, params=rc.make_pre_params(halo_c=0))
    assert e.value.status == rc.RCFAR_ERR_INVALID_ARG
    srv = rc.rcfar_server_create(device=0, budget_bytes=8 << 20, slots=2, max_batch_frames=4, max_rows=256,
                                 max_n=2048, max_window=20, params=p)
    try:
        w = rc.make_window(4, 4, 1, 1, 1e-3)
        big = torch.zeros((300, 512), dtype=torch.float32).pin_memory()  # more rows than configured
        det = torch.zeros((300, 64), dtype=torch.uint8)
        with pytest.raises(rc.RcfarError) as e:
            rc.rcfar_server_submit(srv, big, w, det, tag=1)
        assert e.value.status == rc.RCFAR_ERR_UNSUPPORTED
        # fits the maxima but not one slot's share of the 8 MB budget
        x = torch.zeros((256, 2048), dtype=torch.float32).pin_memory()
        det = torch.zeros((256, 128), dtype=torch.uint8)
        with pytest.raises(rc.RcfarError) as e:
            rc.rcfar_server_submit(srv, x, w, det, tag=2)
        assert e.value.status == rc.RCFAR_ERR_UNSUPPORTED
    finally:
        rc.rcfar_server_destroy(srv)


def test_serving_destroy_completes_queued_frames(rc):
    arrivals, drones, variants, cases = synth.serving_stream(
        n_requests=12, n_drones=2, rate_hz=1e6, seed=5, m_range=(64, 128), n_range=(256, 512), n_variants=1)
    srv = rc.rcfar_server_create(device=0, budget_bytes=128 << 20, slots=1, max_batch_frames=2, max_rows=128,
                                 max_n=512, max_window=20, params=params_of(rc))
    keep = []
    for i, d in enumerate(drones):
        c = cases[int(d)][0]
        x = torch.from_numpy(synth.radar_frame(c.spec)).pin_memory()
        det = torch.full((c.spec.M, band_cols(rc, c.spec.N, c.window)), 7, dtype=torch.uint8).pin_memory()
        keep.append((x, det))
        rc.rcfar_server_submit(srv, x, win_of(rc, c.window), det, tag=i)
    rc.rcfar_server_destroy(srv)  # returns once every queued frame has run
    for x, det in keep:
        assert int((det == 7).sum()) == 0  # every decision byte was written (0 or 1)


def test_serving_padded_host_rows(rc):
    """Frames whose host rows are padded (ldx > N, odd and even pitches) take the
    pitched copy; frames without padding the linear one. Both give the frame's
    decisions run alone from a contiguous device copy."""
    arrivals, drones, variants, cases = synth.serving_stream(
        n_requests=8, n_drones=2, rate_hz=1e6, seed=21, m_range=(64, 200), n_range=(256, 900), n_variants=2)
    srv = rc.rcfar_server_create(device=0, budget_bytes=128 << 20, slots=2, max_batch_frames=4, max_rows=200,
                                 max_n=900, max_window=20, params=params_of(rc))
    subs = []
    try:
        for i, (d, v) in enumerate(zip(drones, variants)):
            c = cases[int(d)][int(v)]
            X = torch.from_numpy(synth.radar_frame(c.spec))
            pad = (0, 13, 4, 1)[i % 4]
            wide = torch.zeros((c.spec.M, c.spec.N + pad), dtype=torch.float32).pin_memory()
            wide[:, :c.spec.N] = X
            x = wide[:, :c.spec.N]
            assert x.stride(0) == c.spec.N + pad
            det = torch.full((c.spec.M, band_cols(rc, c.spec.N, c.window)), 7, dtype=torch.uint8).pin_memory()
            subs.append((X, c.window, det, wide))
            rc.rcfar_server_submit(srv, x, win_of(rc, c.window), det, tag=i)
        done = {}
        deadline = time.time() + 60
        while len(done) < len(subs) and time.time() < deadline:
            for cpl in rc.rcfar_server_poll(srv, 64, 100):
                done[cpl.tag] = cpl
    finally:
        rc.rcfar_server_destroy(srv)
    assert len(done) == len(subs) and all(cpl.status == rc.RCFAR_OK for cpl in done.values())
    h = rc.rcfar_create(device=0, max_rows=200, max_cols=520, max_n=900, max_window=20, max_frames=1,
                        batch_bytes=64 << 20)
    try:
        for X, w, det, _ in subs:
            det1 = torch.empty(det.shape, dtype=torch.uint8, device="cuda")
            rc.rcfar_run_batch(h, [rc.frame_desc(X.cuda(), win_of(rc, w), det1)], params_of(rc))
            assert torch.equal(det, det1.cpu())
        assert rc.rcfar_get_error(h) == rc.RCFAR_OK
    finally:
        rc.rcfar_destroy(h)


def test_serving_burst_through_submit_many(rc):
    # a burst of host and device requests queued in one call: every result equals the frame alone
    arrivals, drones, variants, cases = synth.serving_stream(
        n_requests=40, n_drones=4, rate_hz=1e6, seed=13, m_range=(64, 200), n_range=(256, 900), n_variants=2)
    srv = rc.rcfar_server_create(device=0, budget_bytes=256 << 20, slots=2, max_batch_frames=16, max_rows=200,
                                 max_n=900, max_window=20, params=params_of(rc))
    h = rc.rcfar_create(device=0, max_rows=200, max_cols=460, max_n=900, max_window=20, max_frames=1,
                        batch_bytes=64 << 20)
    try:
        reqs, dets, alone = [], [], []
        for i, (d, v) in enumerate(zip(drones, variants)):
            c = cases[int(d)][int(v)]
            x = torch.from_numpy(synth.radar_frame(c.spec))
            C = band_cols(rc, c.spec.N, c.window)
            if i % 2:
                x = x.cuda()
                det = torch.full((c.spec.M, C), 7, dtype=torch.uint8, device="cuda")
            else:
                x = x.pin_memory()
                det = torch.full((c.spec.M, C), 7, dtype=torch.uint8).pin_memory()
            reqs.append(rc.server_request(x, win_of(rc, c.window), det, tag=i))
            dets.append((x, det))
            d1 = torch.empty((c.spec.M, C), dtype=torch.uint8, device="cuda")
            rc.rcfar_run_batch(h, [rc.frame_desc(x.cuda(), win_of(rc, c.window), d1)], params_of(rc))
            alone.append(d1.cpu())
        torch.cuda.synchronize()
        assert rc.rcfar_server_submit_many(srv, reqs) == len(reqs)
        done = {}
        deadline = time.time() + 60
        while len(done) < len(reqs) and time.time() < deadline:
            for c in rc.rcfar_server_poll(srv, 256, 100):
                done[c.tag] = c
        assert len(done) == len(reqs) and all(c.status == rc.RCFAR_OK for c in done.values())
        assert max(c.batch_frames for c in done.values()) > 1  # the burst was batched
        for i, (x, det) in enumerate(dets):
            assert torch.equal(det.cpu(), alone[i]), i
        # a refused request stops the burst after the ones before it
        bad = rc.rcfar_request.from_buffer_copy(reqs[0])
        bad.M = 0
        with pytest.raises(rc.RcfarError):
            rc.rcfar_server_submit_many(srv, [reqs[0], bad, reqs[1]])
    finally:
        rc.rcfar_server_destroy(srv)
        rc.rcfar_destroy(h)
