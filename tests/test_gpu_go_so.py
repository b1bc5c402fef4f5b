"""GPU parity of the greatest-of / smallest-of CFAR variants (built on the same
eq. 3 table and eq. 4 lookups as the paper's cell averaging), through the C ABI.

Every path that takes a window supports them: the table CFAR in each table
mode (the streaming kernel for I64, the tiled kernel otherwise), the fused
SAT + CFAR, the cell-by-cell direct CFAR, the batched chain, the
allocation-free path and the server. Tolerances as for cell averaging:
decisions bit-exact outside the 1e-5 tie margin of the FP64 oracle,
thresholds within 1e-6 (exact tables) or 1e-5 (FP32 sums) of it; the float
tables (TILE_F32, NAIVE_F32) within their rounding bound.
"""
import numpy as np
import pytest

import oracle
from oracle import cfar as ocfar
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MARGIN = 1e-5
U32 = 2.0 ** -24
KINDS = [("go", 1), ("so", 2)]


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_11077_gb300 import build as b
    b.build()
    import paper_2012_11077_gb300 as pkg
    pkg.lib()
    return pkg


@pytest.fixture(scope="module")
def h(rc):
    hd = rc.rcfar_create(device=0, max_rows=4096, max_cols=4096, max_n=4096, max_window=40, max_frames=32,
                         batch_bytes=1 << 30)
    yield hd
    rc.rcfar_destroy(hd)


def dev_t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [
    ((300, 200), (4, 4, 1, 1, 1e-3), None),
    ((129, 260), (16, 16, 4, 4, 1e-6), (30, 200)),
    ((77, 301), (3, 5, 1, 2, 1e-2), None),
    ((40, 33), (12, 12, 8, 8, 1e-3), None),   # window larger than the map: zero CUTs
    ((500, 150), (1, 1, 0, 0, 1e-1), (3, 140)),
    ((700, 517), (16, 16, 4, 4, 1e-6), None),
    ((1030, 390), (6, 9, 2, 3, 1e-4), (40, 350)),
    ((260, 129), (2, 7, 0, 3, 1e-3), None),  # no guard rows: the halves touch the CUT row
]


def edge_map(shape, seed):
    # exponential noise with a 20 dB step along range and planted targets: the
    # two halves differ systematically next to the step
    R, C = shape
    P = synth.square_law_map(R, C, n_targets=max(1, R * C // 2000), dyn_range_db=30.0, seed=seed)
    P = P.astype(np.float64)
    P[R // 2:] *= 100.0
    return P.astype(np.float32)


def oracle_ref(P, kind, win, cut):
    return ocfar.cfar_go_so_sat(P.astype(np.float64), kind, *win, cut_cols=cut)


def float_table_bound(P, win, kind, mode):
    t = ocfar.go_so_factor(kind, ocfar.half_cells(*win[:4]), win[4])
    R, C = P.shape
    if mode == 0:
        Pp = np.zeros((-(-R // 32) * 32, -(-C // 128) * 128))
        Pp[:R, :C] = np.abs(P)
        ts = Pp.reshape(Pp.shape[0] // 32, 32, Pp.shape[1] // 128, 128).sum(axis=(1, 3)).max()
        return t * 16 * 20 * U32 * ts
    if mode == 2:
        return t * 16 * (40 + 2 * (R // 32 + C // 128)) * U32 * float(np.abs(P).sum())
    return 0.0


@pytest.mark.parametrize("kind,k", KINDS)
@pytest.mark.parametrize("shape,win,cut", CASES)
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_table_cfar_parity(rc, h, kind, k, shape, win, cut, mode):
    P = edge_map(shape, seed=shape[0] + shape[1] + k)
    rows, cols = shape
    Pt = dev_t(P)
    view = rc.rcfar_sat(h, Pt, value_bound=float(P.max()), mode=mode)
    det = torch.full((rows, cols), 7, dtype=torch.uint8, device="cuda")
    thr = torch.full((rows, cols), -1.0, dtype=torch.float32, device="cuda")
    lo, hi = cut if cut is not None else (0, cols - 1)
    rc.rcfar_cfar(h, view, Pt, rc.make_window(*win, kind=k), lo, hi, det, thr)
    assert rc.rcfar_get_error(h) == rc.RCFAR_OK
    det, thr = det.cpu().numpy(), thr.cpu().numpy()
    ref = oracle_ref(P, kind, win, cut)
    assert np.all(det[~ref.cut] == 0) and np.all(thr[~ref.cut] == 0)
    if mode in (1, 3):
        cmp = ocfar.compare_decisions(det, ref.det, P, ref.thr, ref.cut, margin=MARGIN)
        assert cmp.mismatches == 0, cmp
        if ref.cut.any():
            o = ref.thr[ref.cut]
            assert np.all(np.abs(thr[ref.cut] - o) <= 1e-6 * np.abs(o) + 1e-30)
    else:
        eb = float_table_bound(P, win, kind, mode)
        if ref.cut.any():
            err = np.abs(thr[ref.cut].astype(np.float64) - ref.thr[ref.cut])
            assert np.all(err <= eb + 1e-6 * np.abs(ref.thr[ref.cut])), (err.max(), eb)
        tie = ref.cut & (np.abs(P - ref.thr) <= np.abs(ref.thr) * MARGIN + eb)
        assert np.all((det == ref.det) | tie)


@pytest.mark.parametrize("kind,k", KINDS)
@pytest.mark.parametrize("shape,win,cut", CASES)
@pytest.mark.parametrize("map_cut", [True, False])
def test_fused_and_streaming_equal_tiled(rc, h, kind, k, shape, win, cut, map_cut):
    # fused SAT + CFAR and the streaming kernel (I64 table) give exactly the
    # tiled kernel's (TILE_I64 table) decisions and thresholds
    P = edge_map(shape, seed=3 * shape[0] + shape[1] + k)
    rows, cols = shape
    lo, hi = cut if cut is not None else (0, cols - 1)
    w = rc.make_window(*win, kind=k)
    bound = float(P.max())
    Pt = dev_t(P)
    outs = []
    for mode in (rc.RCFAR_SAT_TILE_I64, rc.RCFAR_SAT_I64):
        view = rc.rcfar_sat(h, Pt, value_bound=bound, mode=mode)
        d = torch.full((rows, cols), 7, dtype=torch.uint8, device="cuda")
        t = torch.full((rows, cols), -1.0, dtype=torch.float32, device="cuda")
        rc.rcfar_cfar(h, view, Pt if map_cut else None, w, lo, hi, d, t)
        outs.append((d, t))
    d = torch.full((rows, cols), 7, dtype=torch.uint8, device="cuda")
    t = torch.full((rows, cols), -1.0, dtype=torch.float32, device="cuda")
    rc.rcfar_sat_cfar(h, Pt, bound, w, lo, hi, d, t, map_cut=map_cut)
    outs.append((d, t))
    assert rc.rcfar_get_error(h) == rc.RCFAR_OK
    for d, t in outs[1:]:
        assert torch.equal(d, outs[0][0]) and torch.equal(t, outs[0][1])
    ref = oracle_ref(P, kind, win, cut)
    cmp = ocfar.compare_decisions(outs[0][0].cpu().numpy(), ref.det, P, ref.thr, ref.cut, margin=MARGIN)
    assert cmp.mismatches == 0, cmp


@pytest.mark.parametrize("kind,k", KINDS)
@pytest.mark.parametrize("shape,win,cut", CASES)
def test_direct_parity(rc, h, kind, k, shape, win, cut):
    P = edge_map(shape, seed=5 * shape[0] + shape[1] + k)
    rows, cols = shape
    det = torch.full((rows, cols), 7, dtype=torch.uint8, device="cuda")
    thr = torch.full((rows, cols), -1.0, dtype=torch.float32, device="cuda")
    lo, hi = cut if cut is not None else (0, cols - 1)
    rc.rcfar_cfar_direct(h, dev_t(P), rc.make_window(*win, kind=k), lo, hi, det, thr)
    assert rc.rcfar_get_error(h) == rc.RCFAR_OK
    ref = ocfar.cfar_go_so_direct(P.astype(np.float64), kind, *win, cut_cols=cut)
    cmp = ocfar.compare_decisions(det.cpu().numpy(), ref.det, P, ref.thr, ref.cut, margin=MARGIN)
    assert cmp.mismatches == 0, cmp
    if ref.cut.any():
        o = ref.thr[ref.cut]
        assert np.all(np.abs(thr.cpu().numpy()[ref.cut] - o) <= 1e-5 * np.abs(o))


def test_halves_by_hand(rc, h):
    # one CUT with train 2 / guard 1: a cell in the CUT's row counts in
    # neither half, one inside the guard box in neither, one in row r - 2 in
    # the leading half and one in the lagging corner in the lagging half
    P = np.zeros((7, 7), dtype=np.float32)
    P[3, 3] = 1.0
    P[3, 0] = 5.0
    P[2, 3] = 100.0
    P[1, 3] = 2.0
    P[6, 6] = 0.5
    for k, want in ((rc.RCFAR_CFAR_GO, 2.0), (rc.RCFAR_CFAR_SO, 0.5)):
        w = rc.make_window(2, 2, 1, 1, 1e-3, kind=k)
        t, n = rc.rcfar_threshold_factor(w)
        assert n == 3 * 7 - 3
        Pt = dev_t(P)
        for mode in (1, 3):
            view = rc.rcfar_sat(h, Pt, value_bound=128.0, mode=mode)
            d = torch.zeros((7, 7), dtype=torch.uint8, device="cuda")
            th = torch.zeros((7, 7), dtype=torch.float32, device="cuda")
            rc.rcfar_cfar(h, view, Pt, w, 0, 6, d, th)
            assert abs(float(th[3, 3]) - t * want) <= 1e-6 * t * want
            assert int(d.sum()) == int(d[3, 3]) and int(d[3, 3]) == (1.0 > t * want)
        d = torch.zeros((7, 7), dtype=torch.uint8, device="cuda")
        th = torch.zeros((7, 7), dtype=torch.float32, device="cuda")
        rc.rcfar_sat_cfar(h, Pt, 128.0, w, 0, 6, d, th)
        assert abs(float(th[3, 3]) - t * want) <= 1e-6 * t * want
        rc.rcfar_cfar_direct(h, Pt, w, 0, 6, d, th)
        assert abs(float(th[3, 3]) - t * want) <= 1e-6 * t * want
    assert rc.rcfar_get_error(h) == rc.RCFAR_OK


def test_static_path(rc, h):
    P = edge_map((300, 260), seed=77)
    for k in (1, 2):
        w = rc.make_window(8, 8, 2, 2, 1e-4, kind=k)
        Pt = dev_t(P)
        view = rc.rcfar_sat(h, Pt, value_bound=float(P.max()), mode=rc.RCFAR_SAT_TILE_I64)
        d1 = torch.empty((300, 260), dtype=torch.uint8, device="cuda")
        t1 = torch.empty((300, 260), dtype=torch.float32, device="cuda")
        rc.rcfar_cfar(h, view, Pt, w, 0, 259, d1, t1)
        d2 = torch.empty_like(d1)
        t2 = torch.empty_like(t1)
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        rc.rcfar_sat_cfar_static(Pt, float(P.max()), w, 0, 259, d2, t2, status=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert torch.equal(d1, d2) and torch.equal(t1, t2)


def test_batch_mixed_kinds_all_tunings(rc):
    # a batch mixing cell-averaging, greatest-of and smallest-of frames: every
    # tuning gives identical outputs, each frame matches the FP64 chain of
    # its kind, and a frame alone equals the frame in the batch
    cases = synth.mixed_batch_cases(9, seed=31, m_range=(64, 300), n_range=(256, 1500))
    params = rc.make_pre_params(synth.FS_HZ, mean_len=5, halo_c=-1)
    h2 = rc.rcfar_create(device=0, max_rows=512, max_cols=1100, max_n=2048, max_window=20, max_frames=16,
                         batch_bytes=1 << 30)
    names = ["ca", "go", "so"]
    try:
        keep, frames, outs = [], [], []
        for i, c in enumerate(cases):
            w = c.window
            band = rc.rcfar_band_plan(c.spec.N, rc.make_pre_params(synth.FS_HZ, mean_len=5,
                                                                   halo_c=w.train_c + w.guard_c))
            X = synth.radar_frame(c.spec)
            x = dev_t(X)
            det = torch.empty((c.spec.M, band.cols), dtype=torch.uint8, device="cuda")
            thr = torch.empty((c.spec.M, band.cols), dtype=torch.float32, device="cuda")
            win = rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa, kind=i % 3)
            keep.append((X, x, win))
            frames.append(rc.frame_desc(x, win, det, thr))
            outs.append((det, thr))
        ref = None
        for t in [rc.make_batch_tuning(), rc.make_batch_tuning(2, rc.RCFAR_SAT_I64),
                  rc.make_batch_tuning(0, rc.RCFAR_SAT_TILE_I64, (8, 32)), rc.make_batch_tuning(0, rc.RCFAR_SAT_FUSED)]:
            rc.rcfar_set_batch_tuning(h2, t)
            for d, th in outs:
                d.fill_(7)
                th.fill_(-1.0)
            rc.rcfar_run_batch(h2, frames, params)
            assert rc.rcfar_get_error(h2) == rc.RCFAR_OK
            got = [(d.cpu(), th.cpu()) for d, th in outs]
            if ref is None:
                ref = got
            else:
                for (a, b), (a2, b2) in zip(ref, got):
                    assert torch.equal(a, a2) and torch.equal(b, b2)
        for i, (c, (X, x, win), (d, th)) in enumerate(zip(cases, keep, ref)):
            w = c.window
            P_o, band_o = oracle.preprocess_frame(X, synth.FS_HZ, 5, halo=w.train_c + w.guard_c)
            res = oracle.cfar_chain(P_o, band_o, w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa,
                                    kind=names[i % 3])
            cmp = ocfar.compare_decisions(d.numpy(), res.det, P_o, res.thr, res.cut, margin=MARGIN)
            assert cmp.mismatches == 0, (i, cmp)
        for i in (1, 2):
            X, x, win = keep[i]
            d1 = torch.empty_like(outs[i][0])
            rc.rcfar_run_batch(h2, [rc.frame_desc(x, win, d1)], params)
            assert torch.equal(d1.cpu(), ref[i][0])
    finally:
        rc.rcfar_destroy(h2)


def test_server_go_so_os_frames(rc):
    params = rc.make_pre_params(synth.FS_HZ, mean_len=5, halo_c=-1)
    srv = rc.rcfar_server_create(device=0, budget_bytes=128 << 20, slots=2, max_batch_frames=4, max_rows=256,
                                 max_n=1024, max_window=20, params=params)
    h1 = rc.rcfar_create(device=0, max_rows=256, max_cols=520, max_n=1024, max_window=20, max_frames=1,
                         batch_bytes=64 << 20)
    try:
        subs = []
        for i in range(6):
            c = synth.ChainCase(synth.FrameSpec(M=128 + 16 * i, N=512, n_targets=2, seed=40 + i),
                                synth.Window(8, 8, 2, 2, 1e-4))
            x = torch.from_numpy(synth.radar_frame(c.spec)).pin_memory()
            w = rc.make_window(8, 8, 2, 2, 1e-4, kind=1 + i % 3)  # GO, SO, OS
            C = rc.rcfar_band_plan(512, rc.make_pre_params(synth.FS_HZ, mean_len=5, halo_c=10)).cols
            det = torch.full((c.spec.M, C), 7, dtype=torch.uint8).pin_memory()
            rc.rcfar_server_submit(srv, x, w, det, tag=i)
            subs.append((x, w, det))
        done = {}
        import time
        deadline = time.time() + 60
        while len(done) < len(subs) and time.time() < deadline:
            for c in rc.rcfar_server_poll(srv, 16, 100):
                done[c.tag] = c
        assert len(done) == len(subs) and all(c.status == rc.RCFAR_OK for c in done.values())
        for x, w, det in subs:
            d1 = torch.empty(det.shape, dtype=torch.uint8, device="cuda")
            rc.rcfar_run_batch(h1, [rc.frame_desc(x.cuda(), w, d1)], params)
            assert torch.equal(d1.cpu(), det)
        bad = rc.make_window(8, 8, 2, 2, 1e-4, kind=5)
        with pytest.raises(rc.RcfarError) as e:
            rc.rcfar_server_submit(srv, subs[0][0], bad, subs[0][2], tag=99)
        assert e.value.status == rc.RCFAR_ERR_INVALID_ARG
    finally:
        rc.rcfar_server_destroy(srv)
        rc.rcfar_destroy(h1)


# ------------------------------------------------------------ ordered statistic
OS_CASES = CASES[:3] + CASES[4:] + [((200, 150), (4, 4, 1, 1, 1e-3), None)]


@pytest.mark.parametrize("shape,win,cut", OS_CASES)
@pytest.mark.parametrize("rank", ["default", "first", "last"])
def test_os_direct_parity(rc, h, shape, win, cut, rank):
    # the k-th smallest is selected exactly, so the threshold is alpha_os times
    # the oracle's own cell value (one FP32 rounding of alpha and one of the product)
    P = edge_map(shape, seed=7 * shape[0] + shape[1])
    rows, cols = shape
    nref = ocfar.n_ref(*win[:4])
    k = {"default": 0, "first": 1, "last": nref}[rank]
    det = torch.full((rows, cols), 7, dtype=torch.uint8, device="cuda")
    thr = torch.full((rows, cols), -1.0, dtype=torch.float32, device="cuda")
    lo, hi = cut if cut is not None else (0, cols - 1)
    rc.rcfar_cfar_direct(h, dev_t(P), rc.make_window(*win, kind=rc.RCFAR_CFAR_OS, os_rank=k), lo, hi, det, thr)
    assert rc.rcfar_get_error(h) == rc.RCFAR_OK
    ref = ocfar.cfar_os_direct(P.astype(np.float64), *win, k=k, cut_cols=cut)
    det, thr = det.cpu().numpy(), thr.cpu().numpy()
    assert np.all(det[~ref.cut] == 0) and np.all(thr[~ref.cut] == 0)
    cmp = ocfar.compare_decisions(det, ref.det, P, ref.thr, ref.cut, margin=MARGIN)
    assert cmp.mismatches == 0, cmp
    if ref.cut.any():
        o = ref.thr[ref.cut]
        assert np.all(np.abs(thr[ref.cut] - o) <= 2.5e-7 * np.abs(o) + 1e-30)


def test_os_negative_values_and_ties(rc, h):
    # signed values (the keys must order negatives below positives) and a map
    # of small integers (many equal cells: the rank counts duplicates)
    rng = np.random.default_rng(5)
    for P in (rng.standard_normal((90, 120)).astype(np.float32),
              rng.integers(0, 6, size=(90, 120)).astype(np.float32)):
        for k in (0, 1, 30, 72):
            w = rc.make_window(4, 4, 1, 1, 1e-2, kind=rc.RCFAR_CFAR_OS, os_rank=k)
            det = torch.empty((90, 120), dtype=torch.uint8, device="cuda")
            thr = torch.empty((90, 120), dtype=torch.float32, device="cuda")
            rc.rcfar_cfar_direct(h, dev_t(P), w, 0, 119, det, thr)
            ref = ocfar.cfar_os_direct(P.astype(np.float64), 4, 4, 1, 1, 1e-2, k=k)
            t = thr.cpu().numpy()[ref.cut]
            o = ref.thr[ref.cut]
            assert np.all(np.abs(t - o) <= 2.5e-7 * np.abs(o) + 1e-30), k
            cmp = ocfar.compare_decisions(det.cpu().numpy(), ref.det, P, ref.thr, ref.cut, margin=MARGIN)
            assert cmp.mismatches == 0, (k, cmp)
    assert rc.rcfar_get_error(h) == rc.RCFAR_OK


def test_os_hand_example_and_table_paths_unsupported(rc, h):
    P = np.zeros((5, 5), dtype=np.float32)
    for (r, c), v in zip([(1, 1), (1, 2), (1, 3), (2, 1), (2, 3), (3, 1), (3, 2), (3, 3)],
                         [5.0, 2.0, 8.0, 1.0, 7.0, 3.0, 6.0, 4.0]):
        P[r, c] = v
    w = rc.make_window(1, 1, 0, 0, 1e-2, kind=rc.RCFAR_CFAR_OS)
    a, n = rc.rcfar_threshold_factor(w)
    assert n == 8
    P[2, 2] = 6.0 * a * 1.01
    Pt = dev_t(P)
    det = torch.zeros((5, 5), dtype=torch.uint8, device="cuda")
    thr = torch.zeros((5, 5), dtype=torch.float32, device="cuda")
    rc.rcfar_cfar_direct(h, Pt, w, 0, 4, det, thr)
    assert abs(float(thr[2, 2]) - 6.0 * a) <= 1e-6 * a and int(det[2, 2]) == 1 and int(det.sum()) == 1
    view = rc.rcfar_sat(h, Pt, value_bound=1e6, mode=rc.RCFAR_SAT_I64)
    for call in (lambda: rc.rcfar_cfar(h, view, Pt, w, 0, 4, det),
                 lambda: rc.rcfar_sat_cfar(h, Pt, 1e6, w, 0, 4, det),
                 lambda: rc.rcfar_sat_cfar_static(Pt, 1e6, w, 0, 4, det)):
        with pytest.raises(rc.RcfarError) as e:
            call()
        assert e.value.status == rc.RCFAR_ERR_UNSUPPORTED


def test_batch_with_os_frames(rc):
    # ordered-statistic frames in a batch with cell-averaging and greatest-of
    # frames: every tuning gives identical outputs and each frame matches the
    # FP64 chain of its kind
    cases = synth.mixed_batch_cases(8, seed=41, m_range=(64, 256), n_range=(256, 1200))
    params = rc.make_pre_params(synth.FS_HZ, mean_len=5, halo_c=-1)
    h2 = rc.rcfar_create(device=0, max_rows=512, max_cols=1100, max_n=2048, max_window=20, max_frames=16,
                         batch_bytes=1 << 30)
    kinds = [(rc.RCFAR_CFAR_OS, "os"), (rc.RCFAR_CFAR_CA, "ca"), (rc.RCFAR_CFAR_OS, "os"), (rc.RCFAR_CFAR_GO, "go")]
    try:
        keep, frames, outs = [], [], []
        for i, c in enumerate(cases):
            w = c.window
            band = rc.rcfar_band_plan(c.spec.N, rc.make_pre_params(synth.FS_HZ, mean_len=5,
                                                                   halo_c=w.train_c + w.guard_c))
            X = synth.radar_frame(c.spec)
            x = dev_t(X)
            det = torch.empty((c.spec.M, band.cols), dtype=torch.uint8, device="cuda")
            thr = torch.empty((c.spec.M, band.cols), dtype=torch.float32, device="cuda")
            win = rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa, kind=kinds[i % 4][0])
            keep.append((X, x, win))
            frames.append(rc.frame_desc(x, win, det, thr))
            outs.append((det, thr))
        ref = None
        for t in [rc.make_batch_tuning(), rc.make_batch_tuning(2, rc.RCFAR_SAT_I64),
                  rc.make_batch_tuning(0, rc.RCFAR_SAT_FUSED)]:
            rc.rcfar_set_batch_tuning(h2, t)
            for d, th in outs:
                d.fill_(7)
                th.fill_(-1.0)
            rc.rcfar_run_batch(h2, frames, params)
            assert rc.rcfar_get_error(h2) == rc.RCFAR_OK
            got = [(d.cpu(), th.cpu()) for d, th in outs]
            if ref is None:
                ref = got
            else:
                for (a, b), (a2, b2) in zip(ref, got):
                    assert torch.equal(a, a2) and torch.equal(b, b2)
        for i, (c, (X, x, win), (d, th)) in enumerate(zip(cases, keep, ref)):
            w = c.window
            P_o, band_o = oracle.preprocess_frame(X, synth.FS_HZ, 5, halo=w.train_c + w.guard_c)
            res = oracle.cfar_chain(P_o, band_o, w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa,
                                    kind=kinds[i % 4][1])
            cmp = ocfar.compare_decisions(d.numpy(), res.det, P_o, res.thr, res.cut, margin=MARGIN)
            assert cmp.mismatches == 0, (i, cmp)
    finally:
        rc.rcfar_destroy(h2)
