"""GPU parity at the full sizes the benchmark runs, in the launch configuration it times.

* The 8192 x 8192 square-law map (200 targets over 80 dB, training 16 / guard 4,
  Pfa 1e-6) through the fused streaming SAT + CFAR call with the CUT value from
  the map, and through the split path (int64 table in device memory, then the
  table CFAR). Every one of the 67 million decisions and every CUT's threshold
  of both paths is compared with the FP64 oracle's SAT CFAR (eq. 3 table, eq. 4
  lookups; near ties counted); as a second, independent oracle, sampled CUTs --
  every target cell and its window's corners, the corners and edges of the
  interior, and a seeded uniform sample -- are checked one by one against the
  oracle's direct window sums; every non-interior cell must decide H0.
* The 1024 x 4096 raw frame through the chain exactly as the benchmark runs it
  (rcfar_preprocess, then rcfar_sat_cfar with the CUT value from the table),
  against the oracle's whole chain; and the same frames eight at a time
  through rcfar_run_batch under the fused and the tiled schedules, identical
  to the per-frame results.

Tolerances as in test_gpu_parity: band map within 1e-4 relative of FP64
(floored a million times below the map's largest value), thresholds within
1e-4 relative, decisions exact outside the 1e-5 tie margin (counted).
"""
import numpy as np
import pytest

import oracle
from oracle import cfar as ocfar
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

REL = 1e-4
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


def _sample_cuts(R, C, wr, wc, tr, tc, rng, n_uniform=3000):
    rows, cols = [], []
    lo_r, hi_r, lo_c, hi_c = wr, R - 1 - wr, wc, C - 1 - wc
    # every target and the CUTs whose window edges fall on it
    for r, c in zip(tr, tc):
        for dr in (0, -wr, wr, -wr - 1, wr + 1):
            for dc in (0, -wc, wc, -wc - 1, wc + 1):
                rr, cc = r + dr, c + dc
                if lo_r <= rr <= hi_r and lo_c <= cc <= hi_c:
                    rows.append(rr)
                    cols.append(cc)
    # corners and edges of the interior
    for rr in (lo_r, hi_r):
        for cc in (lo_c, hi_c):
            rows.append(rr)
            cols.append(cc)
    edge = rng.integers(lo_c, hi_c + 1, size=64)
    rows += [lo_r] * 64 + [hi_r] * 64
    cols += list(edge) + list(edge)
    edge = rng.integers(lo_r, hi_r + 1, size=64)
    rows += list(edge) + list(edge)
    cols += [lo_c] * 64 + [hi_c] * 64
    rows += list(rng.integers(lo_r, hi_r + 1, size=n_uniform))
    cols += list(rng.integers(lo_c, hi_c + 1, size=n_uniform))
    return np.asarray(rows), np.asarray(cols)


def test_map_8192_fused_and_split_sampled_parity(rc):
    R = 8192
    P, tg = synth.square_law_map(R, R, n_targets=200, seed=0, return_targets=True)
    w = synth.map_case_window()
    wr, wc = w.guard_r + w.train_r, w.guard_c + w.train_c
    h = rc.rcfar_create(device=0, max_rows=R, max_cols=R, max_n=4096, max_window=40, max_frames=1, batch_bytes=0)
    try:
        Pt = torch.from_numpy(P).cuda()
        bound = float(P.max())
        win = rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
        det_f = torch.full((R, R), 7, dtype=torch.uint8, device="cuda")
        thr_f = torch.full((R, R), -1.0, dtype=torch.float32, device="cuda")  # written everywhere: 0 off the CUTs
        rc.rcfar_sat_cfar(h, Pt, bound, win, 0, R - 1, det_f, thr_f)
        det_s = torch.full((R, R), 7, dtype=torch.uint8, device="cuda")
        thr_s = torch.full((R, R), -1.0, dtype=torch.float32, device="cuda")
        view = rc.rcfar_sat(h, Pt, value_bound=bound, mode=rc.RCFAR_SAT_I64)
        rc.rcfar_cfar(h, view, Pt, win, 0, R - 1, det_s, thr_s)
        assert rc.rcfar_get_error(h) == rc.RCFAR_OK
        assert torch.equal(det_f, det_s)
        # every decision and threshold of both paths against the FP64 SAT CFAR
        o = ocfar.cfar_sat(P, w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
        for name, d_t, t_t in (("fused", det_f, thr_f), ("split", det_s, thr_s)):
            cmp = ocfar.compare_decisions(d_t.cpu().numpy(), o.det, P, o.thr, o.cut, margin=MARGIN)
            print(f"8192^2 {name}: {cmp.compared} cells compared, {cmp.mismatches} mismatches, "
                  f"{cmp.near_ties} near ties, {int(o.det.sum())} oracle detections")
            assert cmp.mismatches == 0, (name, cmp)
            tt = t_t.cpu().numpy()
            rel = np.abs(tt[o.cut].astype(np.float64) - o.thr[o.cut]) / np.abs(o.thr[o.cut])
            print(f"8192^2 {name}: threshold max rel err {rel.max():.2e}")
            assert rel.max() <= REL, (name, rel.max())
            assert np.all(tt[~o.cut] == 0.0)
            del tt, rel
        # non-interior cells decide H0 (and no byte is left unwritten)
        assert int(det_f[:wr].sum()) == 0 and int(det_f[R - wr:].sum()) == 0
        assert int(det_f[:, :wc].sum()) == 0 and int(det_f[:, R - wc:].sum()) == 0
        assert int((det_f > 1).sum()) == 0
        rows, cols = _sample_cuts(R, R, wr, wc, tg.rows, tg.cols, np.random.default_rng(8192))
        d_o, t_o = ocfar.cfar_direct_at(P, rows, cols, w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
        ri, ci = torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()
        d_g = det_f[ri, ci].cpu().numpy()
        t_g = thr_f[ri, ci].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(t_g - t_o) <= REL * np.abs(t_o)), np.max(np.abs(t_g - t_o) / np.abs(t_o))
        cut = P[rows, cols].astype(np.float64)
        near = np.abs(cut - t_o) < MARGIN * np.abs(t_o)
        bad = (d_g != d_o) & ~near
        assert not bad.any(), (rows[bad][:5], cols[bad][:5])
        # targets far above the noise, with no other target in their window, are
        # detected at their own cells
        strong = tg.power > 1e3 * 15.0
        inside = (tg.rows >= wr) & (tg.rows < R - wr) & (tg.cols >= wc) & (tg.cols < R - wc)
        dr = np.abs(tg.rows[:, None] - tg.rows[None, :])
        dc = np.abs(tg.cols[:, None] - tg.cols[None, :])
        alone = ((dr <= wr) & (dc <= wc)).sum(axis=1) == 1
        st = strong & inside & alone
        if st.any():
            got = det_f[torch.from_numpy(tg.rows[st]).cuda(), torch.from_numpy(tg.cols[st]).cuda()]
            assert int(got.sum()) == int(st.sum())
    finally:
        rc.rcfar_destroy(h)


def test_chain_1024x4096_as_benchmarked(rc):
    case = synth.large_frame_case(0)
    w = case.window
    M, N = case.spec.M, case.spec.N
    X = synth.radar_frame(case.spec)
    P_o, band_o, res_o = oracle.run_chain(X, synth.FS_HZ, case.mean_len, w.train_r, w.train_c, w.guard_r, w.guard_c,
                                          w.pfa)
    params = rc.make_pre_params(synth.FS_HZ, mean_len=case.mean_len, halo_c=case.halo_c)
    band = rc.rcfar_band_plan(N, params)
    C = band.cols
    win = rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
    h = rc.rcfar_create(device=0, max_rows=M, max_cols=1024, max_n=N, max_window=32, max_frames=8,
                        batch_bytes=1 << 30)
    try:
        x = torch.from_numpy(X).cuda()
        P = torch.empty((M, C), dtype=torch.float32, device="cuda")
        det = torch.full((M, C), 7, dtype=torch.uint8, device="cuda")
        thr = torch.full((M, C), -1.0, dtype=torch.float32, device="cuda")
        rc.rcfar_preprocess(h, x, params, P)
        rc.rcfar_sat_cfar(h, P, band.value_bound, win, band.k_lo - band.c0, band.k_hi - band.c0, det, thr,
                          map_cut=False)
        assert rc.rcfar_get_error(h) == rc.RCFAR_OK
        e = np.abs(P.cpu().numpy().astype(np.float64) - P_o) / np.maximum(np.abs(P_o), 1e-6 * np.abs(P_o).max())
        print(f"1024x4096 band map: max rel err {e.max():.2e}, cells above 1e-4: {int((e > REL).sum())}")
        assert e.max() <= REL
        cmp = ocfar.compare_decisions(det.cpu().numpy(), res_o.det, P_o, res_o.thr, res_o.cut, margin=MARGIN)
        assert cmp.mismatches == 0, cmp
        t_g = thr.cpu().numpy().astype(np.float64)[res_o.cut]
        t_o = res_o.thr[res_o.cut]
        assert np.all(np.abs(t_g - t_o) <= REL * np.abs(t_o))
        # eight such frames per batch call, under the fused and the tiled schedule
        frames = [x] + [torch.from_numpy(synth.radar_frame(synth.FrameSpec(M=M, N=N, n_targets=8, seed=s))).cuda()
                        for s in range(1, 8)]
        pb = rc.make_pre_params(synth.FS_HZ, mean_len=case.mean_len, halo_c=-1)
        alone = []
        for f in frames:
            d1 = torch.empty((M, C), dtype=torch.uint8, device="cuda")
            rc.rcfar_preprocess(h, f, params, P)
            rc.rcfar_sat_cfar(h, P, band.value_bound, win, band.k_lo - band.c0, band.k_hi - band.c0, d1,
                              map_cut=False)
            alone.append(d1)
        assert torch.equal(alone[0], det)
        for sat_mode in (rc.RCFAR_SAT_FUSED, rc.RCFAR_SAT_TILE_I64):
            rc.rcfar_set_batch_tuning(h, rc.make_batch_tuning(0, sat_mode))
            dets = [torch.full((M, C), 7, dtype=torch.uint8, device="cuda") for _ in frames]
            rc.rcfar_run_batch(h, [rc.frame_desc(f, win, d) for f, d in zip(frames, dets)], pb)
            assert rc.rcfar_get_error(h) == rc.RCFAR_OK
            for d, a in zip(dets, alone):
                assert torch.equal(d, a), sat_mode
    finally:
        rc.rcfar_destroy(h)
