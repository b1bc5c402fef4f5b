"""Precision study on the 8192 x 8192 map: each storage of the summed-area
table (eq. 3) against the FP64 oracle.

The map: iid Exp(1) square-law noise plus 200 point targets spanning 80 dB
(the configuration the precision question is about: an FP32 prefix sum of
it loses the small reference sums to cancellation). Window training 16 /
guard 4 per side, Pfa 1e-6, every cell a CUT candidate. Modes:

* I64       : S in 64-bit fixed point (round(x 2^s), sums modulo 2^64).
              Exact up to the map's quantisation (half a unit of 2^-s per
              cell): entries within 1e-7 of FP64, thresholds within 1e-6 (the
              final FP32 rounding), no decision differs outside the 1e-5 tie
              margin.
* TILE_F32  : FP32 tile-local table (32 x 128 tiles) plus exact int64
              carries. Each local entry carries at most ~20 roundings of
              u times its tile's sum of |x|; a threshold reads 8 entries, so
              |dT| <= (alpha / n_ref) 8 * 20 u max_tile_sum; decisions may
              differ only where |CUT - T| is within that.
* FP16 map  : the map stored in FP16 times 2^e (e puts the largest value
              below 65504) with an exact table. Each cell is rounded to 11
              bits: |dS_ref| <= 2^-11 sum|x| over the window, so thresholds
              stay within 2^-11 relative and the CUT itself within 2^-11;
              decisions may differ only where |CUT - T| / T < 2^-10.
* NAIVE_F32 : S itself in FP32 -- the contrast case; its errors are reported
              (printed), not bounded.
Table entries are compared relative to max(S, 1) (1 = the noise mean, so the
first few cells of the table, whose sums can be tiny, are compared in absolute
terms).
"""
import math

import numpy as np
import pytest

from oracle import cfar as ocfar
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_11077_gb300 import build as b
    b.build()
    import paper_2012_11077_gb300 as pkg
    pkg.lib()
    return pkg


def max_tile_sum(P):
    R, C = P.shape
    Pp = np.zeros((-(-R // 32) * 32, -(-C // 128) * 128))
    Pp[:R, :C] = np.abs(P)
    return float(Pp.reshape(Pp.shape[0] // 32, 32, Pp.shape[1] // 128, 128).sum(axis=(1, 3)).max())


def test_table_storage_modes_against_fp64_on_the_80db_map(rc):
    R = 8192
    P = synth.square_law_map(R, R, n_targets=200, seed=0)
    w = synth.map_case_window()
    nr = ocfar.n_ref(w.train_r, w.train_c, w.guard_r, w.guard_c)
    k = ocfar.alpha(nr, w.pfa) / nr
    o = ocfar.cfar_sat(P, w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
    S_o = ocfar.sat(P)
    cut = o.cut
    T_o = o.thr[cut]
    gap = np.abs(P[cut].astype(np.float64) - T_o)  # |CUT - T| at each CUT
    bound = float(P.max())
    exp2 = int(math.ceil(math.log2(bound / 60000.0)))
    h = rc.rcfar_create(device=0, max_rows=R, max_cols=R, max_n=4096, max_window=40, max_frames=1, batch_bytes=0)
    try:
        Pt = torch.from_numpy(P).cuda()
        P16 = (Pt / 2.0 ** exp2).half()
        win = rc.make_window(w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
        det = torch.empty((R, R), dtype=torch.uint8, device="cuda")
        thr = torch.empty((R, R), dtype=torch.float32, device="cuda")
        S = torch.empty((R, R), dtype=torch.float64, device="cuda")
        report = {}
        for name, mode, Pm, e2 in (("I64", rc.RCFAR_SAT_I64, Pt, 0), ("TILE_F32", rc.RCFAR_SAT_TILE_F32, Pt, 0),
                                   ("FP16", rc.RCFAR_SAT_TILE_I64, P16, exp2),
                                   ("NAIVE_F32", rc.RCFAR_SAT_NAIVE_F32, Pt, 0)):
            # FP16 rounding can lift the largest value slightly above the float32 map's
            b = bound if e2 == 0 else max(bound, float(Pm.float().max()) * 2.0 ** e2)
            v = rc.rcfar_sat(h, Pm, value_bound=b, mode=mode, map_exp2=e2)
            rc.rcfar_cfar(h, v, Pm, win, 0, R - 1, det, thr, map_exp2=e2)
            rc.rcfar_sat_materialize(h, v, S)
            assert rc.rcfar_get_error(h) == rc.RCFAR_OK
            sat_rel = float(np.max(np.abs(S.cpu().numpy() - S_o) / np.maximum(S_o, 1.0)))
            t = thr.cpu().numpy().astype(np.float64)[cut]
            thr_abs = np.abs(t - T_o)
            thr_rel = float(np.max(thr_abs / T_o))
            diff = (det.cpu().numpy() != o.det)
            d_cut = diff[cut]
            assert not diff[~cut].any(), name  # non-CUT cells decide H0 in every mode
            tie = gap < 1e-5 * T_o
            report[name] = (sat_rel, thr_rel, int((d_cut & ~tie).sum()), int((d_cut & tie).sum()))
            print(f"{name:9s}: SAT max rel err {sat_rel:.2e}, threshold max rel err {thr_rel:.2e}, "
                  f"mismatches outside / inside the 1e-5 margin {report[name][2]} / {report[name][3]}")
            if name == "I64":
                assert sat_rel <= 1e-7 and thr_rel <= 1e-6 and report[name][2] == 0
            elif name == "TILE_F32":
                dT = k * 8 * 20 * U32 * max_tile_sum(P)
                assert np.all(thr_abs <= dT + 1e-6 * T_o)
                assert np.all(gap[d_cut] <= dT + 1e-6 * T_o[d_cut])
            elif name == "FP16":
                assert thr_rel <= 2.0 ** -11
                assert np.all(gap[d_cut] < 2.0 ** -10 * T_o[d_cut])
    finally:
        rc.rcfar_destroy(h)
