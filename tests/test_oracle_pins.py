"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself: a
library routine that solves the same textbook problem, a closed form, an
invariant, brute force on tiny inputs, a hand-worked example, or a Monte-Carlo
false-alarm rate. All run on CPU (`-m "not gpu"`).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import cfar as ocfar
from oracle import preprocess as opre
import synth
from tests._golden import worked_example


# ---------------------------------------------------------------- a2 detrend
def test_detrend_matches_least_squares_line_fit():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(37, 11)) + rng.uniform(-2, 2, size=(1, 11))
    Y = opre.detrend_fast_time(X)
    m = np.arange(37)
    for n in range(11):
        slope, icpt = np.polyfit(m, X[:, n], 1)  # library least-squares line
        np.testing.assert_allclose(Y[:, n], X[:, n] - (slope * m + icpt), atol=1e-12)


def test_detrend_invariants():
    rng = np.random.default_rng(2)
    X = rng.normal(size=(64, 20))
    Y = opre.detrend_fast_time(X)
    m = np.arange(64) - 31.5
    np.testing.assert_allclose(Y.sum(axis=0), 0.0, atol=1e-11)
    np.testing.assert_allclose(m @ Y, 0.0, atol=1e-9)
    # any per-trace affine function of m is removed exactly
    a = rng.normal(size=20)
    b = rng.normal(size=20)
    X2 = X + a[None, :] + np.outer(np.arange(64), b)
    np.testing.assert_allclose(opre.detrend_fast_time(X2), Y, atol=1e-10)


# ------------------------------------------------------------ a3 mean filter
@pytest.mark.parametrize("L", [1, 3, 5, 7])
def test_mean_filter_matches_convolution(L):
    rng = np.random.default_rng(3)
    X = rng.normal(size=(5, 23))
    Y = opre.mean_filter_slow_time(X, L)
    ones = np.ones(L)
    cnt = np.convolve(np.ones(23), ones, mode="same")
    for m in range(5):
        ref = np.convolve(X[m], ones, mode="same") / cnt
        np.testing.assert_allclose(Y[m], ref, atol=1e-12)


def test_mean_filter_preserves_constants_and_rejects_even_length():
    X = np.full((3, 9), 2.5)
    np.testing.assert_allclose(opre.mean_filter_slow_time(X, 5), X, atol=0)
    with pytest.raises(ValueError):
        opre.mean_filter_slow_time(X, 4)


def test_mean_filter_brute_force_tiny():
    X = np.arange(6, dtype=float)[None, :] ** 2  # 0 1 4 9 16 25
    Y = opre.mean_filter_slow_time(X, 5)
    expect = [(0 + 1 + 4) / 3, (0 + 1 + 4 + 9) / 4, (0 + 1 + 4 + 9 + 16) / 5,
              (1 + 4 + 9 + 16 + 25) / 5, (4 + 9 + 16 + 25) / 4, (9 + 16 + 25) / 3]
    np.testing.assert_allclose(Y[0], expect, atol=1e-14)


# ------------------------------------------------------------ a4 normalise
def test_normalise():
    rng = np.random.default_rng(4)
    Y = rng.normal(size=(10, 10))
    Z = opre.normalise(Y)
    assert abs(np.max(np.abs(Z)) - 1.0) < 1e-15
    np.testing.assert_allclose(Z * np.max(np.abs(Y)), Y, rtol=1e-15)
    zero = np.zeros((3, 4))
    np.testing.assert_array_equal(opre.normalise(zero), zero)


# ------------------------------------------------------------ a5 band DFT
@pytest.mark.parametrize("N", [16, 17, 97, 512, 600])
def test_band_dft_matches_library_fft(N):
    rng = np.random.default_rng(N)
    Y = rng.normal(size=(4, N))
    c0, c1 = 1, N // 2
    P = opre.band_dft_magnitude(Y, c0, c1)
    ref = np.abs(np.fft.rfft(Y, axis=1))[:, c0:c1 + 1]
    np.testing.assert_allclose(P, ref, rtol=1e-10, atol=1e-10)


def test_band_dft_pure_tone_closed_form():
    N, k, A = 600, 37, 1.7
    n = np.arange(N)
    y = A * np.cos(2 * np.pi * k * n / N + 0.3)
    P = opre.band_dft_magnitude(y[None, :], 30, 45)[0]
    expect = np.zeros(16)
    expect[k - 30] = A * N / 2
    np.testing.assert_allclose(P, expect, atol=1e-9)


def test_band_plan_integer_form():
    # fs = 20 Hz: k_lo = ceil(0.3 N / 20) = ceil(3N/200), k_hi = floor(8N/200)
    for N in range(256, 4097):
        b = opre.band_plan(N, 20.0, 0.3, 0.8, halo=0)
        assert b.k_lo == -((-3 * N) // 200)
        assert b.k_hi == (8 * N) // 200
    b = opre.band_plan(512, 20.0, halo=10)
    assert (b.k_lo, b.k_hi, b.c0, b.c1) == (8, 20, 0, 30)
    b = opre.band_plan(4096, 20.0, halo=20)
    assert (b.k_lo, b.k_hi, b.c0, b.c1) == (62, 163, 42, 183)
    b = opre.band_plan(400, 20.0)  # exact integer edges are inside the band
    assert (b.k_lo, b.k_hi) == (6, 16)


# ------------------------------------------------------------ a6/a7 SAT, eq. 3 and eq. 4
def test_sat_matches_double_cumsum():
    rng = np.random.default_rng(6)
    P = rng.exponential(size=(33, 47))
    np.testing.assert_allclose(ocfar.sat(P), np.cumsum(np.cumsum(P, 0), 1), rtol=1e-13)


def test_sat_brute_force_tiny():
    P = synth.integer_map(5, 6, seed=7).astype(float)
    S = ocfar.sat(P)
    for r in range(5):
        for c in range(6):
            assert S[r, c] == P[:r + 1, :c + 1].sum()


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (4, 7), (9, 13)])
def test_box_sum_all_rectangles(shape):
    P = synth.integer_map(*shape, seed=shape[0] * 31 + shape[1]).astype(float)
    S = ocfar.sat(P)
    R, C = shape
    for r0, r1 in itertools.combinations_with_replacement(range(R), 2):
        for c0, c1 in itertools.combinations_with_replacement(range(C), 2):
            got = ocfar.box_sum(S, r0, r1, c0, c1)
            assert got == P[r0:r1 + 1, c0:c1 + 1].sum()


# ------------------------------------------------------------ a8 eq. 2
def test_n_ref_matches_mask_count():
    for tr, gd in itertools.product([1, 2, 4, 8, 16], [0, 1, 2, 4]):
        w = tr + gd
        yy, xx = np.mgrid[-w:w + 1, -w:w + 1]
        ring = ~((np.abs(yy) <= gd) & (np.abs(xx) <= gd))
        assert ocfar.n_ref(tr, tr, gd, gd) == int(ring.sum())
    yy, xx = np.mgrid[-5:6, -3:4]
    ring = ~((np.abs(yy) <= 1) & (np.abs(xx) <= 2))
    assert ocfar.n_ref(4, 1, 1, 2) == int(ring.sum())


@pytest.mark.parametrize("nr,pfa", [(16, 1e-3), (112, 1e-3), (416, 1e-4), (1600, 1e-6)])
def test_alpha_inverts_exponential_false_alarm_law(nr, pfa):
    # For iid Exp(1) noise, P(CUT > alpha * mean of nr cells) = (1 + alpha/nr)^(-nr).
    a = ocfar.alpha(nr, pfa)
    assert a > 0
    assert abs((1.0 + a / nr) ** (-nr) - pfa) / pfa < 1e-12
    assert ocfar.alpha_as_printed(nr, pfa) < 0  # the printed eq. 2 cannot be a threshold


def test_alpha_values_and_limit():
    assert abs(ocfar.alpha(416, 1e-4) - 9.313057) < 1e-6
    assert abs(ocfar.alpha(1600, 1e-6) - 13.875329) < 1e-6
    assert abs(ocfar.alpha(112, 1e-3) - 7.125226) < 1e-6
    assert abs(ocfar.alpha(10 ** 9, 1e-4) - (-math.log(1e-4))) < 1e-5


# ------------------------------------------------------------ a9/a10 CFAR
def test_worked_example_by_hand():
    P, (tr, tc, gr, gc, pfa), sref, det = worked_example()
    a = ocfar.alpha(ocfar.n_ref(tr, tc, gr, gc), pfa)
    for fn in (ocfar.cfar_direct, ocfar.cfar_sat):
        res = fn(P, tr, tc, gr, gc, pfa)
        np.testing.assert_array_equal(res.det, det)
        np.testing.assert_allclose(res.thr[2:5, 2:5], a * sref / 16.0, rtol=1e-14)
        assert res.cut.sum() == 9


def test_direct_equals_sat_random_maps():
    rng = np.random.default_rng(9)
    for shape, win in [((40, 50), (3, 2, 1, 2, 1e-2)), ((64, 31), (8, 8, 2, 2, 1e-4)),
                       ((25, 25), (4, 4, 0, 0, 1e-1))]:
        P = rng.exponential(size=shape)
        P[rng.integers(0, shape[0], 5), rng.integers(0, shape[1], 5)] += 30
        d = ocfar.cfar_direct(P, *win)
        s = ocfar.cfar_sat(P, *win)
        np.testing.assert_allclose(s.thr, d.thr, rtol=1e-12, atol=1e-12)
        cmp = ocfar.compare_decisions(s.det, d.det, P, d.thr, d.cut, margin=1e-9)
        assert cmp.mismatches == 0


@pytest.mark.parametrize("shape,win", [((40, 50), (3, 2, 1, 2, 1e-2)),    # non-square window
                                       ((37, 61), (2, 6, 3, 0, 1e-3)),    # zero guard columns, guard rows > train
                                       ((25, 25), (4, 4, 0, 0, 1e-1)),    # no guard at all
                                       ((64, 31), (8, 8, 2, 2, 1e-4))])
def test_direct_at_equals_sliding_window_every_cut(shape, win):
    # cfar_direct_at (outer box sum minus guard box sum, per CUT) against
    # cfar_direct (the n_ref offsets summed one at a time) at every interior
    # CUT, and against a third form that masks the window cell by cell
    rng = np.random.default_rng(21)
    P = rng.exponential(size=shape)
    P[rng.integers(0, shape[0], 6), rng.integers(0, shape[1], 6)] += 40.0
    tr, tc, gr, gc, pfa = win
    d = ocfar.cfar_direct(P, *win)
    rs, cs = np.nonzero(d.cut)
    assert rs.size > 0
    det, thr = ocfar.cfar_direct_at(P, rs, cs, *win)
    np.testing.assert_allclose(thr, d.thr[rs, cs], rtol=1e-13)
    np.testing.assert_array_equal(det, d.det[rs, cs])
    wr, wc = gr + tr, gc + tc
    nr = ocfar.n_ref(tr, tc, gr, gc)
    a = ocfar.alpha(nr, pfa)
    dr, dc = np.meshgrid(np.arange(-wr, wr + 1), np.arange(-wc, wc + 1), indexing="ij")
    train = ~((np.abs(dr) <= gr) & (np.abs(dc) <= gc))
    assert int(train.sum()) == nr
    for i in rng.choice(rs.size, size=min(rs.size, 40), replace=False):
        r, c = rs[i], cs[i]
        t = a * P[r - wr:r + wr + 1, c - wc:c + wc + 1][train].sum() / nr
        assert abs(thr[i] - t) <= 1e-13 * t
        assert det[i] == (1 if P[r, c] > t else 0)


def test_direct_at_worked_example():
    P, (tr, tc, gr, gc, pfa), sref, det = worked_example()
    a = ocfar.alpha(ocfar.n_ref(tr, tc, gr, gc), pfa)
    rs, cs = np.meshgrid(np.arange(2, 5), np.arange(2, 5), indexing="ij")
    d, t = ocfar.cfar_direct_at(P, rs.ravel(), cs.ravel(), tr, tc, gr, gc, pfa)
    np.testing.assert_array_equal(d, det[2:5, 2:5].ravel())
    np.testing.assert_allclose(t, a * sref.ravel() / 16.0, rtol=1e-14)


def test_scale_invariance_power_of_two():
    rng = np.random.default_rng(10)
    P = rng.exponential(size=(48, 48))
    base = ocfar.cfar_sat(P, 4, 4, 1, 1, 1e-3)
    for k in (-7, 3, 20):
        res = ocfar.cfar_sat(P * 2.0 ** k, 4, 4, 1, 1, 1e-3)
        np.testing.assert_array_equal(res.det, base.det)


def test_planted_target_detected_at_its_cell():
    rng = np.random.default_rng(11)
    P = rng.exponential(size=(60, 60))
    P[30, 25] += 200.0
    res = ocfar.cfar_sat(P, 8, 8, 2, 2, 1e-6)
    assert res.det[30, 25] == 1
    assert res.det.sum() == 1


def test_zero_interior_cuts_and_column_restriction():
    P = np.ones((10, 10))
    res = ocfar.cfar_sat(P, 8, 8, 2, 2, 1e-4)  # window larger than the map
    assert res.cut.sum() == 0 and res.det.sum() == 0
    res = ocfar.cfar_direct(P, 1, 1, 1, 1, 1e-3, cut_cols=(4, 5))
    assert res.cut.sum() == 6 * 2
    # a constant map never detects: CUT = A and alpha > 1
    assert res.det.sum() == 0


@pytest.mark.parametrize("pfa,shape,win", [(1e-2, (2200, 2200), (4, 4, 1, 1)),
                                           (1e-3, (3300, 3300), (4, 4, 1, 1))])
def test_monte_carlo_false_alarm_rate(pfa, shape, win):
    # CUTs on a stride of 2W+1 have disjoint windows on an iid Exp(1) map, so
    # their decisions are independent Bernoulli(Pfa): an exact binomial test.
    P = synth.square_law_map(*shape, n_targets=0, seed=12).astype(np.float64)
    tr, tc, gr, gc = win
    res = ocfar.cfar_sat(P, tr, tc, gr, gc, pfa)
    w = tr + gr
    stride = 2 * w + 1
    sel = res.det[w:shape[0] - w:stride, w:shape[1] - w:stride]
    n = sel.size
    k = int(sel.sum())
    mu = n * pfa
    sd = math.sqrt(n * pfa * (1 - pfa))
    assert abs(k - mu) < 5 * sd, (k, mu, sd)


def test_compare_decisions_margin():
    P = np.array([[1.0, 2.0], [3.0, 4.0]])
    thr = np.array([[1.0 + 1e-7, 1.0], [3.5, 4.0]])
    cut = np.ones((2, 2), dtype=bool)
    det_ref = (P > thr).astype(np.uint8)
    det = det_ref.copy()
    det[0, 0] ^= 1  # inside the margin: tolerated
    det[1, 1] ^= 1  # P == T exactly: a tie, tolerated
    c = ocfar.compare_decisions(det, det_ref, P, thr, cut)
    assert c.mismatches == 0 and c.near_ties == 2
    det[1, 0] ^= 1
    assert ocfar.compare_decisions(det, det_ref, P, thr, cut).mismatches == 1


# ------------------------------------------------------------ whole chain sanity
def test_chain_detects_planted_respiration_targets():
    # Sanity, not a pin: no dataset or printed detection map exists. Every
    # detection of the small frame lies near a planted target's range bin, and
    # the detected bins lie inside the respiration band around f * N / fs.
    case = synth.small_frame_case(seed=0)
    X, truth = synth.radar_frame(case.spec, return_truth=True)
    w = case.window
    P, band, res = oracle.run_chain(X, synth.FS_HZ, case.mean_len, w.train_r, w.train_c,
                                    w.guard_r, w.guard_c, w.pfa)
    assert P.shape == (256, band.cols)
    rows, cols = np.nonzero(res.det)
    assert len(rows) > 0
    for r, c in zip(rows, cols):
        k = c + band.c0
        assert band.k_lo <= k <= band.k_hi
        near = np.min(np.abs(truth.target_bins - r))
        assert near <= 12, (r, truth.target_bins)


# ---- square-law detector and per-range-bin z-score (next-step variants) ----

def test_square_law_pure_tone_closed_form():
    # a real tone a cos(2 pi k0 n / N) has |DFT| = a N / 2 at bin k0: square law (a N / 2)^2
    N, k0, a = 256, 9, 0.75
    n = np.arange(N)
    Y = (a * np.cos(2 * np.pi * k0 * n / N))[None, :]
    P = oracle.preprocess.band_dft_magnitude(Y, 0, 20)
    assert abs(P[0, k0] - a * N / 2) < 1e-9 * N
    spec = synth.FrameSpec(M=32, N=N, n_targets=1, seed=4)
    X = synth.radar_frame(spec)
    Pm, _ = oracle.preprocess_frame(X, synth.FS_HZ, 5, halo=4)
    Ps, _ = oracle.preprocess_frame(X, synth.FS_HZ, 5, halo=4, detector="square")
    np.testing.assert_allclose(Ps, Pm * Pm, rtol=1e-13, atol=0)


def test_row_zscore_invariants():
    rng = np.random.default_rng(8)
    Y = rng.standard_normal((6, 200)) * 3.0 + 2.0
    Y[3] = 5.0  # a constant row stays zero
    Z = oracle.normalise_row_zscore(Y)
    ok = np.arange(6) != 3
    np.testing.assert_allclose(Z[ok].mean(axis=1), 0.0, atol=1e-12)
    np.testing.assert_allclose(Z[ok].std(axis=1), 1.0, rtol=1e-12)
    assert np.all(Z[3] == 0)
    # invariant to a positive scale and an offset per row
    s = rng.uniform(0.5, 4.0, size=(6, 1))
    o = rng.uniform(-3, 3, size=(6, 1))
    np.testing.assert_allclose(oracle.normalise_row_zscore(Y * s + o)[ok], Z[ok], atol=1e-12)
    # Parseval on the full spectrum of a z-scored row: sum_k |Z_k|^2 = N sum_n z^2 = N^2
    N = Y.shape[1]
    F = np.fft.fft(Z[0])
    assert abs(np.sum(np.abs(F) ** 2) - N * N) < 1e-8 * N * N


def test_row_zscore_chain_is_scale_invariant():
    # the chain is linear up to the normalisation: scaling the raw frame by a
    # positive factor leaves every z-scored row, hence P, unchanged
    spec = synth.FrameSpec(M=24, N=300, n_targets=2, seed=6)
    X = synth.radar_frame(spec)
    P1, _ = oracle.preprocess_frame(X, synth.FS_HZ, 5, halo=6, normalisation="row_zscore")
    P2, _ = oracle.preprocess_frame(X.astype(np.float64) * 3.5, synth.FS_HZ, 5, halo=6, normalisation="row_zscore")
    np.testing.assert_allclose(P2, P1, rtol=1e-10, atol=1e-12)
    with pytest.raises(ValueError):
        oracle.preprocess_frame(X, synth.FS_HZ, 5, detector="log")


# ------------------------------------------------------------ greatest-of / smallest-of CFAR
def _law_by_quadrature(t, n, kind):
    # E[exp(-t Z)], Z = min or max of two iid Gamma(n, 1), from the order
    # statistic densities 2 f (1 - F) and 2 f F, integrated numerically.
    from scipy import integrate, stats
    g = stats.gamma(n)
    if kind == ocfar.SO:
        dens = lambda x: 2.0 * g.pdf(x) * g.sf(x)
    else:
        dens = lambda x: 2.0 * g.pdf(x) * g.cdf(x)
    val, _ = integrate.quad(lambda x: math.exp(-t * x) * dens(x), 0.0, np.inf, limit=400, epsabs=0, epsrel=1e-11)
    return val


@pytest.mark.parametrize("n", [1, 3, 12, 40])
def test_go_so_law_matches_quadrature(n):
    pytest.importorskip("scipy")
    for t in (0.05, 0.3, 1.0, 4.0):
        so = ocfar.pfa_smallest_of(t, n)
        go = ocfar.pfa_greatest_of(t, n)
        assert abs(so - _law_by_quadrature(t, n, ocfar.SO)) <= 1e-8 * so + 1e-300
        assert abs(go - _law_by_quadrature(t, n, ocfar.GO)) <= 1e-8 * go + 1e-300
        assert go < so  # the larger half sum gives the higher threshold


def test_go_so_factor_inverts_law_and_limits():
    for n, pfa in [(1, 1e-2), (20, 1e-3), (112, 1e-4), (800, 1e-6)]:
        tg = ocfar.go_so_factor(ocfar.GO, n, pfa)
        ts = ocfar.go_so_factor(ocfar.SO, n, pfa)
        assert abs(ocfar.pfa_greatest_of(tg, n) - pfa) <= 1e-10 * pfa
        assert abs(ocfar.pfa_smallest_of(ts, n) - pfa) <= 1e-10 * pfa
        assert ts > tg > 0
    # n = 1: min of two Exp(1) is Exp(2), so P_SO = 2 / (2 + t) and t = 2 / pfa - 2
    assert abs(ocfar.go_so_factor(ocfar.SO, 1, 0.01) - 198.0) < 1e-9
    # many cells: min, max and the mean of each half concentrate at n, so
    # n t -> -ln(pfa), the cell-averaging limit
    for kind in (ocfar.GO, ocfar.SO):
        nt = 4000 * ocfar.go_so_factor(kind, 4000, 1e-3)
        assert abs(nt - (-math.log(1e-3))) < 0.05 * -math.log(1e-3)
    # the two halves plus the CUT row's 2 T_c training cells make up the ring
    for tr, tc, gr, gc in [(4, 4, 1, 1), (3, 5, 1, 2), (16, 16, 4, 4), (2, 7, 0, 3)]:
        assert 2 * ocfar.half_cells(tr, tc, gr, gc) + 2 * tc == ocfar.n_ref(tr, tc, gr, gc)
    assert ocfar.half_cells(3, 5, 1, 2) == 4 * 15 - 1 * 5


def test_go_so_halves_by_hand():
    # 9 x 9 map, one interior CUT at (4, 4) with train 2 / guard 1 on both axes
    # (outer half-sizes 3): cells in the CUT's row never count; a cell in rows
    # 1..3 outside the guard box counts in the leading half only.
    tr, gd = 2, 1
    t_go = ocfar.go_so_factor(ocfar.GO, ocfar.half_cells(tr, tr, gd, gd), 1e-3)
    for kind in (ocfar.GO, ocfar.SO):
        P = np.zeros((7, 7))
        P[3, 3] = 1e-30
        P[3, 0] = 5.0  # CUT row training cell: in neither half
        for fn in (ocfar.cfar_go_so_direct, ocfar.cfar_go_so_sat):
            res = fn(P, kind, tr, tr, gd, gd, 1e-3)
            assert res.cut.sum() == 1 and res.thr[3, 3] == 0.0 and res.det[3, 3] == 1
        P[1, 3] = 2.0  # leading half, outside the guard rows
        P[2, 3] = 100.0  # inside the guard box: ignored
        P[6, 6] = 0.5  # lagging half corner
        for fn in (ocfar.cfar_go_so_direct, ocfar.cfar_go_so_sat):
            res = fn(P, kind, tr, tr, gd, gd, 1e-3)
            want = 2.0 if kind == ocfar.GO else 0.5
            t = ocfar.go_so_factor(kind, ocfar.half_cells(tr, tr, gd, gd), 1e-3)
            assert abs(res.thr[3, 3] - t * want) <= 1e-12 * t * want
    assert t_go > 0


def test_go_so_direct_equals_sat_random_maps():
    rng = np.random.default_rng(21)
    for kind in (ocfar.GO, ocfar.SO):
        for shape, win in [((40, 50), (3, 2, 1, 2, 1e-2)), ((64, 31), (8, 8, 2, 2, 1e-4)),
                           ((25, 25), (4, 4, 0, 0, 1e-1))]:
            P = rng.exponential(size=shape)
            P[rng.integers(0, shape[0], 5), rng.integers(0, shape[1], 5)] += 30
            d = ocfar.cfar_go_so_direct(P, kind, *win)
            s = ocfar.cfar_go_so_sat(P, kind, *win)
            np.testing.assert_allclose(s.thr, d.thr, rtol=1e-12, atol=1e-12)
            cmp = ocfar.compare_decisions(s.det, d.det, P, d.thr, d.cut, margin=1e-9)
            assert cmp.mismatches == 0
            base = s.det
            np.testing.assert_array_equal(ocfar.cfar_go_so_sat(P * 2.0 ** 9, kind, *win).det, base)


def test_go_so_clutter_edge_behaviour():
    # A step in the noise level along rows: GO takes the noisier half, so its
    # threshold is never below the cell-averaging one near the edge and it
    # raises no more alarms there. SO takes the quieter half, so a target
    # beside a strong interferer in one half stays detected where cell
    # averaging loses it.
    rng = np.random.default_rng(22)
    P = rng.exponential(size=(80, 60))
    P[40:] *= 100.0
    go = ocfar.cfar_go_so_sat(P, ocfar.GO, 6, 6, 1, 1, 1e-3)
    ca = ocfar.cfar_sat(P, 6, 6, 1, 1, 1e-3)
    assert go.det.sum() <= ca.det.sum()
    Q = rng.exponential(size=(60, 60))
    Q[30, 30] += 60.0
    Q[33, 27:34] += 4000.0  # interferer inside the lagging half only
    so = ocfar.cfar_go_so_sat(Q, ocfar.SO, 6, 6, 1, 1, 1e-4)
    ca = ocfar.cfar_sat(Q, 6, 6, 1, 1, 1e-4)
    assert so.det[30, 30] == 1 and ca.det[30, 30] == 0


@pytest.mark.parametrize("kind", ["go", "so"])
def test_go_so_monte_carlo_false_alarm_rate(kind):
    # Disjoint windows on an iid Exp(1) map: independent Bernoulli(Pfa) CUTs.
    pfa, shape, (tr, tc, gr, gc) = 1e-2, (2200, 2200), (4, 4, 1, 1)
    P = synth.square_law_map(*shape, n_targets=0, seed=23).astype(np.float64)
    res = ocfar.cfar_go_so_sat(P, kind, tr, tc, gr, gc, pfa)
    w = tr + gr
    stride = 2 * w + 1
    sel = res.det[w:shape[0] - w:stride, w:shape[1] - w:stride]
    n = sel.size
    k = int(sel.sum())
    mu = n * pfa
    sd = math.sqrt(n * pfa * (1 - pfa))
    assert abs(k - mu) < 5 * sd, (k, mu, sd)


# ------------------------------------------------------------ ordered-statistic CFAR
@pytest.mark.parametrize("n,k", [(8, 6), (72, 54), (112, 84), (400, 1), (400, 400)])
def test_os_law_matches_beta_function_form(n, k):
    # X_(k) = -ln(1 - U_(k)) with U_(k) ~ Beta(k, n - k + 1), so
    # E[exp(-a X_(k))] = E[(1 - U)^a] = B(k, n - k + 1 + a) / B(k, n - k + 1)
    special = pytest.importorskip("scipy.special")
    for a in (0.01, 0.5, 3.0, 40.0):
        want = math.exp(special.betaln(k, n - k + 1 + a) - special.betaln(k, n - k + 1))
        got = ocfar.pfa_ordered_statistic(a, n, k)
        assert abs(got - want) <= 1e-10 * want


def test_os_factor_inverts_law_and_closed_forms():
    for n, k, pfa in [(8, 6, 1e-2), (112, 84, 1e-4), (1600, 1200, 1e-6)]:
        a = ocfar.os_factor(n, k, pfa)
        assert abs(ocfar.pfa_ordered_statistic(a, n, k) - pfa) <= 1e-10 * pfa
    # k = 1: X_(1) ~ Exp(n), P = n / (n + a)
    assert abs(ocfar.os_factor(50, 1, 0.01) - 50 * 99) <= 1e-8 * 50 * 99
    assert ocfar.os_rank_default(112) == 84 and ocfar.os_rank_default(8) == 6 and ocfar.os_rank_default(1) == 1


def test_os_hand_example():
    # 5 x 5 map, train 1 / guard 0: the ring of the centre CUT holds 1..8, so
    # X_(6) = 6 and T = alpha 6
    P = np.zeros((5, 5))
    ring = [(1, 1), (1, 2), (1, 3), (2, 1), (2, 3), (3, 1), (3, 2), (3, 3)]
    vals = [5.0, 2.0, 8.0, 1.0, 7.0, 3.0, 6.0, 4.0]
    for (r, c), v in zip(ring, vals):
        P[r, c] = v
    a = ocfar.os_factor(8, 6, 1e-2)
    P[2, 2] = 6.0 * a * 1.01
    res = ocfar.cfar_os_direct(P, 1, 1, 0, 0, 1e-2)
    assert res.cut.sum() == 9
    assert abs(res.thr[2, 2] - 6.0 * a) <= 1e-12 * a and res.det[2, 2] == 1
    res = ocfar.cfar_os_direct(P, 1, 1, 0, 0, 1e-2, k=2)
    assert abs(res.thr[2, 2] - 2.0 * ocfar.os_factor(8, 2, 1e-2)) <= 1e-12 * res.thr[2, 2]


def test_os_robust_to_one_interferer_and_scale_invariant():
    rng = np.random.default_rng(31)
    Q = rng.exponential(size=(60, 60))
    Q[30, 30] += 60.0
    Q[33, 27] += 1e5  # one strong cell in the CUT's window
    os_ = ocfar.cfar_os_direct(Q, 6, 6, 1, 1, 1e-4)
    ca = ocfar.cfar_sat(Q, 6, 6, 1, 1, 1e-4)
    assert os_.det[30, 30] == 1 and ca.det[30, 30] == 0
    np.testing.assert_array_equal(ocfar.cfar_os_direct(Q * 2.0 ** 7, 6, 6, 1, 1, 1e-4).det, os_.det)


def test_os_monte_carlo_false_alarm_rate():
    # disjoint windows on an iid Exp(1) map: independent Bernoulli(Pfa) CUTs
    pfa, shape, (tr, tc, gr, gc) = 2e-2, (1100, 1100), (4, 4, 1, 1)
    P = synth.square_law_map(*shape, n_targets=0, seed=33).astype(np.float64)
    res = ocfar.cfar_os_direct(P, tr, tc, gr, gc, pfa)
    w = tr + gr
    stride = 2 * w + 1
    sel = res.det[w:shape[0] - w:stride, w:shape[1] - w:stride]
    n = sel.size
    k = int(sel.sum())
    mu = n * pfa
    sd = math.sqrt(n * pfa * (1 - pfa))
    assert abs(k - mu) < 5 * sd, (k, mu, sd)
