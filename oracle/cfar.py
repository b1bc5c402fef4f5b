"""FP64 2D CA-CFAR, summed-area table and four-corner sums (paper Sec. II.B).

Test infrastructure: imported only by tests, the smoke check and the CPU
baseline of the benchmark. Never by the product path.

Readings of the paper (Sec. II.B, eqs. 1-4) taken here:
  * eq. 2 prints alpha = N (Pfa^{1/N} - 1), which is negative for Pfa < 1.
    The exponent's sign is a misprint: alpha = N (Pfa^{-1/N} - 1), the factor
    for which a cell-averaging CFAR on iid exponential (square-law) noise has
    false-alarm probability exactly Pfa. The printed form is kept as
    `alpha_as_printed` for the record.
  * The "N" of eq. 2 (reference-cell count) is written n_ref here; it is not
    the slow-time length N of Sec. II.A.
  * "A" is the average of the reference cells in eq. 2 but a region sum in
    eq. 4: S_ref is the sum, A = S_ref / n_ref, T = alpha * A.
  * eq. 1 leaves CUT == T undefined: it decides H0 (detection iff CUT > T).
  * Window: per-side counts per dimension. The guard rectangle
    [r - G_r, r + G_r] x [c - G_c, c + G_c] contains the CUT; the training
    ring lies between it and the outer rectangle with half-sizes
    W_r = G_r + T_r, W_c = G_c + T_c. n_ref = (2W_r+1)(2W_c+1) - (2G_r+1)(2G_c+1).
  * Edge policy: only interior CUTs (outer rectangle fully inside the map)
    are tested; every other cell decides H0. CUT columns may further be
    restricted to a column range (the respiration band).
  * eq. 4 corner labels (Fig. 2 is missing; Viola-Jones labelling): for the
    rectangle [r0, r1] x [c0, c1], L1 = S(r0-1, c0-1), L2 = S(r0-1, c1),
    L3 = S(r1, c0-1), L4 = S(r1, c1), with S(-1, .) = S(., -1) = 0, so that
    the region sum is L1 + L4 - (L2 + L3).
"""
from __future__ import annotations

from typing import NamedTuple, Optional, Tuple

import numpy as np

from .preprocess import preprocess_frame


def n_ref(train_r: int, train_c: int, guard_r: int, guard_c: int) -> int:
    """Number of reference (training) cells around a CUT (Sec. II.B)."""
    wr, wc = guard_r + train_r, guard_c + train_c
    return (2 * wr + 1) * (2 * wc + 1) - (2 * guard_r + 1) * (2 * guard_c + 1)


def alpha(nref: int, pfa: float) -> float:
    """Threshold factor of eq. 2 with the exponent's sign corrected.

    alpha = n_ref * (Pfa^(-1/n_ref) - 1)
    """
    if nref <= 0 or not (0.0 < pfa < 1.0):
        raise ValueError("need n_ref > 0 and 0 < pfa < 1")
    return nref * (pfa ** (-1.0 / nref) - 1.0)


def alpha_as_printed(nref: int, pfa: float) -> float:
    """eq. 2 exactly as printed (negative for Pfa < 1; recorded, not used)."""
    return nref * (pfa ** (1.0 / nref) - 1.0)


def sat(P: np.ndarray) -> np.ndarray:
    """Summed-area table by the recurrence of eq. 3.

    s(r, c) = i(r, c) + s(r-1, c) + s(r, c-1) - s(r-1, c-1), with s = 0 outside.
    Rows are produced in order; within a row the dependence on s(r, c-1) is a
    running sum of d(c) = i(r, c) + s(r-1, c) - s(r-1, c-1).
    """
    P = np.asarray(P, dtype=np.float64)
    R, C = P.shape
    S = np.zeros((R, C), dtype=np.float64)
    prev = np.zeros(C + 1)  # s(r-1, c-1 .. C-1) with a leading 0 for c = -1
    for r in range(R):
        d = P[r] + prev[1:] - prev[:-1]
        row = np.cumsum(d)
        S[r] = row
        prev[1:] = row
    return S


def _at(S: np.ndarray, r, c):
    """S(r, c) with S(-1, .) = S(., -1) = 0 (vectorised over r, c arrays)."""
    r = np.asarray(r)
    c = np.asarray(c)
    ok = (r >= 0) & (c >= 0)
    out = np.zeros(np.broadcast(r, c).shape, dtype=np.float64)
    rr = np.broadcast_to(r, out.shape)
    cc = np.broadcast_to(c, out.shape)
    out[ok] = S[rr[ok], cc[ok]]
    return out


def box_sum(S: np.ndarray, r0, r1, c0, c1):
    """Region sum over [r0, r1] x [c0, c1] from four SAT corners (eq. 4).

    A = L1 + L4 - (L2 + L3), L1 = S(r0-1, c0-1), L2 = S(r0-1, c1),
    L3 = S(r1, c0-1), L4 = S(r1, c1).
    """
    L1 = _at(S, np.asarray(r0) - 1, np.asarray(c0) - 1)
    L2 = _at(S, np.asarray(r0) - 1, c1)
    L3 = _at(S, r1, np.asarray(c0) - 1)
    L4 = _at(S, r1, c1)
    return L1 + L4 - (L2 + L3)


class CfarResult(NamedTuple):
    det: np.ndarray  # uint8, 1 = H1
    thr: np.ndarray  # float64 threshold T at CUTs, 0 elsewhere
    cut: np.ndarray  # bool mask of tested CUTs


def _cut_mask(shape, train_r, train_c, guard_r, guard_c, cut_cols: Optional[Tuple[int, int]]):
    R, C = shape
    wr, wc = guard_r + train_r, guard_c + train_c
    mask = np.zeros((R, C), dtype=bool)
    r_lo, r_hi = wr, R - 1 - wr
    c_lo, c_hi = wc, C - 1 - wc
    if cut_cols is not None:
        c_lo = max(c_lo, cut_cols[0])
        c_hi = min(c_hi, cut_cols[1])
    if r_lo <= r_hi and c_lo <= c_hi:
        mask[r_lo:r_hi + 1, c_lo:c_hi + 1] = True
    return mask


def cfar_direct(P: np.ndarray, train_r: int, train_c: int, guard_r: int, guard_c: int, pfa: float,
                cut_cols: Optional[Tuple[int, int]] = None) -> CfarResult:
    """Direct sliding-window 2D CA-CFAR (Sec. II.B, eqs. 1-2; Table I "CA-CFAR").

    For every interior CUT, S_ref is the explicit FP64 sum of its n_ref
    training cells (outer rectangle minus guard rectangle), T = alpha * S_ref
    / n_ref and the decision is CUT > T.
    """
    P = np.asarray(P, dtype=np.float64)
    R, C = P.shape
    wr, wc = guard_r + train_r, guard_c + train_c
    nr = n_ref(train_r, train_c, guard_r, guard_c)
    a = alpha(nr, pfa)
    mask = _cut_mask(P.shape, train_r, train_c, guard_r, guard_c, cut_cols)
    det = np.zeros((R, C), dtype=np.uint8)
    thr = np.zeros((R, C), dtype=np.float64)
    if not mask.any():
        return CfarResult(det, thr, mask)
    rs, cs = np.nonzero(mask)
    r_lo, r_hi, c_lo, c_hi = rs.min(), rs.max(), cs.min(), cs.max()
    sref = np.zeros((r_hi - r_lo + 1, c_hi - c_lo + 1))
    # sum the reference cells one offset at a time
    for dr in range(-wr, wr + 1):
        for dc in range(-wc, wc + 1):
            if abs(dr) <= guard_r and abs(dc) <= guard_c:
                continue
            sref += P[r_lo + dr:r_hi + 1 + dr, c_lo + dc:c_hi + 1 + dc]
    T = a * sref / nr
    blk = mask[r_lo:r_hi + 1, c_lo:c_hi + 1]
    cut = P[r_lo:r_hi + 1, c_lo:c_hi + 1]
    thr[r_lo:r_hi + 1, c_lo:c_hi + 1] = np.where(blk, T, 0.0)
    det[r_lo:r_hi + 1, c_lo:c_hi + 1] = (blk & (cut > T)).astype(np.uint8)
    return CfarResult(det, thr, mask)


def cfar_direct_at(P: np.ndarray, rows, cols, train_r: int, train_c: int, guard_r: int, guard_c: int,
                   pfa: float):
    """Direct CA-CFAR at a list of interior CUTs (one explicit window sum each).

    Returns (det, thr) arrays aligned with rows/cols. Used for sampled checks on
    maps too large for the full sliding window.
    """
    P = np.asarray(P)
    wr, wc = guard_r + train_r, guard_c + train_c
    nr = n_ref(train_r, train_c, guard_r, guard_c)
    a = alpha(nr, pfa)
    det = np.zeros(len(rows), dtype=np.uint8)
    thr = np.zeros(len(rows))
    for i, (r, c) in enumerate(zip(rows, cols)):
        outer = P[r - wr:r + wr + 1, c - wc:c + wc + 1].astype(np.float64).sum()
        guard = P[r - guard_r:r + guard_r + 1, c - guard_c:c + guard_c + 1].astype(np.float64).sum()
        T = a * (outer - guard) / nr
        thr[i] = T
        det[i] = 1 if float(P[r, c]) > T else 0
    return det, thr


def cfar_sat(P: np.ndarray, train_r: int, train_c: int, guard_r: int, guard_c: int, pfa: float,
             cut_cols: Optional[Tuple[int, int]] = None, S: Optional[np.ndarray] = None) -> CfarResult:
    """SAT ("integral image") 2D CA-CFAR (Sec. II.B, eqs. 3-4; Table I "II CA-CFAR").

    S_ref = A(outer rectangle) - A(guard rectangle), each from eq. 4 on the
    eq. 3 table; T = alpha * S_ref / n_ref; decision CUT > T.
    """
    P = np.asarray(P, dtype=np.float64)
    R, C = P.shape
    if S is None:
        S = sat(P)
    wr, wc = guard_r + train_r, guard_c + train_c
    nr = n_ref(train_r, train_c, guard_r, guard_c)
    a = alpha(nr, pfa)
    mask = _cut_mask(P.shape, train_r, train_c, guard_r, guard_c, cut_cols)
    det = np.zeros((R, C), dtype=np.uint8)
    thr = np.zeros((R, C), dtype=np.float64)
    if not mask.any():
        return CfarResult(det, thr, mask)
    rs, cs = np.nonzero(mask)
    outer = box_sum(S, rs - wr, rs + wr, cs - wc, cs + wc)
    guard = box_sum(S, rs - guard_r, rs + guard_r, cs - guard_c, cs + guard_c)
    T = a * (outer - guard) / nr
    thr[rs, cs] = T
    det[rs, cs] = (P[rs, cs] > T).astype(np.uint8)
    return CfarResult(det, thr, mask)


class Comparison(NamedTuple):
    mismatches: int  # decisions that differ outside the margin
    near_ties: int  # tested CUTs with |CUT - T| / T < margin (not compared)
    compared: int


def compare_decisions(det: np.ndarray, det_ref: np.ndarray, P_ref: np.ndarray, thr_ref: np.ndarray,
                      cut_mask: np.ndarray, margin: float = 1e-5) -> Comparison:
    """Decision parity with a tie margin.

    Cells whose reference CUT value is within `margin` relative of the
    reference threshold are counted as near ties and not compared; every other
    cell (CUT or not) must agree exactly.
    """
    det = np.asarray(det).astype(np.uint8)
    det_ref = np.asarray(det_ref).astype(np.uint8)
    P_ref = np.asarray(P_ref, dtype=np.float64)
    thr_ref = np.asarray(thr_ref, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.abs(P_ref - thr_ref) / np.abs(thr_ref)
    tie = cut_mask & (rel < margin)
    diff = (det != det_ref) & ~tie
    return Comparison(int(diff.sum()), int(tie.sum()), int(det.size - tie.sum()))


def cfar_chain(P: np.ndarray, band, train_r: int, train_c: int, guard_r: int, guard_c: int, pfa: float,
               method: str = "sat", kind: str = "ca") -> CfarResult:
    """CFAR on a band map: CUT columns restricted to the respiration band bins.
    kind: "ca" (Sec. II.B), or the greatest-of / smallest-of / ordered-statistic
    variants "go", "so", "os" (default rank)."""
    cut_cols = (band.k_lo - band.c0, band.k_hi - band.c0)
    if kind == OS:
        return cfar_os_direct(P, train_r, train_c, guard_r, guard_c, pfa, cut_cols=cut_cols)
    if kind != "ca":
        fn = cfar_go_so_sat if method == "sat" else cfar_go_so_direct
        return fn(P, kind, train_r, train_c, guard_r, guard_c, pfa, cut_cols=cut_cols)
    fn = cfar_sat if method == "sat" else cfar_direct
    return fn(P, train_r, train_c, guard_r, guard_c, pfa, cut_cols=cut_cols)


def run_chain(X: np.ndarray, fs_hz: float, mean_len: int, train_r: int, train_c: int, guard_r: int,
              guard_c: int, pfa: float, method: str = "sat"):
    """Raw frame -> (P, band, CfarResult): the whole data path of Sec. II."""
    P, band = preprocess_frame(X, fs_hz, mean_len, halo=train_c + guard_c)
    res = cfar_chain(P, band, train_r, train_c, guard_r, guard_c, pfa, method)
    return P, band, res


# ---- greatest-of / smallest-of CFAR (next-step variants; not in the paper) ----
#
# Reading (recorded in the design notes): the training cells are split along
# range into a leading half (the outer window's rows r - wr .. r - 1 minus the
# guard rows r - gr .. r - 1) and a lagging half (rows r + 1 .. r + wr minus
# r + 1 .. r + gr); the training cells of the CUT's own row belong to
# neither. Each half holds n = wr (2 wc + 1) - gr (2 gc + 1) cells.
# GO: T = t * max(S_lead, S_lag); SO: T = t * min(S_lead, S_lag), with t the
# multiplier of the half SUM that gives the requested Pfa on iid exponential
# (square-law) noise of any mean: for X, Y ~ Gamma(n, 1) independent and the
# CUT ~ Exp(1), P(CUT > t min(X, Y)) = E[exp(-t min(X, Y))]
#   = 2 sum_{k=0}^{n-1} C(n-1+k, k) (2 + t)^-(n+k)
# and, with 1 - F of Gamma(n, 1) written as the tail of a Poisson sum,
#   P(CUT > t max(X, Y)) = 2 sum_{k>=n} C(n-1+k, k) (2 + t)^-(n+k),
# a series of positive terms (no cancellation); the two laws add up to
# E[e^{-tX}] + E[e^{-tY}] = 2 (1 + t)^-n.

GO, SO = "go", "so"


def half_cells(train_r: int, train_c: int, guard_r: int, guard_c: int) -> int:
    wr, wc = guard_r + train_r, guard_c + train_c
    return wr * (2 * wc + 1) - guard_r * (2 * guard_c + 1)


def _log_term(n: int, k: int, l2t: float) -> float:
    from math import lgamma
    return lgamma(n + k) - lgamma(k + 1) - lgamma(n) - (n + k) * l2t


def pfa_smallest_of(t: float, n: int) -> float:
    """P(CUT > t min(X, Y)) for CUT ~ Exp(1), X, Y ~ Gamma(n, 1)."""
    if n <= 0 or t < 0:
        raise ValueError("need n > 0 and t >= 0")
    from math import exp, log
    l2t = log(2.0 + t)
    return 2.0 * sum(exp(_log_term(n, k, l2t)) for k in range(n))


def pfa_greatest_of(t: float, n: int) -> float:
    """P(CUT > t max(X, Y)): the series over k >= n, summed until its terms,
    which shrink by (n + k) / ((k + 1)(2 + t)) < 1 from there on, are below
    1e-18 of the total."""
    if n <= 0 or t < 0:
        raise ValueError("need n > 0 and t >= 0")
    from math import exp, log
    l2t = log(2.0 + t)
    acc, k = 0.0, n
    while True:
        term = exp(_log_term(n, k, l2t))
        acc += term
        k += 1
        if (n + k) < (k + 1) * (2.0 + t) and term <= 1e-18 * acc:
            break
    return 2.0 * acc


def go_so_factor(kind: str, n: int, pfa: float) -> float:
    """Multiplier t of the half sum for the requested Pfa (bisection in FP64;
    both false-alarm laws decrease in t)."""
    if kind not in (GO, SO) or n <= 0 or not (0.0 < pfa < 1.0):
        raise ValueError("bad GO/SO request")
    f = pfa_greatest_of if kind == GO else pfa_smallest_of
    lo, hi = 0.0, 1.0
    while f(hi, n) > pfa:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid, n) > pfa:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-15 * hi:
            break
    return 0.5 * (lo + hi)


def _halves_direct(P, rs, cs, train_r, train_c, guard_r, guard_c):
    wr, wc = guard_r + train_r, guard_c + train_c
    lead = np.zeros(rs.shape)
    lag = np.zeros(rs.shape)
    for dr in range(1, wr + 1):
        for dc in range(-wc, wc + 1):
            if dr <= guard_r and abs(dc) <= guard_c:
                continue
            lead += P[rs - dr, cs + dc]
            lag += P[rs + dr, cs + dc]
    return lead, lag


def cfar_go_so_direct(P: np.ndarray, kind: str, train_r: int, train_c: int, guard_r: int, guard_c: int,
                      pfa: float, cut_cols: Optional[Tuple[int, int]] = None) -> CfarResult:
    """GO / SO CFAR with each half summed cell by cell (FP64)."""
    P = np.asarray(P, dtype=np.float64)
    n = half_cells(train_r, train_c, guard_r, guard_c)
    t = go_so_factor(kind, n, pfa)
    mask = _cut_mask(P.shape, train_r, train_c, guard_r, guard_c, cut_cols)
    det = np.zeros(P.shape, dtype=np.uint8)
    thr = np.zeros(P.shape, dtype=np.float64)
    if not mask.any():
        return CfarResult(det, thr, mask)
    rs, cs = np.nonzero(mask)
    lead, lag = _halves_direct(P, rs, cs, train_r, train_c, guard_r, guard_c)
    T = t * (np.maximum(lead, lag) if kind == GO else np.minimum(lead, lag))
    thr[rs, cs] = T
    det[rs, cs] = (P[rs, cs] > T).astype(np.uint8)
    return CfarResult(det, thr, mask)


def cfar_go_so_sat(P: np.ndarray, kind: str, train_r: int, train_c: int, guard_r: int, guard_c: int,
                   pfa: float, cut_cols: Optional[Tuple[int, int]] = None, S: Optional[np.ndarray] = None) -> CfarResult:
    """GO / SO CFAR with each half from eq. 4 on the eq. 3 table: half =
    A(outer rows of the half) - A(guard rows of the half)."""
    P = np.asarray(P, dtype=np.float64)
    if S is None:
        S = sat(P)
    wr, wc = guard_r + train_r, guard_c + train_c
    n = half_cells(train_r, train_c, guard_r, guard_c)
    t = go_so_factor(kind, n, pfa)
    mask = _cut_mask(P.shape, train_r, train_c, guard_r, guard_c, cut_cols)
    det = np.zeros(P.shape, dtype=np.uint8)
    thr = np.zeros(P.shape, dtype=np.float64)
    if not mask.any():
        return CfarResult(det, thr, mask)
    rs, cs = np.nonzero(mask)
    lead = box_sum(S, rs - wr, rs - 1, cs - wc, cs + wc) - box_sum(S, rs - guard_r, rs - 1, cs - guard_c, cs + guard_c)
    lag = box_sum(S, rs + 1, rs + wr, cs - wc, cs + wc) - box_sum(S, rs + 1, rs + guard_r, cs - guard_c, cs + guard_c)
    T = t * (np.maximum(lead, lag) if kind == GO else np.minimum(lead, lag))
    thr[rs, cs] = T
    det[rs, cs] = (P[rs, cs] > T).astype(np.uint8)
    return CfarResult(det, thr, mask)


# ---- ordered-statistic CFAR (next-step variant; not in the paper) ----
#
# Reading (recorded in the design notes): the reference set is the same
# training ring as cell averaging (n_ref cells); T = alpha * X_(k), X_(k)
# the k-th smallest reference value (1-based), k = ceil(3 n_ref / 4) unless
# given. For iid exponential noise the k-th order statistic of n cells is a
# sum of independent exponentials with rates n, n-1, ..., n-k+1 (Renyi), so
#   P(CUT > alpha X_(k)) = prod_{i=0}^{k-1} (n - i) / (n - i + alpha),
# which falls monotonically in alpha; alpha comes by bisection. An order
# statistic is not a region sum, so this variant cannot use the eq. 3 table.
OS = "os"


def os_rank_default(nref: int) -> int:
    return -(-3 * nref // 4)


def pfa_ordered_statistic(alpha: float, n: int, k: int) -> float:
    """P(CUT > alpha X_(k)) for n iid Exp(1) reference cells (log-space product)."""
    if not (1 <= k <= n) or alpha < 0:
        raise ValueError("need 1 <= k <= n and alpha >= 0")
    from math import exp, log1p
    return exp(-sum(log1p(alpha / (n - i)) for i in range(k)))


def os_factor(n: int, k: int, pfa: float) -> float:
    """alpha with pfa_ordered_statistic(alpha, n, k) = pfa (bisection in FP64)."""
    if not (0.0 < pfa < 1.0):
        raise ValueError("need 0 < pfa < 1")
    lo, hi = 0.0, 1.0
    while pfa_ordered_statistic(hi, n, k) > pfa:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if pfa_ordered_statistic(mid, n, k) > pfa:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-15 * hi:
            break
    return 0.5 * (lo + hi)


def cfar_os_direct(P: np.ndarray, train_r: int, train_c: int, guard_r: int, guard_c: int, pfa: float,
                   k: Optional[int] = None, cut_cols: Optional[Tuple[int, int]] = None) -> CfarResult:
    """OS CFAR: the k-th smallest of each CUT's n_ref training cells, times alpha (FP64)."""
    P = np.asarray(P, dtype=np.float64)
    nref = n_ref(train_r, train_c, guard_r, guard_c)
    if k is None or k == 0:
        k = os_rank_default(nref)
    alpha_os = os_factor(nref, k, pfa)
    wr, wc = guard_r + train_r, guard_c + train_c
    yy, xx = np.mgrid[-wr:wr + 1, -wc:wc + 1]
    ring = ~((np.abs(yy) <= guard_r) & (np.abs(xx) <= guard_c))
    dr, dc = yy[ring], xx[ring]
    mask = _cut_mask(P.shape, train_r, train_c, guard_r, guard_c, cut_cols)
    det = np.zeros(P.shape, dtype=np.uint8)
    thr = np.zeros(P.shape, dtype=np.float64)
    rs, cs = np.nonzero(mask)
    for start in range(0, rs.size, 4096):  # chunks keep the gathered windows small
        r = rs[start:start + 4096, None]
        c = cs[start:start + 4096, None]
        cells = P[r + dr[None, :], c + dc[None, :]]
        xk = np.partition(cells, k - 1, axis=1)[:, k - 1]
        T = alpha_os * xk
        thr[rs[start:start + 4096], cs[start:start + 4096]] = T
        det[rs[start:start + 4096], cs[start:start + 4096]] = (P[rs[start:start + 4096], cs[start:start + 4096]] > T)
    return CfarResult(det, thr, mask)
