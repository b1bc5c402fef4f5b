"""Fused SAT + CFAR on wide float32 maps whose rows start on 16-byte
boundaries: the streaming kernel whose stages arrive as tensor-memory-
accelerator boxes.

Every case runs rcfar_sat_cfar and the split path (rcfar_sat with the exact
I64 table, then rcfar_cfar) on the same map and asserts identical decisions
and thresholds bit for bit; decisions are also compared with the oracle's
FP64 CFAR (eq. 1, eq. 2, eq. 4 on the eq. 3 table; Sec. II.B), exact outside
the 1e-5 tie margin. The trace records which fused kernel ran: maps whose
row stride is not a multiple of 4 floats take the cp.async-fed kernel, and
the two must agree too. Cases cover ragged strips and row runs, windows up to
the widest halo the 8-column-per-lane layout holds (train + guard = 62 columns
per side), guard-free windows, partial CUT column ranges, greatest-of and
smallest-of, and the decision from the table's own CUT value.
"""
import numpy as np
import pytest

from oracle import cfar as ocfar
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MARGIN = 1e-5

CASES = [
    # (rows, cols), (train_r, train_c, guard_r, guard_c, pfa), CUT columns
    ((700, 516), (16, 16, 4, 4, 1e-6), None),
    ((1030, 392), (6, 9, 2, 3, 1e-4), (40, 350)),
    ((300, 1024), (1, 1, 0, 0, 1e-1), None),
    ((257, 260), (8, 26, 2, 4, 1e-3), (30, 200)),   # halo 30: the widest the 6-column layout holds
    ((129, 388), (5, 27, 1, 4, 1e-3), None),        # halo 31: 8 columns per lane
    ((96, 640), (3, 60, 2, 2, 1e-2), (70, 600)),    # halo 62: the widest streaming halo
    ((2000, 300), (30, 2, 8, 0, 1e-4), None),       # tall window, no guard columns
]
KINDS = [("ca", 0), ("go", 1), ("so", 2)]


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
    hd = rc.rcfar_create(device=0, max_rows=2048, max_cols=1100, max_n=256, max_window=64, max_frames=1)
    yield hd
    rc.rcfar_destroy(hd)


def stream_map(shape, seed):
    R, C = shape
    P = synth.square_law_map(R, C, n_targets=max(1, R * C // 2000), dyn_range_db=30.0, seed=seed).astype(np.float64)
    P[R // 2:] *= 100.0  # a 20 dB step: the half sums of greatest-of / smallest-of differ next to it
    return P.astype(np.float32)


def padded(P, extra):
    """P on the device in a buffer whose rows are len + extra floats apart."""
    R, C = P.shape
    buf = torch.zeros((R, C + extra), dtype=torch.float32, device="cuda")
    buf[:, :C] = torch.from_numpy(P).cuda()
    return buf[:, :C]


def run_fused(rc, h, Pt, w, lo, hi, map_cut):
    rows, cols = Pt.shape
    d = torch.full((rows, cols), 7, dtype=torch.uint8, device="cuda")
    t = torch.full((rows, cols), -1.0, dtype=torch.float32, device="cuda")
    rc.rcfar_trace_enable(h, True)
    rc.rcfar_sat_cfar(h, Pt, float(Pt.max()), w, lo, hi, d, t, map_cut=map_cut)
    tr = rc.rcfar_trace_read(h)
    rc.rcfar_trace_enable(h, False)
    assert rc.rcfar_get_error(h) == rc.RCFAR_OK
    return d, t, set(tr)


@pytest.mark.parametrize("kind,k", KINDS)
@pytest.mark.parametrize("shape,win,cut", CASES)
@pytest.mark.parametrize("map_cut", [True, False])
def test_tma_stream_equals_split_and_oracle(rc, h, kind, k, shape, win, cut, map_cut):
    P = stream_map(shape, seed=shape[0] + 3 * shape[1] + k)
    rows, cols = shape
    lo, hi = cut if cut is not None else (0, cols - 1)
    w = rc.make_window(*win, kind=k)
    Pt = padded(P, 8)  # row stride a multiple of 4 floats: the TMA-fed kernel
    d, t, fams = run_fused(rc, h, Pt, w, lo, hi, map_cut)
    assert "sat_cfar_fused_tma" in fams, fams
    view = rc.rcfar_sat(h, Pt, value_bound=float(P.max()), mode=rc.RCFAR_SAT_I64)
    d1 = torch.full((rows, cols), 7, dtype=torch.uint8, device="cuda")
    t1 = torch.full((rows, cols), -1.0, dtype=torch.float32, device="cuda")
    rc.rcfar_cfar(h, view, Pt if map_cut else None, w, lo, hi, d1, t1)
    assert rc.rcfar_get_error(h) == rc.RCFAR_OK
    assert torch.equal(d, d1) and torch.equal(t, t1)
    # the cp.async-fed kernel (row stride not a multiple of 4 floats) agrees
    d2, t2, fams2 = run_fused(rc, h, padded(P, 3), w, lo, hi, map_cut)
    assert "sat_cfar_fused_tma" not in fams2, fams2
    assert torch.equal(d, d2) and torch.equal(t, t2)
    if k == 0:
        ref = ocfar.cfar_sat(P.astype(np.float64), *win, cut_cols=cut)
    else:
        ref = ocfar.cfar_go_so_sat(P.astype(np.float64), kind, *win, cut_cols=cut)
    cmp = ocfar.compare_decisions(d.cpu().numpy(), ref.det, P, ref.thr, ref.cut, margin=MARGIN)
    assert cmp.mismatches == 0, cmp


def test_tma_stream_range_error(rc, h):
    P = torch.ones((300, 512), device="cuda")
    P[100, 300] = 1e9
    d = torch.empty((300, 512), dtype=torch.uint8, device="cuda")
    rc.rcfar_trace_enable(h, True)
    rc.rcfar_sat_cfar(h, P, 100.0, rc.make_window(4, 4, 1, 1, 1e-3), 0, 511, d)
    fams = set(rc.rcfar_trace_read(h))
    rc.rcfar_trace_enable(h, False)
    assert "sat_cfar_fused_tma" in fams
    assert rc.rcfar_get_error(h) == rc.RCFAR_ERR_RANGE
