"""The allocation-free entry point, rcfar_sat_cfar_static.

Some callers cannot allocate device memory -- a real-time radar loop whose
memory is fixed at start-up (an allocation can synchronise the device and
stall the loop), or a host whose device memory belongs to another memory
manager -- so they cannot create a handle. This entry point keeps its scratch
in a fixed array inside the library. The test calls it through the C ABI
twice in a row, on two different maps, and checks each result against the
handle path (rcfar_sat + rcfar_cfar on an exact table) with the tolerances of
the other parity tests, and against the FP64 oracle's SAT CFAR directly; a
further call must leave the device's free memory unchanged. The file sorts
last so that a run stopping at the first failure has run every other test
first.
"""
import numpy as np
import pytest

import synth
from oracle import cfar as ocfar

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_11077_gb300 import build as b
    b.build()
    import paper_2012_11077_gb300 as pkg
    pkg.lib()
    return pkg


def handle_path(rc, P, win, cut):
    h = rc.rcfar_create(device=0, max_rows=P.shape[0], max_cols=P.shape[1], max_n=256, max_window=32)
    try:
        Pt = torch.from_numpy(P).cuda()
        v = rc.rcfar_sat(h, Pt, value_bound=float(P.max()), mode=rc.RCFAR_SAT_TILE_I64)
        det = torch.empty(P.shape, dtype=torch.uint8, device="cuda")
        thr = torch.empty(P.shape, dtype=torch.float32, device="cuda")
        rc.rcfar_cfar(h, v, Pt, win, cut[0], cut[1], det, thr)
        assert rc.rcfar_get_error(h) == rc.RCFAR_OK
        return det.cpu().numpy(), thr.cpu().numpy()
    finally:
        rc.rcfar_destroy(h)


def test_static_entry_matches_handle_path_twice(rc):
    cases = [
        (synth.square_law_map(700, 300, n_targets=40, dyn_range_db=40.0, seed=31), (8, 8, 2, 2, 1e-4), (5, 290)),
        (synth.square_law_map(257, 513, n_targets=20, dyn_range_db=60.0, seed=32), (4, 6, 1, 2, 1e-3), (0, 512)),
    ]
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for P, w, cut in cases:
        win = rc.make_window(*w)
        det_ref, thr_ref = handle_path(rc, P, win, cut)
        Pt = torch.from_numpy(P).cuda()
        det = torch.full(P.shape, 7, dtype=torch.uint8, device="cuda")
        thr = torch.full(P.shape, -1.0, dtype=torch.float32, device="cuda")
        rc.rcfar_sat_cfar_static(Pt, float(P.max()), win, cut[0], cut[1], det, thr, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        np.testing.assert_array_equal(det.cpu().numpy(), det_ref)
        t, tr = thr.cpu().numpy().astype(np.float64), thr_ref.astype(np.float64)
        assert np.all(np.abs(t - tr) <= 1e-6 * np.abs(tr))
        # and against the FP64 oracle (eq. 3 table, eq. 4 lookups), independent of the library
        o = ocfar.cfar_sat(P.astype(np.float64), *w, cut_cols=cut)
        cmp = ocfar.compare_decisions(det.cpu().numpy(), o.det, P, o.thr, o.cut, margin=1e-5)
        assert cmp.mismatches == 0, cmp
        assert np.all(np.abs(t[o.cut] - o.thr[o.cut]) <= 1e-4 * np.abs(o.thr[o.cut]))
        assert np.all(t[~o.cut] == 0.0)


def test_static_entry_allocates_no_device_memory(rc):
    P = synth.square_law_map(600, 400, n_targets=30, dyn_range_db=50.0, seed=34)
    win = rc.make_window(8, 8, 2, 2, 1e-4)
    Pt = torch.from_numpy(P).cuda()
    det = torch.empty(P.shape, dtype=torch.uint8, device="cuda")
    thr = torch.empty(P.shape, dtype=torch.float32, device="cuda")
    status = torch.zeros((1,), dtype=torch.int32, device="cuda")
    rc.rcfar_sat_cfar_static(Pt, float(P.max()), win, 0, P.shape[1] - 1, det, thr, status)  # warm: set-up done
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    torch0 = torch.cuda.memory_allocated()
    for _ in range(3):
        rc.rcfar_sat_cfar_static(Pt, float(P.max()), win, 0, P.shape[1] - 1, det, thr, status)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == torch0
    assert int(status.item()) == 0


def test_static_entry_rejects_oversized_maps_and_reports_range(rc):
    win = rc.make_window(8, 8, 2, 2, 1e-4)
    big = torch.zeros((4096, 4096), dtype=torch.float32, device="cuda")
    det = torch.empty((4096, 4096), dtype=torch.uint8, device="cuda")
    with pytest.raises(rc.RcfarError) as e:
        rc.rcfar_sat_cfar_static(big, 1.0, win, 0, 4095, det)
    assert e.value.status == rc.RCFAR_ERR_UNSUPPORTED
    P = synth.square_law_map(128, 128, n_targets=0, seed=33)
    P[5, 5] = 1e6  # above the stated bound
    status = torch.zeros((1,), dtype=torch.int32, device="cuda")
    d = torch.empty((128, 128), dtype=torch.uint8, device="cuda")
    rc.rcfar_sat_cfar_static(torch.from_numpy(P).cuda(), 100.0, win, 0, 127, d, None, status)
    torch.cuda.synchronize()
    assert int(status.item()) != 0
