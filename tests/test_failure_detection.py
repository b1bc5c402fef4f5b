"""Failure detection without a fault.

Every waiting kernel gives up after a bounded number of polls, records a
timeout in the status word and returns; the host reads RCFAR_ERR_TIMEOUT and
the context stays usable. The self-test entry point makes one such wait run
out on purpose (a barrier that nothing completes).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rc():
    from paper_2012_11077_gb300 import build as b
    b.build()
    import paper_2012_11077_gb300 as pkg
    pkg.lib()
    return pkg


def test_selftest_rejects_bad_bounds(rc):
    # argument checks happen before any device work (no GPU needed)
    assert rc.rcfar_selftest_wait(0, 0) == rc.RCFAR_ERR_INVALID_ARG
    assert rc.rcfar_selftest_wait(0, (1 << 20) + 1) == rc.RCFAR_ERR_INVALID_ARG


@pytest.mark.gpu
def test_bounded_wait_times_out_and_device_stays_usable(rc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    assert rc.rcfar_selftest_wait(0, 2000) == rc.RCFAR_ERR_TIMEOUT
    # the context is intact: a normal SAT + CFAR still runs and reports OK
    h = rc.rcfar_create(device=0, max_rows=256, max_cols=256, max_n=512, max_window=8)
    try:
        P = torch.from_numpy(synth.square_law_map(200, 200, n_targets=3, dyn_range_db=30.0, seed=1)).cuda()
        det = torch.empty((200, 200), dtype=torch.uint8, device="cuda")
        v = rc.rcfar_sat(h, P, value_bound=float(P.max()), mode=rc.RCFAR_SAT_I64)
        rc.rcfar_cfar(h, v, P, rc.make_window(4, 4, 1, 1, 1e-3), 0, 199, det)
        assert rc.rcfar_get_error(h) == rc.RCFAR_OK
        assert int(det.sum()) >= 1
    finally:
        rc.rcfar_destroy(h)
