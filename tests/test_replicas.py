"""Replicas across ranks (host logic), world size 2 on CPU with gloo.

Frames are independent, so N GPUs run N independent copies of the chain.
This checks the host side on CPU processes: the frame partition covers every
frame exactly once, per-rank results gathered from two ranks equal the
single-process results (here from the FP64 oracle on small frames; no GPU),
and the job time is the maximum over ranks.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2012_11077_gb300 import replicas  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _frame_result(i: int):
    """Oracle decisions of frame i (a small seeded frame)."""
    import oracle
    import synth
    spec = synth.FrameSpec(M=48, N=256, n_targets=2, seed=100 + i)
    w = synth.Window(4, 4, 1, 1, 1e-3)
    P, band = oracle.preprocess_frame(synth.radar_frame(spec), synth.FS_HZ, 5, halo=w.train_c + w.guard_c)
    res = oracle.cfar_chain(P, band, w.train_r, w.train_c, w.guard_r, w.guard_c, w.pfa)
    return i, res.det.astype(np.uint8).tobytes(), float(res.thr.sum())


def _rank_main(rank, world, port, n_frames, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w, _, d = replicas.setup(backend="gloo")
    assert (r, w) == (rank, world) and d is not None
    mine = [_frame_result(i) for i in replicas.shard(n_frames, r, w)]
    gathered = [None] * w
    d.all_gather_object(gathered, mine)
    t_max = replicas.max_over_ranks(1.5 * (r + 1), d)
    t_sum = replicas.sum_over_ranks(float(len(mine)), d)
    replicas.barrier(d)
    if r == 0:
        out_q.put((gathered, t_max, t_sum))
    d.destroy_process_group()


def test_shard_partition():
    for n in (0, 1, 7, 64, 65):
        for world in (1, 2, 3, 8):
            parts = [list(replicas.shard(n, r, world)) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def test_single_process_is_identity():
    os.environ.pop("WORLD_SIZE", None)
    assert replicas.setup()[3] is None
    assert replicas.max_over_ranks(2.5, None) == 2.5


def test_two_ranks_gloo():
    n_frames, world = 5, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n_frames, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, t_max, t_sum = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t_max == 3.0 and t_sum == n_frames
    by_rank = [sorted(i for i, _, _ in g) for g in gathered]
    assert by_rank == [list(replicas.shard(n_frames, r, world)) for r in range(world)]
    merged = {i: (det, s) for g in gathered for i, det, s in g}
    for i in range(n_frames):
        j, det, s = _frame_result(i)
        assert merged[i] == (det, s)
