"""The multi-GPU path of the bench on CPU: two gloo ranks (no GPU).  Ranks take disjoint
pair ranges of the workload, solve them independently (here with the oracle, the same
d^2 a GPU rank computes) and meet only in the max-over-ranks of their times; the whole-job
rate counts every rank's pairs over the slowest rank's time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import synth
        from oracle import dense
        wl = synth.workload_ba_small()
        g = wl.graph
        first, count = bench.rank_pair_range(rank)
        X, Y = wl.pairs(first, count)
        d2 = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y)
        local_ms = 10.0 * (rank + 1)                    # rank 1 is the slower one
        total = bench.job_time(local_ms, dist, "cpu")
        rate = bench.job_rate(count, world, 3, total)
        gathered = [None] * world
        dist.all_gather_object(gathered, (first, count, d2.tolist(), total, rate))
        if rank == 0:
            np.save(os.path.join(out_dir, "result.npy"), np.array(gathered, dtype=object), allow_pickle=True)
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_pairs_and_take_the_max_time(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = np.load(tmp_path / "result.npy", allow_pickle=True)
    (f0, c0, d0, t0, r0), (f1, c1, d1, t1, r1) = res
    assert (f0, c0, f1, c1) == (0, 8, 8, 8)                       # disjoint, contiguous shares
    assert t0 == t1 == 20.0                                       # both ranks see the slowest time
    assert r0 == r1 == pytest.approx(2 * 8 * 3 / 0.020)
    # sharding changes nothing about the results: the same pairs solved in one process
    import synth
    from oracle import dense
    wl = synth.workload_ba_small()
    g = wl.graph
    X, Y = wl.pairs(0, 16)
    want = dense.ge_d2_eig(g.n, g.rowptr, g.colidx, g.w, X, Y)
    assert np.allclose(np.concatenate([d0, d1]), want, rtol=1e-13, atol=0)
