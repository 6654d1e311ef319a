"""Replicas across GPUs (weak scaling), host side on two CPU ranks (gloo):
every rank's orbit seeds are its own (rank 0 keeps the single-GPU workload's),
and the timing reduction gives every rank the slowest rank's time and the sum
of the ranks' counts, as bench.py reports them for N GPUs."""
import multiprocessing as mp
import socket

from paper_1403_0555_b300.replicas import rank_seed, reduce_timing

import replica_worker


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_single_rank_is_the_identity():
    assert reduce_timing(None, 12.5, 7) == (12.5, 7.0)
    assert [rank_seed(0, j) for j in range(8)] == list(range(1, 9))


def test_two_gloo_ranks_reduce_and_own_seeds():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=replica_worker.run, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        results = [q.get(timeout=120) for _ in range(world)]
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()
    assert all(p.exitcode == 0 for p in procs)
    assert sorted(r[0] for r in results) == [0, 1]
    for rank, ms, count, gathered in results:
        assert ms == 11.0                 # the slower rank's time
        assert count == 300.0             # 100 + 200
        assert gathered[0] == list(range(1, 9))
        flat = [s for seeds in gathered for s in seeds]
        assert len(set(flat)) == len(flat) == 16
