"""The N>1 host logic of the benchmark on CPU: two gloo ranks, each an
independent replica with its own seeded events (no collective on the data
path), the slowest rank's time taken by a MAX all-reduce, and the whole-job
value summed over ranks.  The ranks' work is the CPU oracle on their shard,
so this runs without a GPU."""
import multiprocessing as mp
import os
import socket
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from oracle import oracle
    from paper_2004_04334_gb300 import synth

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seed = bench.rank_seed(rank, world)
        w = synth.workload("tiny", n_events=4, seed=seed)
        t0 = time.perf_counter()
        ref = oracle.reconstruct_workload(w)
        time.sleep(0.05 * (rank + 1))  # make the ranks' times differ
        t = time.perf_counter() - t0
        t_max = bench.max_over_ranks(t, world)
        q.put((rank, seed, w.words[:64].tobytes(), int(ref.n_clusters), t, t_max,
               bench.job_value(w.n_events, 1, t_max, world)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    (r0, s0, w0, c0, t0, m0, v0), (r1, s1, w1, c1, t1, m1, v1) = out
    assert (r0, r1) == (0, 1)
    assert s0 != s1 and w0 != w1  # each rank reconstructs its own events
    assert c0 > 0 and c1 > 0
    assert m0 == m1 == max(t0, t1)  # both ranks see the slowest rank's time
    assert v0 == v1 == 2 * 4 / max(t0, t1)


def test_single_rank_needs_no_collective():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.rank_seed(0, 1) is None
    assert bench.max_over_ranks(1.5, 1) == 1.5
    assert np.isclose(bench.job_value(256, 20, 2.0, 1), 2560.0)
