"""The multi-rank host logic of bench.py on CPU: two gloo ranks.

Each rank computes its own independent product (weak scaling, no collective
on the data path); the only collectives are the barrier around the timed
region and the max over ranks of the step time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    try:
        import numpy as np
        import torch.distributed as dist

        import bench
        from paper_2103_02605_gb300 import inputs as I
        got_ws, got_rank, _ = bench.dist_init(ws, backend="gloo")
        assert (got_ws, got_rank) == (ws, rank)
        bench.barrier(ws)
        # the slowest rank's time sets the job time
        t = bench.max_over_ranks(1.0 + rank, ws)
        # each rank's inputs are its own
        seed = bench.rank_seed(rank)
        P, Q = I.poly_pair(256, seed=seed)
        seeds = [None] * ws
        digests = [None] * ws
        dist.all_gather_object(seeds, seed)
        dist.all_gather_object(digests, (int(P.astype(np.uint64).sum()), int(Q[:7].astype(np.uint64).sum())))
        # the reference arm runs on rank 0 only; other ranks leave at once
        class A:
            gpus, steps, warmup = ws, 1, 3
        ref_rc = bench.run_reference(A, ws, rank) if rank != 0 else 0
        bench.barrier(ws)
        dist.destroy_process_group()
        q.put((rank, t, seeds, digests, ref_rc))
    except Exception as e:   # report to the parent instead of hanging it
        q.put((rank, "error", repr(e), None, None))


def test_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    try:
        for _ in range(2):
            r = q.get(timeout=180)
            res[r[0]] = r
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    for r in (0, 1):
        assert res[r][1] != "error", res[r]
        _, t, seeds, digests, ref_rc = res[r]
        assert t == 2.0
        assert len(set(seeds)) == 2 and len(set(digests)) == 2
        assert ref_rc == 0
    from paper_2103_02605_gb300 import inputs as I
    assert res[0][2][0] == I.SEED_BASE + 1   # rank 0 keeps the single-GPU workload


def test_job_value_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_value(4, 2.0) == pytest.approx(4 * bench.job_value(1, 2.0))
    assert bench.job_value(1, 1.0) == pytest.approx(bench.UNITS / 1e-3 / 1e9)
