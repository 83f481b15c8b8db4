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


def _shard_rank_main(rank, ws, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    try:
        import numpy as np
        import torch.distributed as dist

        import bench
        import paper_2103_02605_gb300 as F
        from paper_2103_02605_gb300 import inputs as I
        from oracle import oracle
        bench.dist_init(ws, backend="gloo")
        # a CPU-sized uneven batch of the benchmark's shape (sizes 2^2..2^8)
        nn, f, off, a, x = I.batched_mod(count=240, log_lo=2, log_hi=8)
        members, loads = F.batched_partition(off, ws, rank)
        loc, fs, as_, xs = F.batched_shard(members, off, f, a, x)
        # this rank's products, on its packed shard alone (the oracle stands
        # in for the GPU here: what is checked is the split and the packing)
        got = oracle.fcirc_matvec_mod_batched(I.P1, fs, loc, as_, xs)
        everything = oracle.fcirc_matvec_mod_batched(I.P1, f, off, a, x)
        want = np.concatenate([everything[int(off[i]):int(off[i + 1])] for i in members]) if len(members) else \
            np.zeros(0, np.uint32)
        all_members = [None] * ws
        all_loads = [None] * ws
        dist.all_gather_object(all_members, members.tolist())
        dist.all_gather_object(all_loads, loads.tolist())
        dist.destroy_process_group()
        q.put((rank, bool(np.array_equal(got, want)), all_members, all_loads,
               [float(v) for v in nn.astype(np.float64)]))
    except Exception as e:   # report to the parent instead of hanging it
        q.put((rank, "error", repr(e), None, None))


def test_batched_shard_over_two_gloo_ranks():
    """Each rank computes the same LPT partition on its own (no exchange),
    the two shards cover the batch once, their costs differ by at most one
    instance's, and each rank's packed shard gives its instances' products."""
    import multiprocessing as mp
    from paper_2103_02605_gb300 import build
    build.build()   # the children load the library for the partition
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    try:
        for _ in range(2):
            r = q.get(timeout=300)
            res[r[0]] = r
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    for r in (0, 1):
        assert res[r][1] != "error", res[r]
        assert res[r][1] is True, f"rank {r}: shard products differ from the oracle's"
    m0, m1 = res[0][2], res[1][2]
    assert res[0][2] == res[1][2] and res[0][3] == res[1][3]   # every rank computed the same split
    assert sorted(m0[0] + m0[1]) == list(range(240)) and not set(m0[0]) & set(m0[1])
    import math
    nn = res[0][4]
    cost = [n * max(math.ceil(math.log2(n)), 1) for n in nn]
    loads = res[0][3][0]
    assert loads[0] == sum(cost[i] for i in m0[0]) and loads[1] == sum(cost[i] for i in m0[1])
    assert abs(loads[0] - loads[1]) <= max(cost)


def test_partition_edge_cases():
    """Host-only checks of fcirc_batched_partition: one rank takes all, more
    ranks than instances leaves some empty, bad arguments are rejected."""
    import numpy as np
    from paper_2103_02605_gb300 import build
    build.build()
    import paper_2103_02605_gb300 as F
    off = np.array([0, 4, 8, 72, 73, 1097], dtype=np.uint64)
    m, loads = F.batched_partition(off, 1, 0)
    assert m.tolist() == [0, 1, 2, 3, 4] and loads.tolist() == [4 * 2 + 4 * 2 + 64 * 6 + 1 + 1024 * 10]
    parts = [F.batched_partition(off, 8, r)[0].tolist() for r in range(8)]
    assert sorted(sum(parts, [])) == [0, 1, 2, 3, 4]
    # largest first: the 1024 instance alone on rank 0, the 64 on rank 1, ...
    assert parts[0] == [4] and parts[1] == [2] and parts[5:] == [[], [], []]
    for bad in ((off, 0, 0), (off, 2, 2), (off[::-1].copy(), 2, 0)):
        with pytest.raises(F.FcircError):
            F.batched_partition(*bad)
    m, _ = F.batched_partition(np.zeros(1, np.uint64), 3, 1)   # an empty batch
    assert m.size == 0
