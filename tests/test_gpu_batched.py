"""GPU parity of the persistent batched product (uneven sizes, distinct f)
against the CPU oracle, instance by instance: bit-exact."""
import numpy as np
import pytest

from paper_2103_02605_gb300 import inputs as I

pytestmark = pytest.mark.gpu
P1 = I.P1


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2103_02605_gb300 import build
    build.build()
    import paper_2103_02605_gb300 as F
    F.load()
    return F


def dev(v, dt=np.int32):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v).view(dt)).cuda()


def run(F, f, offsets, a, x, p=P1):
    import torch
    c = F.fcirc_matvec_batched(p, dev(f), dev(offsets, np.int64), dev(a), dev(x))
    torch.cuda.synchronize()
    return c.cpu().numpy().view(np.uint32)


def check(orc, p, f, offsets, a, x, c, rows_per_big=24, seed=0):
    rng = np.random.default_rng(seed)
    for i in range(len(f)):
        s, e = int(offsets[i]), int(offsets[i + 1])
        n = e - s
        if n <= 4096:
            assert np.array_equal(c[s:e], orc.fcirc_matvec_mod(p, int(f[i]), a[s:e], x[s:e])), (i, n)
        else:
            rows = np.unique(np.concatenate([[0, 1, n - 1, n // 2, 4095, 4096],
                                             rng.integers(0, n, rows_per_big)])).astype(np.uint64)
            want = orc.fcirc_matvec_mod_rows(p, int(f[i]), a[s:e], x[s:e], rows)
            assert np.array_equal(c[s:e][rows.astype(np.int64)], want), (i, n)


def make_batch(sizes, p=P1, seed=1):
    rng = np.random.default_rng(seed)
    sizes = np.array(sizes, dtype=np.uint64)
    offsets = np.zeros(len(sizes) + 1, np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    g = I.SplitMix64(seed)
    a = g.uniform_mod(p, int(offsets[-1]))
    x = g.uniform_mod(p, int(offsets[-1]))
    f = np.array([pow(int(rng.integers(2, p)), max(int(n) // 2, 1), p) for n in sizes], np.uint32)
    return f, offsets, a, x


def test_every_size_once(F, orc):
    sizes = [1 << m for m in range(0, 17)]
    f, off, a, x = make_batch(sizes)
    check(orc, P1, f, off, a, x, run(F, f, off, a, x))


def test_mixed_sizes_and_primes(F, orc):
    rng = np.random.default_rng(3)
    for p in (P1, I.P2, 12289):
        v = ((p - 1) & -(p - 1)).bit_length() - 1
        sizes = [1 << int(m) for m in rng.integers(0, min(16, v + 1) + 1, 60)]
        f, off, a, x = make_batch(sizes, p=p, seed=int(p % 1000))
        check(orc, p, f, off, a, x, run(F, f, off, a, x, p=p), seed=p)


def test_invalid_instances_are_reported_and_skipped(F, orc):
    import torch
    f, off, a, x = make_batch([64, 128, 256])
    f[1] = 3                                       # 3 has no square root mod P1
    c = F.fcirc_matvec_batched(P1, dev(f), dev(off, np.int64), dev(a), dev(x))
    assert F.sync_status() == 2                    # FCIRC_ENOROOT
    c = c.cpu().numpy().view(np.uint32)
    for i in (0, 2):
        s, e = int(off[i]), int(off[i + 1])
        assert np.array_equal(c[s:e], orc.fcirc_matvec_mod(P1, int(f[i]), a[s:e], x[s:e]))
    off2 = np.array([0, 64, 64 + 48, 64 + 48 + 32], np.uint64)   # 48 is not a power of two
    f2 = np.array([1, 1, 1], np.uint32)
    g = I.SplitMix64(2)
    a2, x2 = g.uniform_mod(P1, 144), g.uniform_mod(P1, 144)
    c2 = F.fcirc_matvec_batched(P1, dev(f2), dev(off2, np.int64), dev(a2), dev(x2))
    assert F.sync_status() == 1                    # FCIRC_EINVAL
    c2 = c2.cpu().numpy().view(np.uint32)
    assert np.array_equal(c2[:64], orc.fcirc_matvec_mod(P1, 1, a2[:64], x2[:64]))
    assert np.array_equal(c2[112:], orc.fcirc_matvec_mod(P1, 1, a2[112:], x2[112:]))
    assert F.sync_status() == 0


def test_config3_workload_sampled(F, orc):
    """10,000 instances, n log-uniform in 2^6..2^16, f = w^((k n) mod 2^23)."""
    n, f, off, a, x = I.batched_mod()
    c = run(F, f, off, a, x)
    assert F.sync_status() == 0
    rng = np.random.default_rng(17)
    pick = np.unique(np.concatenate([[0, 1, len(n) - 1], rng.integers(0, len(n), 60)]))
    for i in pick:
        s, e = int(off[i]), int(off[i + 1])
        ni = e - s
        if ni <= 4096:
            assert np.array_equal(c[s:e], orc.fcirc_matvec_mod(P1, int(f[i]), a[s:e], x[s:e])), i
        else:
            rows = np.unique(np.concatenate([[0, ni - 1], rng.integers(0, ni, 16)])).astype(np.uint64)
            assert np.array_equal(c[s:e][rows.astype(np.int64)],
                                  orc.fcirc_matvec_mod_rows(P1, int(f[i]), a[s:e], x[s:e], rows)), i
    assert c.max() < P1


def test_graph_replay_follows_inputs(F, orc):
    import torch
    f, off, a, x = make_batch([256, 4096, 1 << 14, 32, 8192], seed=5)
    df, doff, da, dx = dev(f), dev(off, np.int64), dev(a), dev(x)
    out = torch.empty_like(da)
    g = F.BatchedGraph(P1, df, doff, da, dx, out, int(off[-1]))
    g.launch()
    torch.cuda.synchronize()
    check(orc, P1, f, off, a, x, out.cpu().numpy().view(np.uint32))
    # new inputs in the same buffers: the replay computes the new products
    f2, _, a2, x2 = make_batch([256, 4096, 1 << 14, 32, 8192], seed=6)
    df.copy_(dev(f2))
    da.copy_(dev(a2))
    dx.copy_(dev(x2))
    g.launch()
    torch.cuda.synchronize()
    check(orc, P1, f2, off, a2, x2, out.cpu().numpy().view(np.uint32))
    g.destroy()


def test_autotune_then_batched(F, orc):
    import torch
    rng = np.random.default_rng(11)
    sizes = [1 << int(m) for m in rng.integers(6, 17, 200)]
    f, off, a, x = make_batch(sizes, seed=11)
    df, doff, da, dx = dev(f), dev(off, np.int64), dev(a), dev(x)
    idx, cps, tl = F.batched_autotune(P1, df, doff, da, dx)
    assert 0 <= idx and cps >= 1 and tl in (11, 12)
    c = F.fcirc_matvec_batched(P1, df, doff, da, dx)
    torch.cuda.synchronize()
    check(orc, P1, f, off, a, x, c.cpu().numpy().view(np.uint32), rows_per_big=8)


def test_host_buffers(F, orc):
    import torch
    f, off, a, x = make_batch([16, 2048, 8192, 2], seed=8)
    c = F.fcirc_matvec_batched(P1, torch.from_numpy(f.view(np.int32)), torch.from_numpy(off.view(np.int64)),
                               torch.from_numpy(a.view(np.int32)), torch.from_numpy(x.view(np.int32)))
    check(orc, P1, f, off, a, x, c.numpy().view(np.uint32))


@pytest.mark.parametrize("ws", [2, 3])
def test_sharded_batch_equals_the_whole(F, orc, ws):
    """The batch split with fcirc_batched_partition, each shard packed and run
    on its own (the ranks of a multi-GPU job, here one after the other on
    one GPU): every instance's result equals the unsplit launch's, and the
    oracle's."""
    sizes = [1 << e for e in np.random.default_rng(ws).integers(0, 15, 150)]
    f, off, a, x = make_batch(sizes, seed=40 + ws)
    whole = run(F, f, off, a, x)
    check(orc, P1, f, off, a, x, whole, seed=ws)
    seen = np.zeros(len(sizes), bool)
    for r in range(ws):
        members, loads = F.batched_partition(off, ws, r)
        loc, fs, as_, xs = F.batched_shard(members, off, f, a, x)
        part = run(F, fs, loc, as_, xs)
        for j, i in enumerate(members):
            assert np.array_equal(part[int(loc[j]):int(loc[j + 1])], whole[int(off[i]):int(off[i + 1])]), (r, i)
        seen[members] = True
    assert seen.all()
