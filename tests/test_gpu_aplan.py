"""GPU parity of fixed-matrix plans (fcirc_aplan_*): the row vector's tree of
Algorithm 1 runs once, each product runs the other two trees.  Every product
through a plan must equal fcirc_matvec bit for bit, and the oracle."""
import numpy as np
import pytest

from paper_2103_02605_gb300 import inputs as I

pytestmark = pytest.mark.gpu

P1, P2 = I.P1, I.P2


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2103_02605_gb300 import build
    build.build()
    import paper_2103_02605_gb300 as F
    F.load()
    return F


def dev(v):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v, np.uint32).view(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


def f_with_root(p, n, seed):
    r = int(np.random.default_rng(seed).integers(2, p))
    return pow(r, max(n // 2, 1), p)


@pytest.mark.parametrize("m", [0, 1, 3, 10, 12, 13, 16, 20, 24])
def test_plan_equals_plain_product(F, orc, m):
    import torch
    p = P1 if m % 2 == 0 else P2
    n = 1 << m
    g = I.SplitMix64(7000 + m)
    a = g.uniform_mod(p, n)
    f = 1 if m in (12, 24) else f_with_root(p, n, m)
    with F.APlan(p, f, dev(a)) as plan:
        for k in range(2):
            x = g.uniform_mod(p, n)
            got = host(plan.matvec(dev(x)))
            want = host(F.fcirc_matvec(p, f, dev(a), dev(x)))
            torch.cuda.synchronize()
            assert np.array_equal(got, want), (m, k)
            if n <= 1 << 12:
                assert np.array_equal(got, orc.fcirc_matvec_mod(p, f, a, x))
            else:
                # the plan's tile variants against the oracle too, on rows
                # spread over every tile and both ends
                rows = np.unique(np.r_[0, 1, 4095, 4096, n // 2, n - 2, n - 1,
                                       np.random.default_rng(m + 10 * k).integers(0, n, 96)]).astype(np.uint64)
                assert np.array_equal(got[rows.astype(np.int64)], orc.fcirc_matvec_mod_rows(p, f, a, x, rows)), (m, k)


def test_plan_on_two_streams_and_host_buffers(F, orc):
    import torch
    n, p = 1 << 14, P1
    f = f_with_root(p, n, 5)
    g = I.SplitMix64(7100)
    a = g.uniform_mod(p, n)
    plan = F.APlan(p, f, torch.from_numpy(a.view(np.int32)))      # host row vector
    xs = [g.uniform_mod(p, n) for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    xd = [dev(x) for x in xs]
    torch.cuda.synchronize()   # the plan and the inputs are in place before the side streams read them
    outs = [plan.matvec(v, stream=st) for v, st in zip(xd, streams)]
    for st in streams:
        st.synchronize()
    for x, c in zip(xs, outs):
        assert np.array_equal(host(c), orc.fcirc_matvec_mod_rows(p, f, a, x, np.arange(n, dtype=np.uint64)))
    ch = plan.matvec(torch.from_numpy(xs[0].view(np.int32)))     # host vector and result
    assert np.array_equal(ch.numpy().view(np.uint32), host(outs[0]))
    plan.destroy()
    plan.destroy()   # a second destroy is a no-op


def test_plan_errors(F):
    import ctypes
    import torch
    L = F.load()
    z = torch.zeros(8, dtype=torch.int32, device="cuda")
    h = ctypes.c_void_p()
    assert L.fcirc_aplan_create(P1, 1, z.data_ptr(), 6, None, ctypes.byref(h)) == 1
    assert L.fcirc_aplan_create(P1, 1, None, 8, None, ctypes.byref(h)) == 1
    assert L.fcirc_aplan_create(P1, 0, z.data_ptr(), 8, None, ctypes.byref(h)) == 2
    assert L.fcirc_aplan_create(P1, 1, z.data_ptr(), 8, None, None) == 1
    assert L.fcirc_matvec_aplan(None, z.data_ptr(), z.data_ptr(), None) == 1
    assert L.fcirc_aplan_destroy(None) == 0
    with F.APlan(P1, 1, z) as plan:
        with pytest.raises(ValueError):
            plan.matvec(torch.zeros(16, dtype=torch.int32, device="cuda"))
