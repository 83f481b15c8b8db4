"""fcirc_matvec_noalloc, the entry point for callers that cannot let the
library allocate device memory (fixed memory pools reserved up front, or no
allocation-induced device synchronisation allowed while their streams run):
its results must equal those of fcirc_matvec, call after call, while the
library allocates nothing.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2103_02605_gb300 import inputs as I

pytestmark = pytest.mark.gpu

P1 = I.P1


def _dev(v):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v, np.uint32).view(np.int32)).cuda()


def _lib():
    import torch
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    from paper_2103_02605_gb300 import build
    build.build()
    import paper_2103_02605_gb300 as F
    return F.load()


def _case(lib, m, seed):
    import torch
    n = 1 << m
    a, x = I.single_mod(n, P1, seed=I.SEED_BASE + 500 + seed)
    # f with an n/2-th root, so that every n here has the roots Theorem 1 needs
    f = pow(int(np.random.default_rng(seed).integers(2, P1)), max(n // 2, 1), P1)
    da, dx = _dev(a), _dev(x)
    want = torch.empty_like(da)
    # the existing entry point, for reference (also loads every kernel once)
    assert lib.fcirc_matvec(P1, f, da.data_ptr(), dx.data_ptr(), want.data_ptr(), n, None) == 0
    return dict(n=n, f=f, a=a, x=x, da=da, dx=dx, want=want)


def test_noalloc_matches_fcirc_matvec_on_calls_in_a_row(orc):
    """Calls alternate between plans, so both the table upload (a new
    (p, f, n)) and the cached tables (the same (p, f, n) again) run: sizes
    2^20 and 2^16 take the column pass, 4096 and 2 only the tile kernel."""
    import torch
    lib = _lib()
    cases = [_case(lib, m, seed) for m, seed in ((20, 11), (16, 12), (12, 13), (1, 14))]
    torch.cuda.synchronize()
    # the reference itself against the oracle: in full for the tile-only
    # sizes, on sampled rows for the large ones
    for c in cases:
        want = c["want"].cpu().numpy().view(np.uint32)
        if c["n"] <= 4096:
            assert np.array_equal(want, orc.fcirc_matvec_mod(P1, c["f"], c["a"], c["x"]))
        else:
            rows = np.unique(np.r_[0, 1, c["n"] - 1, np.arange(0, c["n"], 4099)]).astype(np.uint64)
            assert np.array_equal(want[rows.astype(np.int64)],
                                  orc.fcirc_matvec_mod_rows(P1, c["f"], c["a"], c["x"], rows))

    order = [0, 1, 0, 0, 2, 3, 2, 1]        # new tables, cached tables, and back
    gots = [torch.empty_like(cases[i]["da"]) for i in order]
    torch.cuda.synchronize()
    outs = []
    free_after_first = None
    for k, i in enumerate(order):
        c = cases[i]
        got = gots[k]
        rc = lib.fcirc_matvec_noalloc(P1, c["f"], c["da"].data_ptr(), c["dx"].data_ptr(), got.data_ptr(),
                                      c["n"], None)
        assert rc == 0, lib.fcirc_last_error().decode()
        torch.cuda.synchronize()
        # integer results: the tolerance is exact equality
        assert torch.equal(got, c["want"]), f"call {k} (n = {c['n']}): noalloc differs from fcirc_matvec"
        outs.append((got, c["want"]))
        free_now = torch.cuda.mem_get_info()[0]
        if free_after_first is None:
            free_after_first = free_now
        else:
            # every later call allocated nothing on the device (the outputs of
            # this test are allocated before the first measurement)
            assert free_now >= free_after_first - (1 << 20), f"call {k}"
    # every output is still that of its own call
    for got, want in outs:
        assert torch.equal(got, want)


def test_noalloc_refuses_a_capturing_stream():
    """The tables the array holds are remembered on the host, so a call on a
    stream that is being captured returns FCIRC_EINVAL and enqueues nothing;
    the next eager call is exact."""
    import torch
    lib = _lib()
    c = _case(lib, 14, 21)
    got = torch.zeros_like(c["da"])
    assert lib.fcirc_matvec_noalloc(P1, c["f"], c["da"].data_ptr(), c["dx"].data_ptr(), got.data_ptr(),
                                    c["n"], None) == 0
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    other = torch.zeros(16, device="cuda")
    rc = None
    with torch.cuda.graph(g, stream=s):
        other.add_(1)                        # the graph is not empty
        rc = lib.fcirc_matvec_noalloc(P1, c["f"], c["da"].data_ptr(), c["dx"].data_ptr(), got.data_ptr(),
                                      c["n"], torch.cuda.current_stream().cuda_stream)
    assert rc == 1
    assert b"captured" in lib.fcirc_last_error()
    got.zero_()
    assert lib.fcirc_matvec_noalloc(P1, c["f"], c["da"].data_ptr(), c["dx"].data_ptr(), got.data_ptr(),
                                    c["n"], None) == 0
    torch.cuda.synchronize()
    assert torch.equal(got, c["want"])


def test_noalloc_rejects_what_it_cannot_hold():
    import torch
    lib = _lib()
    big = torch.zeros(1 << 21, dtype=torch.int32, device="cuda")
    assert lib.fcirc_matvec_noalloc(P1, 1, big.data_ptr(), big.data_ptr(), big.data_ptr(), 1 << 21, None) == 1
    assert b"2^20" in lib.fcirc_last_error()
    host = torch.zeros(1024, dtype=torch.int32)
    dev = torch.zeros(1024, dtype=torch.int32, device="cuda")
    assert lib.fcirc_matvec_noalloc(P1, 1, host.data_ptr(), dev.data_ptr(), dev.data_ptr(), 1024, None) == 1
    assert lib.fcirc_matvec_noalloc(P1, 1, dev.data_ptr(), dev.data_ptr(), dev.data_ptr(), 1000, None) == 1
