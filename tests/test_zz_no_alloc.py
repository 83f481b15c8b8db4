"""fcirc_matvec_noalloc, the entry point for callers that cannot let the
library allocate device memory (fixed memory pools reserved up front, or no
allocation-induced device synchronisation allowed while their streams run):
its results must equal those of fcirc_matvec, call after call, while the
library allocates nothing.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2103_02605_gb300 import inputs as I

pytestmark = pytest.mark.gpu

P1 = I.P1


def _dev(v):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v, np.uint32).view(np.int32)).cuda()


def test_noalloc_matches_fcirc_matvec_on_two_calls_in_a_row():
    import torch
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    from paper_2103_02605_gb300 import build
    build.build()
    import paper_2103_02605_gb300 as F
    lib = F.load()

    cases = []
    for m, seed in ((20, 11), (16, 12)):
        n = 1 << m
        a, x = I.single_mod(n, P1, seed=I.SEED_BASE + 500 + seed)
        f = pow(int(np.random.default_rng(seed).integers(2, P1)), n // 2, P1)
        da, dx = _dev(a), _dev(x)
        want = torch.empty_like(da)
        got = torch.empty_like(da)
        # the existing entry point, for reference (also loads every kernel once)
        assert lib.fcirc_matvec(P1, f, da.data_ptr(), dx.data_ptr(), want.data_ptr(), n, None) == 0
        cases.append((n, f, da, dx, want, got))
    torch.cuda.synchronize()

    free_after_first = None
    for k, (n, f, da, dx, want, got) in enumerate(cases):
        rc = lib.fcirc_matvec_noalloc(P1, f, da.data_ptr(), dx.data_ptr(), got.data_ptr(), n, None)
        assert rc == 0, lib.fcirc_last_error().decode()
        torch.cuda.synchronize()
        # integer results: the tolerance is exact equality
        assert torch.equal(got, want), f"call {k}: noalloc result differs from fcirc_matvec"
        free_now = torch.cuda.mem_get_info()[0]
        if free_after_first is None:
            free_after_first = free_now
        else:
            # the second call (new size, new tables) allocated nothing
            assert free_now >= free_after_first - (1 << 20)
    # both outputs are still those of their own call
    assert torch.equal(cases[0][5], cases[0][4]) and torch.equal(cases[1][5], cases[1][4])


def test_noalloc_rejects_what_it_cannot_hold():
    import torch
    import paper_2103_02605_gb300 as F
    lib = F.load()
    big = torch.zeros(1 << 21, dtype=torch.int32, device="cuda")
    assert lib.fcirc_matvec_noalloc(P1, 1, big.data_ptr(), big.data_ptr(), big.data_ptr(), 1 << 21, None) == 1
    assert b"2^20" in lib.fcirc_last_error()
    host = torch.zeros(1024, dtype=torch.int32)
    dev = torch.zeros(1024, dtype=torch.int32, device="cuda")
    assert lib.fcirc_matvec_noalloc(P1, 1, host.data_ptr(), dev.data_ptr(), dev.data_ptr(), 1024, None) == 1
    assert lib.fcirc_matvec_noalloc(P1, 1, dev.data_ptr(), dev.data_ptr(), dev.data_ptr(), 1000, None) == 1
