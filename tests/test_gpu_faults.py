"""Failure handling without a GPU fault: input checks that report through the
device status word, and host-side allocation failures injected at every
allocation site in turn (fcirc_set_checks, fcirc_debug_fail_alloc).  After
each failure the library must answer the next call correctly."""
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
    yield F
    F.set_checks(False)
    F.load().fcirc_debug_fail_alloc(-1)


def dev(v):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v, np.uint32).view(np.int32)).cuda()


def test_input_checks_report_through_the_status_word(F, orc):
    import torch
    n = 1 << 13
    a, x = I.single_mod(n, P1, seed=41)
    bad = a.copy()
    bad[123] = P1            # one residue out of range
    assert F.sync_status() == 0
    F.set_checks(True)
    try:
        F.fcirc_matvec(P1, 1, dev(a), dev(x))
        assert F.sync_status() == 0
        F.fcirc_matvec(P1, 1, dev(bad), dev(x))
        assert F.sync_status() == 1          # FCIRC_EINVAL, then cleared
        assert F.sync_status() == 0
        F.fcirc_toeplitz_matvec(P1, dev(np.concatenate([a, a[1:]])), dev(bad))
        assert F.sync_status() == 1
        g = np.zeros((2, 64, 2), np.uint32)
        g[1, 7, 1] = (1 << 31) - 1           # not canonical in GF(p^2)
        F.fcirc_matvec_gf(dev(g), dev(np.zeros_like(g)), (1, 0))
        assert F.sync_status() == 1
    finally:
        F.set_checks(False)
    # checks off: no report (the product's result for such input is unspecified)
    F.fcirc_matvec(P1, 1, dev(bad), dev(x))
    assert F.sync_status() == 0
    c = F.fcirc_matvec(P1, 1, dev(a), dev(x))
    torch.cuda.synchronize()
    rows = np.array([0, 5, n - 1], np.uint64)
    assert np.array_equal(c.cpu().numpy().view(np.uint32)[rows.astype(np.int64)],
                          orc.fcirc_matvec_mod_rows(P1, 1, a, x, rows))


def test_every_allocation_site_fails_cleanly(F, orc):
    """Release every cache, make the k-th allocation fail for k = 0, 1, ...
    until a call needs no more than k allocations; every failure is
    FCIRC_ENOMEM and the call right after it is exact."""
    import torch
    L = F.load()
    n = 1 << 16                                # plan tables, prime tables, scratch
    a, x = I.single_mod(n, P1, seed=43)
    f = pow(7, n // 2, P1)                     # has the 2^15-th root 7
    want = orc.fcirc_matvec_mod_rows(P1, f, a, x, np.arange(0, n, 997, dtype=np.uint64))
    da, dx = dev(a), dev(x)
    failures = 0
    for k in range(64):
        torch.cuda.synchronize()
        F.release()
        L.fcirc_debug_fail_alloc(k)
        try:
            F.fcirc_matvec(P1, f, da, dx)
            torch.cuda.synchronize()
            L.fcirc_debug_fail_alloc(-1)
            break                             # k was past the last allocation
        except F.FcircError as e:
            assert e.status == 3, e
            failures += 1
        L.fcirc_debug_fail_alloc(-1)
        c = F.fcirc_matvec(P1, f, da, dx)
        torch.cuda.synchronize()
        got = c.cpu().numpy().view(np.uint32)[0:n:997]
        assert np.array_equal(got, want), k
    assert failures >= 3                      # prime tables, plan tables, scratch at least


def test_fixed_matrix_plan_allocation_failure(F, orc):
    import torch
    L = F.load()
    n = 1 << 14
    a, x = I.single_mod(n, P1, seed=44)
    F.fcirc_matvec(P1, 1, dev(a), dev(x))     # plan and scratch in place
    torch.cuda.synchronize()
    L.fcirc_debug_fail_alloc(0)
    with pytest.raises(F.FcircError) as e:
        F.APlan(P1, 1, dev(a))                # the plan's own buffer
    assert e.value.status == 3
    L.fcirc_debug_fail_alloc(-1)
    with F.APlan(P1, 1, dev(a)) as plan:
        c = plan.matvec(dev(x))
        torch.cuda.synchronize()
        assert np.array_equal(c.cpu().numpy().view(np.uint32)[:64], orc.fcirc_matvec_mod_rows(
            P1, 1, a, x, np.arange(64, dtype=np.uint64)))
    assert F.sync_status() == 0


def test_status_word_allocation_failure():
    """The device status word is allocated through the same function as every
    other device buffer, so an injected failure reaches it too.  It is kept
    for the life of the process, hence a fresh process: its first use fails
    with FCIRC_ENOMEM, and the next succeeds."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import paper_2103_02605_gb300 as F\n"
        "L = F.load()\n"
        "L.fcirc_debug_fail_alloc(0)\n"
        "rc = L.fcirc_sync_status(None)\n"
        "L.fcirc_debug_fail_alloc(-1)\n"
        "print(rc, L.fcirc_sync_status(None))\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.split()[-2:] == ["3", "0"], r.stdout


@pytest.mark.parametrize("m", [20, 24])
def test_bounded_tma_wait_reports_a_timeout(F, orc, m):
    """The tile kernel's TMA loads complete on an mbarrier that thread 0
    probes a bounded number of times.  With the bound at zero probes every
    wait gives up at once: the call still completes (each CTA waits for its
    own copies, then leaves its tile), fcirc_sync_status returns
    FCIRC_ETIMEOUT once, and with the default bound the next call is exact."""
    import torch
    L = F.load()
    n = 1 << m
    a, x = I.single_mod(n, P1, seed=45)
    rows = np.array([0, 1, 4097, n // 2 + 3, n - 1], np.uint64)
    want = orc.fcirc_matvec_mod_rows(P1, 1, a, x, rows)
    da, dx = dev(a), dev(x)
    assert F.sync_status() == 0
    L.fcirc_debug_spin_limit(0)
    try:
        F.fcirc_matvec(P1, 1, da, dx)
        torch.cuda.synchronize()
        assert F.sync_status() == 5          # FCIRC_ETIMEOUT, then cleared
        assert F.sync_status() == 0
    finally:
        L.fcirc_debug_spin_limit(-1)
    c = F.fcirc_matvec(P1, 1, da, dx)
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy().view(np.uint32)[rows.astype(np.int64)], want)
    assert F.sync_status() == 0
