"""GPU parity of the large-integer product (Section 3.2) through the C ABI:
bit-exact against the CPU oracle and against Python's exact integers."""
import numpy as np
import pytest

from paper_2103_02605_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2103_02605_gb300 import build
    build.build()
    import paper_2103_02605_gb300 as F
    F.load()
    return F


def dev16(v):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v, np.uint16).view(np.int16)).cuda()


def gpu_mul(F, A, B):
    import torch
    out = F.bigint_mul(dev16(A), dev16(B))
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint16)


@pytest.mark.parametrize("na,nb", [(1, 1), (1, 7), (5, 1), (2, 2), (3, 5), (64, 64), (100, 2000),
                                   (2047, 2049), (4095, 1), (4096, 4096), (5000, 3001), (40000, 123)])
def test_bigint_small_vs_oracle_and_python(F, orc, na, nb):
    A, B = I.bigint_pair(16 * max(na, nb), seed=na * 31 + nb)
    A, B = A[:na], B[:nb]
    got = gpu_mul(F, A, B)
    assert got.size == na + nb
    if na * nb <= 1 << 24:
        assert np.array_equal(got, orc.bigint_mul(A, B))
    assert I.limbs_to_int(got) == I.limbs_to_int(A) * I.limbs_to_int(B)


@pytest.mark.parametrize("n", [1, 3, 16, 17, 4095, 4096, 4097, 1 << 16])
def test_bigint_all_ones_maximal_carries(F, n):
    A = np.full(n, 0xFFFF, np.uint16)
    v = (1 << (16 * n)) - 1
    got = gpu_mul(F, A, A)
    assert I.limbs_to_int(got) == v * v


def test_bigint_long_carry_chains(F):
    """Operands whose product has long runs of 0xFFFF limbs that a single
    carry must ripple through, across thread and chunk boundaries."""
    rng = np.random.default_rng(5)
    for n in (300, 5000, 70000):
        A = rng.integers(0, 1 << 16, n).astype(np.uint16)
        A[n // 4: 3 * n // 4] = 0xFFFF
        B = np.array([1, 1], np.uint16)            # A + A * 2^16
        got = gpu_mul(F, A, B)
        assert I.limbs_to_int(got) == I.limbs_to_int(A) * I.limbs_to_int(B)
        C = np.full(n, 0xFFFF, np.uint16)
        D = np.zeros(n, np.uint16)
        D[0] = 1
        D[-1] = 1
        assert I.limbs_to_int(gpu_mul(F, C, D)) == I.limbs_to_int(C) * I.limbs_to_int(D)


def test_bigint_2e18_limbs_exact(F):
    A, B = I.bigint_pair(16 << 18, seed=77)
    got = gpu_mul(F, A, B)
    assert I.limbs_to_int(got) == I.limbs_to_int(A) * I.limbs_to_int(B)


def test_bigint_config_full_size(F, orc):
    """Two 2^26-bit integers (2^22 limbs each, circulant size 2^23): the
    product modulo independent primes near 2^61, plus sampled column sums."""
    A, B = I.bigint_pair()
    got = gpu_mul(F, A, B)
    assert got.size == 2 * A.size
    for q in ((1 << 61) - 1, 2305843009213693921, (1 << 62) - 57):
        t = (1 << 16) % q
        assert orc.eval_u16_mod(got, t, q) == orc.eval_u16_mod(A, t, q) * orc.eval_u16_mod(B, t, q) % q


def test_bigint_host_buffers(F, orc):
    import torch
    A, B = I.bigint_pair(16 * 3000, seed=9)
    out = F.bigint_mul(torch.from_numpy(A.view(np.int16)), torch.from_numpy(B[:1777].view(np.int16)))
    assert np.array_equal(out.numpy().view(np.uint16), orc.bigint_mul(A, B[:1777]))


def test_bigint_errors(F):
    import torch
    L = F.load()
    z = torch.zeros(4, dtype=torch.int16, device="cuda")
    assert L.bigint_mul(z.data_ptr(), 0, z.data_ptr(), 4, z.data_ptr(), None) == 1
    assert L.bigint_mul(None, 4, z.data_ptr(), 4, z.data_ptr(), None) == 1
    assert L.bigint_mul(z.data_ptr(), 1 << 24, z.data_ptr(), 2, z.data_ptr(), None) == 1
