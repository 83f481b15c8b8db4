"""GPU parity of the products over Z/(2^K + 1) (fcirc_matvec_ssa): every
twiddle a shift, exact against the Python-integer oracle, including the edge
values 0, 1, 2^K - 1 and 2^K = -1."""
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


def dev(words):
    import torch
    return torch.from_numpy(np.ascontiguousarray(words, np.uint64).view(np.int64)).cuda()


@pytest.mark.parametrize("K,n", [(64, 8), (64, 16), (64, 64), (64, 256), (128, 8), (128, 32), (128, 256), (128, 512)])
def test_ssa_products_vs_oracle(F, orc, K, n):
    import torch
    batch = 2
    L = n.bit_length() - 2
    for f_exp in sorted({0, K if K % (1 << L) == 0 else 0, 3 * (1 << L) % (2 * K)}):
        a = [I.ssa_elements(n, K, seed=1500 + 7 * n + b) for b in range(batch)]
        x = [I.ssa_elements(n, K, seed=1600 + 7 * n + b)[::-1] for b in range(batch)]
        A = np.stack([I.ssa_to_words(v, K) for v in a])
        X = np.stack([I.ssa_to_words(v, K) for v in x])
        c = F.fcirc_matvec_ssa(dev(A), dev(X), K, f_exp)
        torch.cuda.synchronize()
        got = c.cpu().numpy().view(np.uint64)
        for b in range(batch):
            assert I.ssa_from_words(got[b]) == orc.fcirc_matvec_ssa(K, f_exp, a[b], x[b]), (K, n, f_exp, b)
        assert ((got[..., -1] == 0) | (got[..., -1] == 1)).all()


def test_ssa_errors(F):
    import torch
    L = F.load()
    z = torch.zeros(3 * 64, dtype=torch.int64, device="cuda")
    assert L.fcirc_matvec_ssa(z.data_ptr(), z.data_ptr(), z.data_ptr(), 96, 0, 8, 1, None) == 1
    assert L.fcirc_matvec_ssa(z.data_ptr(), z.data_ptr(), z.data_ptr(), 64, 0, 512, 1, None) == 1
    assert L.fcirc_matvec_ssa(z.data_ptr(), z.data_ptr(), z.data_ptr(), 64, 128, 8, 1, None) == 1
    assert L.fcirc_matvec_ssa(z.data_ptr(), z.data_ptr(), z.data_ptr(), 64, 1, 8, 1, None) == 2   # 4 does not divide 1
    zz = torch.zeros(3 * 512, dtype=torch.int64, device="cuda")
    # -1 = 2^128 has no 2^8-th root among the powers of 2 in Z/(2^128 + 1)
    assert L.fcirc_matvec_ssa(zz.data_ptr(), zz.data_ptr(), zz.data_ptr(), 128, 128, 512, 1, None) == 2
    assert L.fcirc_matvec_ssa(None, z.data_ptr(), z.data_ptr(), 64, 0, 8, 1, None) == 1
    assert L.fcirc_matvec_ssa(z.data_ptr(), z.data_ptr(), z.data_ptr(), 64, 0, 8, 0, None) == 0
