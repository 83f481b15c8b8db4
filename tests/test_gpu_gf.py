"""GPU parity of the products over the paper's own field GF(p^2) =
Z/pZ[sqrt 3], p = 2^31 - 1 (fcirc_matvec_gf): bit-exact against the oracle,
and the paper's use of it -- integer polynomial products modulo p through a
circulant (Section 3.1)."""
import numpy as np
import pytest

from paper_2103_02605_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GFP = (1 << 31) - 1


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


def pairs(g, shape):
    """Uniform elements of GF(p^2) from the seeded generator: (..., 2) uint32."""
    n = int(np.prod(shape))
    return g.uniform_mod(GFP, 2 * n).reshape(tuple(shape) + (2,))


def gf_pow(a, e):
    r = (1, 0)
    while e:
        if e & 1:
            r = ((r[0] * a[0] + 3 * r[1] * a[1]) % GFP, (r[0] * a[1] + r[1] * a[0]) % GFP)
        a = ((a[0] * a[0] + 3 * a[1] * a[1]) % GFP, (2 * a[0] * a[1]) % GFP)
        e >>= 1
    return r


@pytest.mark.parametrize("m", [3, 4, 7, 10, 12])
@pytest.mark.parametrize("batch", [1, 5])
def test_gf_products_vs_oracle(F, orc, m, batch):
    import torch
    n = 1 << m
    g = I.SplitMix64(1300 + 10 * m + batch)
    a, x = pairs(g, (batch, n)), pairs(g, (batch, n))
    r = tuple(int(v) for v in pairs(g, (1,))[0])
    for f in ((1, 0), (GFP - 1, 0), gf_pow(r, n // 2)):
        got = F.fcirc_matvec_gf(dev(a), dev(x), f)
        torch.cuda.synchronize()
        want = orc.fcirc_matvec_gf(f, a, x)
        assert np.array_equal(got.cpu().numpy().view(np.uint32), want), (m, batch, f)


def test_gf_polynomial_products_mod_p(F):
    """The paper's experiment in miniature: products of integer polynomials
    modulo 2^31 - 1 through circulants of size N = 2n (row vector P reversed
    and zero-padded, vector Q zero-padded, f = 1; coefficient k of the
    product is entry k + 1 of the circulant product).  Checked against
    numpy's exact integer convolution."""
    import torch
    n, batch = 1024, 64
    N = 2 * n
    g = I.SplitMix64(1400)
    P = g.uniform_mod(1 << 16, batch * n).reshape(batch, n).astype(np.int64)
    Q = g.uniform_mod(1 << 16, batch * n).reshape(batch, n).astype(np.int64)
    a = np.zeros((batch, N, 2), np.uint32)
    x = np.zeros((batch, N, 2), np.uint32)
    a[:, :, 0] = np.concatenate([np.zeros((batch, N - n), np.int64), P[:, ::-1]], axis=1)
    x[:, :n, 0] = Q
    c = F.fcirc_matvec_gf(dev(a), dev(x), (1, 0))
    torch.cuda.synchronize()
    c = c.cpu().numpy().view(np.uint32)
    assert not c[:, :, 1].any()
    for b in range(0, batch, 9):
        want = np.convolve(P[b], Q[b]) % GFP                 # exact: below 2^42 before the reduction
        got = np.roll(c[b, :, 0].astype(np.int64), -1)[: 2 * n - 1]
        assert np.array_equal(got, want)


def test_gf_errors(F):
    import torch
    L = F.load()
    z = torch.zeros(2 * 64, dtype=torch.int32, device="cuda")
    assert L.fcirc_matvec_gf(z.data_ptr(), z.data_ptr(), z.data_ptr(), 1, 0, 6, 1, None) == 1
    assert L.fcirc_matvec_gf(z.data_ptr(), z.data_ptr(), z.data_ptr(), 1, 0, 8192, 1, None) == 1
    assert L.fcirc_matvec_gf(z.data_ptr(), z.data_ptr(), z.data_ptr(), 0, 0, 64, 1, None) == 2
    assert L.fcirc_matvec_gf(z.data_ptr(), z.data_ptr(), z.data_ptr(), GFP, 0, 64, 1, None) == 1
    assert L.fcirc_matvec_gf(None, z.data_ptr(), z.data_ptr(), 1, 0, 64, 1, None) == 1
    assert L.fcirc_matvec_gf(z.data_ptr(), z.data_ptr(), z.data_ptr(), 1, 0, 64, 0, None) == 0
