"""GPU parity of the complex FP32 f-circulant layer (forward and hand-written
backward) against the FP64 oracle, through the C ABI and through autograd.
Tolerance: relative L2 error <= 1e-5 * log2(n)."""
import math

import numpy as np
import pytest

from paper_2103_02605_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FS = [1.0, -1.0, complex(math.cos(0.7), math.sin(0.7)), 2.0 - 0.5j, 0.5j]


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2103_02605_gb300 import build
    build.build()
    import paper_2103_02605_gb300 as F
    F.load()
    return F


def tol(n):
    return 1e-5 * math.log2(n)


def rel(got, want):
    got = np.asarray(got, np.complex128).reshape(want.shape)
    num = np.linalg.norm((got - want).reshape(want.shape[0], -1), axis=1)
    den = np.linalg.norm(want.reshape(want.shape[0], -1), axis=1)
    return float(np.max(num / den))


def dev(z):
    import torch
    return torch.from_numpy(np.ascontiguousarray(z, np.complex64)).cuda()


@pytest.mark.parametrize("m", list(range(3, 13)))
@pytest.mark.parametrize("batch", [1, 3])
def test_forward_and_backward_vs_oracle(F, orc, m, batch):
    import torch
    n = 1 << m
    a, x, g = I.complex_layer(batch, n, seed=1000 + m * 10 + batch)
    for f in FS:
        c = F.fcirc_matvec_c64(dev(a), dev(x), f)
        ga, gx = F.fcirc_matvec_backward(dev(a), dev(x), dev(g), f)
        torch.cuda.synchronize()
        assert rel(c.cpu().numpy(), orc.fcirc_matvec_c128(f, a, x)) <= tol(n), (m, f)
        wa, wx = orc.fcirc_grad_c128(f, a, x, g)
        assert rel(ga.cpu().numpy(), wa) <= tol(n), (m, f, "grad_a")
        assert rel(gx.cpu().numpy(), wx) <= tol(n), (m, f, "grad_x")


def test_many_instances_per_cta_ragged_batch(F, orc):
    import torch
    for n, batch in ((8, 129), (16, 37), (64, 5)):
        a, x, g = I.complex_layer(batch, n, seed=n + batch)
        c = F.fcirc_matvec_c64(dev(a), dev(x), 0.6 + 0.8j)
        ga, gx = F.fcirc_matvec_backward(dev(a), dev(x), dev(g), 0.6 + 0.8j)
        torch.cuda.synchronize()
        assert rel(c.cpu().numpy(), orc.fcirc_matvec_c128(0.6 + 0.8j, a, x)) <= tol(n)
        wa, wx = orc.fcirc_grad_c128(0.6 + 0.8j, a, x, g)
        assert rel(ga.cpu().numpy(), wa) <= tol(n) and rel(gx.cpu().numpy(), wx) <= tol(n)


def test_config2_full_batch(F, orc):
    """batch 4096 of f = 1 circulants with n = 1024: every instance against
    numpy's FFT in float64 (the f = 1 circulant is a cyclic correlation), and
    sampled instances of the forward and both gradients against the oracle."""
    import torch
    batch, n = 4096, 1024
    a, x, g = I.complex_layer(batch, n)
    c = F.fcirc_matvec_c64(dev(a), dev(x), 1.0)
    ga, gx = F.fcirc_matvec_backward(dev(a), dev(x), dev(g), 1.0)
    torch.cuda.synchronize()
    a64, x64 = a.astype(np.complex128), x.astype(np.complex128)
    want = np.fft.ifft(n * np.fft.ifft(a64, axis=1) * np.fft.fft(x64, axis=1), axis=1)
    assert rel(c.cpu().numpy(), want) <= tol(n)
    idx = np.array([0, 1, 777, 2048, 4095] + list(range(100, 4096, 157)))
    assert rel(c.cpu().numpy()[idx], orc.fcirc_matvec_c128(1.0, a[idx], x[idx])) <= tol(n)
    wa, wx = orc.fcirc_grad_c128(1.0, a[idx], x[idx], g[idx])
    assert rel(ga.cpu().numpy()[idx], wa) <= tol(n)
    assert rel(gx.cpu().numpy()[idx], wx) <= tol(n)


def test_autograd_layer(F, orc):
    import torch
    batch, n, f = 6, 256, 0.8 - 0.6j
    a, x, g = I.complex_layer(batch, n, seed=4242)
    ta = dev(a).requires_grad_(True)
    tx = dev(x).requires_grad_(True)
    c = F.fcirc_layer(ta, tx, f)
    tg = dev(g)
    loss = torch.real(torch.sum(torch.conj(tg) * c))
    loss.backward()
    wa, wx = orc.fcirc_grad_c128(f, a, x, g)
    assert rel(ta.grad.cpu().numpy(), wa) <= tol(n)
    assert rel(tx.grad.cpu().numpy(), wx) <= tol(n)
    # the same gradients from PyTorch's own autograd through a dense complex128
    # product built from the oracle's columns (a library routine, not ours)
    a0, x0 = a[0].astype(np.complex128), x[0].astype(np.complex128)
    A = np.stack([orc.fcirc_matvec_c128(f, a0, np.eye(n)[j]) for j in range(n)], axis=1)
    tA = torch.tensor(A)
    tx0 = torch.tensor(x0, requires_grad=True)
    l0 = torch.real(torch.sum(torch.conj(torch.tensor(g[0].astype(np.complex128))) * (tA @ tx0)))
    l0.backward()
    assert rel(tx.grad[0:1].cpu().numpy(), tx0.grad.numpy()[None]) <= tol(n)


def test_host_buffers(F, orc):
    import torch
    a, x, g = I.complex_layer(5, 512, seed=31)
    c = F.fcirc_matvec_c64(torch.from_numpy(a), torch.from_numpy(x), -1.0)
    assert rel(c.numpy(), orc.fcirc_matvec_c128(-1.0, a, x)) <= tol(512)
    ga, gx = F.fcirc_matvec_backward(torch.from_numpy(a), torch.from_numpy(x), torch.from_numpy(g), -1.0)
    wa, wx = orc.fcirc_grad_c128(-1.0, a, x, g)
    assert rel(ga.numpy(), wa) <= tol(512) and rel(gx.numpy(), wx) <= tol(512)


def test_errors(F):
    import torch
    L = F.load()
    z = torch.zeros(8192, dtype=torch.complex64, device="cuda")
    for n in (4, 6, 8192):
        assert L.fcirc_matvec_c64(z.data_ptr(), z.data_ptr(), z.data_ptr(), 1.0, 0.0, n, 1, None) == 1
    assert L.fcirc_matvec_c64(z.data_ptr(), z.data_ptr(), z.data_ptr(), 0.0, 0.0, 64, 1, None) == 2
    assert L.fcirc_matvec_backward(z.data_ptr(), z.data_ptr(), z.data_ptr(), 0.0, 0.0, z.data_ptr(),
                                   z.data_ptr(), 64, 1, None) == 2
    assert L.fcirc_matvec_c64(z.data_ptr(), z.data_ptr(), z.data_ptr(), 1.0, 0.0, 64, 0, None) == 0
