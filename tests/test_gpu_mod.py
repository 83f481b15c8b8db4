"""GPU parity of the modular f-circulant product and the polynomial product
against the CPU oracle: bit-exact, element by element, through the C ABI."""
import numpy as np
import pytest

from paper_2103_02605_gb300 import inputs as I

pytestmark = pytest.mark.gpu

P1, P2, P3 = I.P1, I.P2, I.P3


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2103_02605_gb300 import build
    build.build()
    import paper_2103_02605_gb300 as F
    F.load()
    return F


def dev_u32(v):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v, np.uint32).view(np.int32)).cuda()


def dev_u16(v):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v, np.uint16).view(np.int16)).cuda()


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


def f_with_root(p, n, seed):
    """An f that has the (n/2)-th root the plan needs (Theorem 1)."""
    r = int(np.random.default_rng(seed).integers(2, p))
    return pow(r, max(n // 2, 1), p)


def matvec(F, p, f, a, x):
    import torch
    c = F.fcirc_matvec(p, f, dev_u32(a), dev_u32(x))
    torch.cuda.synchronize()
    return host_u32(c)


@pytest.mark.parametrize("p", [P1, P2, P3, 12289, 7681, 17])
def test_matvec_every_small_power_of_two(F, orc, p):
    v = ((p - 1) & -(p - 1)).bit_length() - 1
    g = I.SplitMix64(p)
    for m in range(0, min(12, v + 1) + 1):
        n = 1 << m
        a, x = g.uniform_mod(p, n), g.uniform_mod(p, n)
        for f in (1, p - 1, f_with_root(p, n, m)):
            if n > 2 and f == p - 1 and pow(p - 1, (p - 1) // int(np.gcd(n // 2, p - 1)), p) != 1:
                continue
            got = matvec(F, p, f, a, x)
            assert np.array_equal(got, orc.fcirc_matvec_mod(p, f, a, x)), (p, m, f)


@pytest.mark.parametrize("m", [13, 14, 15])
def test_matvec_multi_tile_full(F, orc, m):
    n = 1 << m
    a, x = I.single_mod(n, P1, seed=I.SEED_BASE + 100 + m)
    for f in (1, f_with_root(P1, n, m)):
        assert np.array_equal(matvec(F, P1, f, a, x), orc.fcirc_matvec_mod(P1, f, a, x)), (m, f)


def sample_rows(n, T=4096, k=48, seed=0):
    rng = np.random.default_rng(seed)
    rows = set([0, 1, n - 1, n - 2, n // 2, n // 2 - 1])
    for t in range(0, n, max(T, n // 8)):
        rows.update([t, t + T - 1 if t + T - 1 < n else n - 1])
    rows.update(int(r) for r in rng.integers(0, n, k))
    return np.array(sorted(rows), dtype=np.uint64)


@pytest.mark.parametrize("m,p", [(17, P1), (20, P2), (24, P1), (25, P2), (26, P3)])
def test_matvec_large_sampled(F, orc, m, p):
    """Large n (several strided passes for 2^25+), checked on sampled rows."""
    n = 1 << m
    a, x = I.single_mod(n, p, seed=I.SEED_BASE + 200 + m)
    f = f_with_root(p, n, 7 * m)
    got = matvec(F, p, f, a, x)
    rows = sample_rows(n, seed=m)
    assert np.array_equal(got[rows.astype(np.int64)], orc.fcirc_matvec_mod_rows(p, f, a, x, rows))
    assert got.max() < p


@pytest.mark.parametrize("m", [21, 22, 23])
def test_matvec_column_pass_shapes(F, orc, m):
    """n = 2^21 .. 2^23: column passes of 9, 10 and 11 levels (clusters of
    two over 2^(12-LF) column quads per CTA), checked on sampled rows."""
    n = 1 << m
    a, x = I.single_mod(n, P1, seed=I.SEED_BASE + 300 + m)
    f = f_with_root(P1, n, 11 * m)
    got = matvec(F, P1, f, a, x)
    rows = sample_rows(n, seed=m + 1)
    assert np.array_equal(got[rows.astype(np.int64)], orc.fcirc_matvec_mod_rows(P1, f, a, x, rows))


@pytest.mark.parametrize("m", [20, 24])
def test_matvec_unaligned_views_take_the_one_column_kernels(F, orc, m):
    """Sources and destination offset by one word (not 16-byte aligned): the
    four-column kernels decline and the one-column kernels run instead."""
    import torch
    n = 1 << m
    a, x = I.single_mod(n, P2, seed=I.SEED_BASE + 400 + m)
    f = f_with_root(P2, n, m)
    buf_a = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    buf_x = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    buf_c = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    buf_a[1:] = dev_u32(a)
    buf_x[1:] = dev_u32(x)
    F.fcirc_matvec(P2, f, buf_a[1:], buf_x[1:], out=buf_c[1:])
    torch.cuda.synchronize()
    got = host_u32(buf_c[1:])
    assert np.array_equal(got, matvec(F, P2, f, a, x))
    rows = sample_rows(n, seed=m + 2)
    assert np.array_equal(got[rows.astype(np.int64)], orc.fcirc_matvec_mod_rows(P2, f, a, x, rows))


@pytest.mark.parametrize("m", [0, 1, 2, 5, 12, 13])
def test_matvec_transposed_vs_oracle(F, orc, m):
    """fcirc_matvec_t (column convention, A^T x) against the oracle's
    a(z) x(z) mod (z^n - f)."""
    import torch
    n = 1 << m
    for p in (P1, P3):
        g = I.SplitMix64(900 + m + p % 97)
        a, x = g.uniform_mod(p, n), g.uniform_mod(p, n)
        for f in (1, p - 1, f_with_root(p, n, 3 * m + 1)):
            if n > 2 and f == p - 1 and pow(p - 1, (p - 1) // int(np.gcd(n // 2, p - 1)), p) != 1:
                continue
            c = F.fcirc_matvec_t(p, f, dev_u32(a), dev_u32(x))
            torch.cuda.synchronize()
            assert np.array_equal(host_u32(c), orc.fcirc_matvec_t_mod(p, f, a, x)), (p, m, f)


def _powers_mod(t, n, p):
    """t^k mod p for k < n (n a power of two), in blocks of 4096."""
    lo = np.empty(min(n, 4096), np.uint64)
    acc = 1
    for k in range(lo.size):
        lo[k] = acc
        acc = acc * t % p
    if n <= 4096:
        return lo
    step = pow(t, 4096, p)
    hi = np.empty(n // 4096, np.uint64)
    acc = 1
    for k in range(hi.size):
        hi[k] = acc
        acc = acc * step % p
    return ((hi[:, None] * lo[None, :]) % p).reshape(-1)


def _eval_mod(coef, pw, p):
    # each product is below 2^60 and reduced before the sum (below 2^54)
    return int(((coef.astype(np.uint64) * pw) % p).sum(dtype=np.uint64) % p)


@pytest.mark.parametrize("m", [20, 24])
def test_matvec_transposed_large_by_evaluation(F, m):
    """A^T x = a(z) x(z) mod (z^n - f): at any root t of z^n - f the values
    satisfy c(t) = a(t) x(t) mod p.  Two roots t = r w^k with f = r^n."""
    import torch
    n, p = 1 << m, P1
    g = I.SplitMix64(950 + m)
    a, x = g.uniform_mod(p, n), g.uniform_mod(p, n)
    r = 123457
    f = pow(r, n, p)
    c = host_u32(F.fcirc_matvec_t(p, f, dev_u32(a), dev_u32(x)))
    torch.cuda.synchronize()
    w = I.primitive_2k_root(p, min(m, 23))   # w^n = 1
    for k in (1, 12345):
        t = r * pow(w, k, p) % p
        assert pow(t, n, p) == f
        pw = _powers_mod(t, n, p)
        ca = _eval_mod(a, pw, p)
        cx = _eval_mod(x, pw, p)
        assert _eval_mod(c, pw, p) == ca * cx % p


@pytest.mark.parametrize("n", [3, 5, 6, 7, 100, 1000, 4095, 5000, 70001, (1 << 20) + 3])
def test_matvec_any_n_corollary1(F, orc, n):
    """n not a power of two: Corollary 1's embedding into a power-of-two
    circulant, any f (no roots of f needed), against the oracle."""
    import torch
    p = P1 if n % 2 else P3
    g = I.SplitMix64(1100 + n)
    a, x = g.uniform_mod(p, n), g.uniform_mod(p, n)
    for f in (0, 1, p - 1, 12345):
        c = F.fcirc_matvec(p, f, dev_u32(a), dev_u32(x))
        torch.cuda.synchronize()
        got = host_u32(c)
        if n <= 5000:
            assert np.array_equal(got, orc.fcirc_matvec_mod(p, f, a, x)), (n, f)
        else:
            rows = sample_rows(n, seed=n % 1000)
            assert np.array_equal(got[rows.astype(np.int64)], orc.fcirc_matvec_mod_rows(p, f, a, x, rows)), (n, f)


@pytest.mark.parametrize("n", [1, 2, 3, 64, 1000, 4097])
def test_toeplitz_vs_oracle(F, orc, n):
    import torch
    g = I.SplitMix64(1200 + n)
    t, x = g.uniform_mod(P2, 2 * n - 1), g.uniform_mod(P2, n)
    c = F.fcirc_toeplitz_matvec(P2, dev_u32(t), dev_u32(x))
    torch.cuda.synchronize()
    assert np.array_equal(host_u32(c), orc.toeplitz_matvec_mod(P2, t, x))
    # host buffers
    ch = F.fcirc_toeplitz_matvec(P2, torch.from_numpy(t.view(np.int32)), torch.from_numpy(x.view(np.int32)))
    assert np.array_equal(ch.numpy().view(np.uint32), host_u32(c))


def test_matvec_config0_full(F, orc):
    """n = 2^12, f = 1, p = 998244353: the single-instance workload, full vector."""
    a, x = I.single_mod(1 << 12)
    assert np.array_equal(matvec(F, P1, 1, a, x), orc.fcirc_matvec_mod(P1, 1, a, x))


def test_matvec_extreme_values(F, orc):
    """Every entry p - 1, for the three primes: each has its own schedule of
    reductions in the tile kernel (room 4, 9 and 25 times p below 2^32)."""
    rng = np.random.default_rng(17)
    for p in (P1, P2, P3):
        for m in (1, 5, 12, 14, 16, 20):
            n = 1 << m
            a = np.full(n, p - 1, np.uint32)
            x = np.full(n, p - 1, np.uint32)
            for f in (1, p - 1):
                got = matvec(F, p, f, a, x)
                if m <= 14:
                    assert np.array_equal(got, orc.fcirc_matvec_mod(p, f, a, x)), (p, m, f)
                else:
                    rows = np.unique(np.concatenate([np.arange(8), n - 1 - np.arange(8),
                                                     rng.integers(0, n, 48)])).astype(np.uint64)
                    assert np.array_equal(got[rows.astype(np.int64)], orc.fcirc_matvec_mod_rows(p, f, a, x, rows)), \
                        (p, m, f)
            if p == P1:
                z = np.zeros(n, np.uint32)
                assert not matvec(F, P1, 3 ** 2 if m == 1 else 1, z, x).any()


def test_matvec_host_buffers_match_device(F, orc):
    import torch
    for m in (3, 12, 16):
        n = 1 << m
        a, x = I.single_mod(n, P2, seed=m)
        f = f_with_root(P2, n, m)
        ah = torch.from_numpy(a.view(np.int32))
        xh = torch.from_numpy(x.view(np.int32))
        ch = F.fcirc_matvec(P2, f, ah, xh)      # host tensors: staged by the library
        assert np.array_equal(ch.numpy().view(np.uint32), matvec(F, P2, f, a, x))
        if m <= 12:
            assert np.array_equal(ch.numpy().view(np.uint32), orc.fcirc_matvec_mod(P2, f, a, x))


def test_matvec_errors(F):
    import torch
    a = dev_u32(np.zeros(8, np.uint32))
    for bad_p in (4, 15, 2, 2147483647):
        with pytest.raises(F.FcircError) as e:
            F.fcirc_matvec(bad_p, 1, a, a)
        assert e.value.status == 1
    with pytest.raises(F.FcircError) as e:
        F.fcirc_matvec(P1, 0, a, a)
    assert e.value.status == 2
    with pytest.raises(F.FcircError) as e:
        F.fcirc_matvec(P1, 3, a, a)          # 3 is a non-residue mod P1
    assert e.value.status == 2
    big = torch.zeros(1 << 25, dtype=torch.int32, device="cuda")
    with pytest.raises(F.FcircError) as e:
        F.fcirc_matvec(P1, 1, big, big)      # needs a 2^24-th root of unity
    assert e.value.status == 2
    # n = 6 is no error (Corollary 1), n = 0 is
    z0 = torch.zeros(0, dtype=torch.int32, device="cuda")
    with pytest.raises(F.FcircError) as e:
        F.fcirc_matvec(P1, 1, z0, z0)
    assert e.value.status == 1
    L = F.load()
    assert L.fcirc_matvec(P1, 1, None, None, None, 8, None) == 1
    assert L.fcirc_matvec(P1, 1, a.data_ptr(), a.data_ptr(), a.data_ptr(), 0, None) == 1
    assert F.sync_status() == 0


# -- polynomial product (Section 3.1) ---------------------------------------------

def poly(F, Pc, Qc):
    import torch
    out = F.poly_mul_int(dev_u16(Pc), dev_u16(Qc))
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("np_,nq", [(1, 1), (1, 2), (2, 1), (3, 5), (64, 64), (2048, 2049),
                                    (4096, 1), (3000, 1097), (4097, 4096), (10000, 333),
                                    (1 << 14, 1 << 14), (70001, 5)])
def test_poly_full(F, orc, np_, nq):
    Pc, Qc = I.poly_pair(np_, seed=np_ * 7 + nq, nq=nq)
    assert np.array_equal(poly(F, Pc, Qc), orc.poly_mul(Pc, Qc))


@pytest.mark.parametrize("lg", [20, 21, 22])
def test_poly_column_pass_shapes(F, orc, lg):
    """Circulant sizes 2^21 .. 2^23 (column passes of 9 .. 11 levels with the
    three-CTA inverse): sampled coefficients exactly, plus evaluation mod a
    61-bit prime."""
    n = 1 << lg
    Pc, Qc = I.poly_pair(n, seed=I.SEED_BASE + 500 + lg, nq=n - 3)
    C = poly(F, Pc, Qc)
    rng = np.random.default_rng(lg)
    idx = np.unique(np.concatenate([[0, 1, n - 1, n, C.size - 1],
                                    rng.integers(0, C.size, 60)])).astype(np.uint64)
    assert np.array_equal(C[idx.astype(np.int64)], orc.poly_mul_coeffs(Pc, Qc, idx))
    q = (1 << 61) - 1
    t = int(rng.integers(2, q))
    assert orc.eval_i64_mod(C, t, q) == orc.eval_u16_mod(Pc, t, q) * orc.eval_u16_mod(Qc, t, q) % q


def test_poly_unaligned_inputs(F, orc):
    """uint16 inputs at odd element offsets: the forward pass falls back to
    the one-column kernel; the result is unchanged."""
    import torch
    n = 1 << 22
    Pc, Qc = I.poly_pair(n, seed=77)
    bp = torch.zeros(n + 1, dtype=torch.int16, device="cuda")
    bq = torch.zeros(n + 3, dtype=torch.int16, device="cuda")
    bp[1:] = dev_u16(Pc)
    bq[3:] = dev_u16(Qc)
    C = F.poly_mul_int(bp[1:], bq[3:])
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), poly(F, Pc, Qc))


def test_poly_output_alignments(F, orc):
    """The output at offsets of 0 .. 3 int64 from a 32-byte boundary: the CRT
    writes whole 32-byte quads only where they are aligned and otherwise
    falls back to 8-byte stores; every placement gives the same product."""
    import torch
    n = 1 << 21
    Pc, Qc = I.poly_pair(n, seed=I.SEED_BASE + 610, nq=n - 1)
    dP, dQ = dev_u16(Pc), dev_u16(Qc)
    buf = torch.full((2 * n + 8,), -1, dtype=torch.int64, device="cuda")
    assert buf.data_ptr() % 32 == 0
    ref = None
    for off in (0, 1, 2, 3):
        buf.fill_(-1)
        out = buf[off:off + 2 * n - 2]
        F.poly_mul_int(dP, dQ, out=out)
        torch.cuda.synchronize()
        B = buf.cpu().numpy()
        assert (B[:off] == -1).all() and (B[off + 2 * n - 2:] == -1).all(), off   # nothing outside
        C = B[off:off + 2 * n - 2]
        if ref is None:
            ref = C.copy()
            idx = np.unique(np.concatenate([[0, 1, 2, 3, n - 1, n, 2 * n - 3],
                                            np.random.default_rng(5).integers(0, 2 * n - 2, 40)])).astype(np.uint64)
            assert np.array_equal(C[idx.astype(np.int64)], orc.poly_mul_coeffs(Pc, Qc, idx))
        else:
            assert np.array_equal(C, ref), off


def test_poly_extreme_coefficients(F):
    n = 1 << 16
    Pc = np.full(n, 0xFFFF, np.uint16)
    k = np.arange(2 * n - 1)
    want = np.minimum(k + 1, 2 * n - 1 - k).astype(np.int64) * 0xFFFF * 0xFFFF
    assert np.array_equal(poly(F, Pc, Pc), want)


def test_poly_config1_full_size(F, orc):
    """Two polynomials of 2^23 uint16 coefficients (circulant size 2^24): sampled
    coefficients exactly, plus evaluation at random points modulo independent
    61-bit primes (P(t) Q(t) = C(t) mod q)."""
    n = 1 << 23
    Pc, Qc = I.poly_pair(n)
    C = poly(F, Pc, Qc)
    assert C.shape == (2 * n - 1,)
    rng = np.random.default_rng(99)
    idx = np.unique(np.concatenate([[0, 1, n - 1, n, 2 * n - 2, 2 * n - 3],
                                    rng.integers(0, 2 * n - 1, 120)])).astype(np.uint64)
    assert np.array_equal(C[idx.astype(np.int64)], orc.poly_mul_coeffs(Pc, Qc, idx))
    for q in ((1 << 61) - 1, (1 << 62) - 57):   # primes
        t = int(rng.integers(2, q))
        assert orc.eval_i64_mod(C, t, q) == orc.eval_u16_mod(Pc, t, q) * orc.eval_u16_mod(Qc, t, q) % q


def test_poly_host_buffers(F, orc):
    import torch
    Pc, Qc = I.poly_pair(5000, nq=3001)
    out = F.poly_mul_int(torch.from_numpy(Pc.view(np.int16)), torch.from_numpy(Qc.view(np.int16)))
    assert np.array_equal(out.numpy(), orc.poly_mul(Pc, Qc))


def test_poly_pinned_buffers_async_on_two_streams(F, orc):
    """Page-locked host buffers: the call is asynchronous on its stream, so
    two products on two streams are in flight together; after both streams
    finish, both outputs are exact."""
    import torch
    pairs = [I.poly_pair(70000, seed=91), I.poly_pair(40000, nq=50001, seed=92)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for (Pc, Qc), st in zip(pairs, streams):
        Ph = torch.from_numpy(Pc.view(np.int16)).pin_memory()
        Qh = torch.from_numpy(Qc.view(np.int16)).pin_memory()
        Oh = torch.full((Pc.size + Qc.size - 1,), -1, dtype=torch.int64).pin_memory()
        F.poly_mul_int(Ph, Qh, out=Oh, stream=st)
        outs.append((Ph, Qh, Oh))
    for st in streams:
        st.synchronize()
    for (Pc, Qc), (_, _, Oh) in zip(pairs, outs):
        idx = np.unique(np.concatenate([np.arange(8), np.arange(Oh.numel() - 8, Oh.numel()),
                                        np.random.default_rng(3).integers(0, Oh.numel(), 200)]))
        assert np.array_equal(Oh.numpy()[idx], orc.poly_mul_coeffs(Pc, Qc, idx.astype(np.uint64)))


def test_poly_errors(F):
    import torch
    L = F.load()
    z = torch.zeros(4, dtype=torch.int16, device="cuda")
    o = torch.zeros(8, dtype=torch.int64, device="cuda")
    assert L.poly_mul_int(z.data_ptr(), 0, z.data_ptr(), 4, o.data_ptr(), None) == 1
    assert L.poly_mul_int(None, 4, z.data_ptr(), 4, o.data_ptr(), None) == 1
    assert L.poly_mul_int(z.data_ptr(), 1 << 24, z.data_ptr(), 2, o.data_ptr(), None) == 1
