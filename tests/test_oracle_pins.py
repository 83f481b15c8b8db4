"""Pins for the CPU oracle: each routine checked against something other than
itself -- the paper's printed example, special cases with a closed form,
library routines (numpy FFT / convolve, Python big integers), brute force of
the paper's Algorithm 1 on tiny inputs, finite differences.  CPU only."""
import os

import numpy as np
import pytest

from paper_2103_02605_gb300 import inputs as I

P = I.P1
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# -- helpers (test side, plain Python integers) -------------------------------

def sqrt_mod(v, p, other=False):
    """A square root of v mod the odd prime p (Tonelli-Shanks); `other` picks
    the negated root.  Raises if v is a non-residue."""
    v %= p
    if v == 0:
        return 0
    assert pow(v, (p - 1) // 2, p) == 1, "non-residue"
    q, s = p - 1, 0
    while q % 2 == 0:
        q //= 2
        s += 1
    z = 2
    while pow(z, (p - 1) // 2, p) != p - 1:
        z += 1
    m, c, t, r = s, pow(z, q, p), pow(v, q, p), pow(v, (q + 1) // 2, p)
    while t != 1:
        i, t2 = 0, t
        while t2 != 1:
            t2 = t2 * t2 % p
            i += 1
        b = pow(c, 1 << (m - i - 1), p)
        m, c, t, r = i, b * b % p, t * b * b % p, r * b % p
    assert r * r % p == v
    return (p - r) % p if other else r


def algorithm1(a, b, f, p, flip=False, dense2=False):
    """The paper's Algorithm 1 applied recursively (Section 2): the f-circulant
    with row vector a times b.  Block row vectors: A_M1 = A1 + sqrt(f) A2 has
    row a_lo + s a_hi and is s-circulant, A_M2 has row a_lo - s a_hi and is
    (-s)-circulant (structure preservation in the proof of Theorem 1)."""
    n = len(a)
    if n == 1:
        return [a[0] * b[0] % p]
    if dense2 and n == 2:
        return [(a[0] * b[0] + a[1] * b[1]) % p, (f * a[1] * b[0] + a[0] * b[1]) % p]
    s = sqrt_mod(f, p, other=flip)
    h = n // 2
    a1, a2, b1, b2 = a[:h], a[h:], b[:h], b[h:]
    m1 = algorithm1([(u + s * v) % p for u, v in zip(a1, a2)],
                    [(s * u + v) % p for u, v in zip(b1, b2)], s, p, flip, dense2)
    m2 = algorithm1([(u - s * v) % p for u, v in zip(a1, a2)],
                    [(s * u - v) % p for u, v in zip(b1, b2)], (-s) % p, p, flip, dense2)
    inv2 = pow(2, p - 2, p)
    inv2s = pow(2 * s, p - 2, p)
    c1 = [(u + v) * inv2s % p for u, v in zip(m1, m2)]
    c2 = [((u + v) * inv2 - v) % p for u, v in zip(m1, m2)]
    return c1 + c2


def rand_mod(rng, n, p=P):
    return rng.integers(0, p, size=n, dtype=np.uint64).astype(np.uint32)


def parse_golden_3x3():
    rows = []
    with open(os.path.join(GOLDEN, "fcirc_3x3_example.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    assert len(rows) == 3 and all(len(r) == 3 for r in rows)
    return rows


def golden_matrix(rows, a, f, mul, one):
    """Matrix from the printed example: entry 'ak' -> a[k-1], 'ak*f' -> a[k-1]*f."""
    M = []
    for r in rows:
        out = []
        for e in r:
            k = int(e[1])
            v = a[k - 1]
            out.append(mul(v, f) if e.endswith("*f") else mul(v, one))
        M.append(out)
    return M


# -- Definition 2 layout: the paper's 3x3 example -----------------------------

def test_layout_3x3_example_mod(orc):
    rows = parse_golden_3x3()
    rng = np.random.default_rng(1)
    for _ in range(20):
        a = [int(v) for v in rng.integers(0, P, 3)]
        x = [int(v) for v in rng.integers(0, P, 3)]
        f = int(rng.integers(0, P))
        M = golden_matrix(rows, a, f, lambda u, v: u * v % P, 1)
        want = [sum(M[i][j] * x[j] for j in range(3)) % P for i in range(3)]
        got = orc.fcirc_matvec_mod(P, f, a, x)
        assert [int(v) for v in got] == want


def test_layout_3x3_example_complex(orc):
    rows = parse_golden_3x3()
    rng = np.random.default_rng(2)
    a = rng.normal(size=3) + 1j * rng.normal(size=3)
    x = rng.normal(size=3) + 1j * rng.normal(size=3)
    f = 0.3 - 1.7j
    M = np.array(golden_matrix(rows, a, f, lambda u, v: u * v, 1.0))
    np.testing.assert_allclose(orc.fcirc_matvec_c128(f, a, x), M @ x, rtol=1e-13)


# -- closed-form special cases -------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 64])
def test_identity_row(orc, n):
    """a = e_0 gives the identity matrix for every f."""
    rng = np.random.default_rng(n)
    x = rand_mod(rng, n)
    a = np.zeros(n, np.uint32)
    a[0] = 1
    for f in (0, 1, 12345, P - 1):
        assert np.array_equal(orc.fcirc_matvec_mod(P, f, a, x), x)


@pytest.mark.parametrize("n", [2, 3, 7, 16])
def test_shift_row(orc, n):
    """a = e_1: c_i = x_{i+1} for i < n-1 and c_{n-1} = f x_0 (the f-shift)."""
    rng = np.random.default_rng(10 + n)
    x = rand_mod(rng, n)
    a = np.zeros(n, np.uint32)
    a[1] = 1
    f = 987654321
    c = orc.fcirc_matvec_mod(P, f, a, x)
    want = np.concatenate([x[1:], [f * int(x[0]) % P]]).astype(np.uint32)
    assert np.array_equal(c, want)


@pytest.mark.parametrize("n", [1, 4, 6, 32, 100])
def test_f1_is_ordinary_circulant_fft(orc, n):
    """f = 1 is the usual circulant (text after Definition 2) in the row
    convention: c_i = sum_k a_k x_{(i+k) mod n}, i.e. a cyclic correlation,
    computed here with numpy's FFT."""
    rng = np.random.default_rng(100 + n)
    a = rng.normal(size=(3, n)) + 1j * rng.normal(size=(3, n))
    x = rng.normal(size=(3, n)) + 1j * rng.normal(size=(3, n))
    want = np.fft.ifft(n * np.fft.ifft(a, axis=-1) * np.fft.fft(x, axis=-1), axis=-1)
    np.testing.assert_allclose(orc.fcirc_matvec_c128(1.0, a, x), want, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("n,f", [(8, 2.0), (16, -1.0), (5, 0.5 + 0.5j), (32, np.exp(0.7j))])
def test_general_f_by_diagonal_scaling_fft(orc, n, f):
    """With r any n-th root of f, A = D_r C(a_k r^k) D_r^{-1} where C is the
    ordinary circulant and D_r = diag(r^i): checked with numpy's FFT."""
    rng = np.random.default_rng(200 + n)
    a = rng.normal(size=n) + 1j * rng.normal(size=n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    r = complex(f) ** (1.0 / n)
    k = np.arange(n)
    a2 = a * r ** k
    x2 = x * r ** (-k)
    circ = np.fft.ifft(n * np.fft.ifft(a2) * np.fft.fft(x2))
    want = r ** k * circ
    np.testing.assert_allclose(orc.fcirc_matvec_c128(f, a, x), want, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 8, 16])
def test_transpose_is_polynomial_product_mod_xn_minus_f(orc, n):
    """Column j of A is A e_j; the transpose of A then multiplies polynomials
    modulo z^n - f: (A^T x)(z) = a(z) x(z) mod (z^n - f)."""
    rng = np.random.default_rng(300 + n)
    a = rand_mod(rng, n)
    x = [int(v) for v in rand_mod(rng, n)]
    f = int(rng.integers(1, P))
    cols = []
    for j in range(n):
        e = np.zeros(n, np.uint32)
        e[j] = 1
        cols.append([int(v) for v in orc.fcirc_matvec_mod(P, f, a, e)])
    # A^T x: (A^T x)_j = sum_i A[i][j] x_i = sum_i cols[j][i] x_i
    atx = [sum(cols[j][i] * x[i] for i in range(n)) % P for j in range(n)]
    prod = np.convolve(np.array([int(v) for v in a], dtype=object), np.array(x, dtype=object))
    red = [0] * n
    for k, v in enumerate(prod):
        red[k % n] = (red[k % n] + (v if k < n else f * v)) % P
    assert atx == red


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16])
def test_column_convention_is_the_transpose(orc, n):
    """The column-convention oracle equals A^T x with A built column by
    column from the row-convention oracle (A e_j), and reduces to the
    identity for a = e_0 and to a for x = e_0."""
    rng = np.random.default_rng(400 + n)
    a = rand_mod(rng, n)
    x = rand_mod(rng, n)
    f = int(rng.integers(1, P))
    cols = []
    for j in range(n):
        e = np.zeros(n, np.uint32)
        e[j] = 1
        cols.append([int(v) for v in orc.fcirc_matvec_mod(P, f, a, e)])
    want = [sum(cols[j][i] * int(x[i]) for i in range(n)) % P for j in range(n)]
    assert [int(v) for v in orc.fcirc_matvec_t_mod(P, f, a, x)] == want
    e0 = np.zeros(n, np.uint32)
    e0[0] = 1
    assert np.array_equal(orc.fcirc_matvec_t_mod(P, f, e0, x), x)
    assert np.array_equal(orc.fcirc_matvec_t_mod(P, f, a, e0), a)


@pytest.mark.parametrize("n", [1, 2, 3, 6, 11])
def test_toeplitz_oracle(orc, n):
    """The Toeplitz oracle against a Python dense product, and against the
    f-circulant oracle for the Toeplitz matrix an f-circulant is (diagonal
    k >= 0 holds a_k, diagonal -m holds f a_{n-m}, Definition 2)."""
    rng = np.random.default_rng(500 + n)
    t = rand_mod(rng, 2 * n - 1)
    x = rand_mod(rng, n)
    want = [sum(int(t[j - i + n - 1]) * int(x[j]) for j in range(n)) % P for i in range(n)]
    assert [int(v) for v in orc.toeplitz_matvec_mod(P, t, x)] == want
    a = rand_mod(rng, n)
    f = int(rng.integers(1, P))
    tc = np.zeros(2 * n - 1, np.uint32)
    for k in range(n):
        tc[n - 1 + k] = a[k]
    for m in range(1, n):
        tc[n - 1 - m] = f * int(a[n - m]) % P
    assert np.array_equal(orc.toeplitz_matvec_mod(P, tc, x), orc.fcirc_matvec_mod(P, f, a, x))


# -- the paper's own field GF(p^2) = Z/pZ[sqrt 3], p = 2^31 - 1 ----------------

GFP = (1 << 31) - 1


def _gf_pairs(rng, n):
    return rng.integers(0, GFP, (n, 2), dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("n", [1, 2, 3, 8, 16])
def test_gf_oracle_is_four_products_over_the_prime_field(orc, n):
    """With f in Z/pZ the product splits: (A1 + s A2)(x1 + s x2) =
    (A1 x1 + 3 A2 x2) + s (A1 x2 + A2 x1), s = sqrt 3, each term a product of
    the modular oracle over p = 2^31 - 1 (linearity of Definition 2 in a)."""
    rng = np.random.default_rng(600 + n)
    a, x = _gf_pairs(rng, n), _gf_pairs(rng, n)
    f = int(rng.integers(1, GFP))
    got = orc.fcirc_matvec_gf((f, 0), a, x)
    m = lambda u, v: orc.fcirc_matvec_mod(GFP, f, u, v).astype(np.uint64)
    a1, a2, x1, x2 = a[:, 0], a[:, 1], x[:, 0], x[:, 1]
    re = (m(a1, x1) + 3 * m(a2, x2)) % GFP
    im = (m(a1, x2) + m(a2, x1)) % GFP
    assert np.array_equal(got[:, 0], re.astype(np.uint32)) and np.array_equal(got[:, 1], im.astype(np.uint32))


@pytest.mark.parametrize("n", [2, 5, 8])
def test_gf_oracle_shift_and_identity_rows(orc, n):
    """a = e_0 gives x; a = e_1 gives the f-shift c_i = x_{i+1}, c_{n-1} = f x_0
    (f with a sqrt 3 part: the only place the field's product with f shows)."""
    rng = np.random.default_rng(700 + n)
    x = _gf_pairs(rng, n)
    fr, fi = (int(v) for v in rng.integers(1, GFP, 2))
    e0 = np.zeros((n, 2), np.uint32)
    e0[0, 0] = 1
    assert np.array_equal(orc.fcirc_matvec_gf((fr, fi), e0, x), x)
    e1 = np.zeros((n, 2), np.uint32)
    e1[1, 0] = 1
    got = orc.fcirc_matvec_gf((fr, fi), e1, x)
    assert np.array_equal(got[:-1], x[1:])
    xr, xi = int(x[0, 0]), int(x[0, 1])
    assert (int(got[-1, 0]), int(got[-1, 1])) == ((fr * xr + 3 * fi * xi) % GFP, (fr * xi + fi * xr) % GFP)


# -- the ring Z/(2^K + 1) of Schoenhage-Strassen multiplication -------------------

@pytest.mark.parametrize("n", [1, 2, 8, 32])
def test_ssa_oracle_small_values_are_the_integer_product(orc, n):
    """Entries below 2^8 keep every sum far below 2^64: the ring product with
    f = 1 is the integer cyclic correlation (numpy), and with f = -1 (2^K) the
    wrapped terms change sign (Definition 2)."""
    rng = np.random.default_rng(800 + n)
    a = rng.integers(0, 256, n)
    x = rng.integers(0, 256, n)
    corr = [int(sum(a[k] * x[(i + k) % n] for k in range(n))) for i in range(n)]
    assert orc.fcirc_matvec_ssa(64, 0, [int(v) for v in a], [int(v) for v in x]) == corr
    M = (1 << 64) + 1
    neg = [int(sum((1 if i + k < n else -1) * a[k] * x[(i + k) % n] for k in range(n))) % M for i in range(n)]
    assert orc.fcirc_matvec_ssa(64, 64, [int(v) for v in a], [int(v) for v in x]) == neg


@pytest.mark.parametrize("K", [64, 128])
def test_ssa_oracle_identity_and_shift_rows(orc, K):
    n = 8
    M = (1 << K) + 1
    x = I.ssa_elements(n, K, seed=K)
    e0 = [1] + [0] * (n - 1)
    assert orc.fcirc_matvec_ssa(K, 5, e0, x) == x
    e1 = [0, 1] + [0] * (n - 2)
    got = orc.fcirc_matvec_ssa(K, 5, e1, x)
    assert got[:-1] == x[1:] and got[-1] == (x[0] << 5) % M


# -- the paper's Algorithm 1 (brute force) agrees with the dense oracle ----------

@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("froot", [1, None])
def test_algorithm1_bruteforce_equals_dense(orc, n, froot):
    rng = np.random.default_rng(400 + n)
    a = [int(v) for v in rand_mod(rng, n)]
    b = [int(v) for v in rand_mod(rng, n)]
    r = 1 if froot == 1 else int(rng.integers(2, P))
    f = pow(r, n, P)                     # an f with an n-th root (Theorem 1)
    want = [int(v) for v in orc.fcirc_matvec_mod(P, f, a, b)]
    assert algorithm1(a, b, f, P) == want
    # either square root may be taken at every node: same product
    assert algorithm1(a, b, f, P, flip=True) == want
    # stopping at dense 2x2 f'-circulant leaves gives the same product
    assert algorithm1(a, b, f, P, dense2=True) == want


def test_algorithm1_n2_closed_form():
    """Algorithm 1 with 1x1 blocks: c1 = a0 b0 + a1 b1, c2 = f a1 b0 + a0 b1."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        a0, a1, b0, b1, r = (int(v) for v in rng.integers(1, P, 5))
        f = r * r % P
        assert algorithm1([a0, a1], [b0, b1], f, P) == [
            (a0 * b0 + a1 * b1) % P, (f * a1 * b0 + a0 * b1) % P]


# -- sampled rows and batches are the same product ----------------------------

def test_rows_and_batched_agree_with_full(orc):
    rng = np.random.default_rng(11)
    n = 257
    a, x = rand_mod(rng, n), rand_mod(rng, n)
    full = orc.fcirc_matvec_mod(P, 77, a, x)
    rows = np.array([0, 1, 100, 255, 256], dtype=np.uint64)
    assert np.array_equal(orc.fcirc_matvec_mod_rows(P, 77, a, x, rows), full[rows])
    ns = [4, 1, 16, 9]
    offs = np.concatenate([[0], np.cumsum(ns)]).astype(np.uint64)
    A, X = rand_mod(rng, offs[-1]), rand_mod(rng, offs[-1])
    fs = np.array([3, 1, P - 1, 12], np.uint32)
    got = orc.fcirc_matvec_mod_batched(P, fs, offs, A, X)
    for i in range(len(ns)):
        s, e = int(offs[i]), int(offs[i + 1])
        assert np.array_equal(got[s:e], orc.fcirc_matvec_mod(P, int(fs[i]), A[s:e], X[s:e]))


# -- complex gradients: finite differences and the adjoint identity ----------

@pytest.mark.parametrize("f", [1.0, -1.0, 0.6 + 0.8j, 2.0 - 0.5j])
def test_complex_gradients_finite_differences(orc, f):
    rng = np.random.default_rng(500)
    n = 8
    a = rng.normal(size=n) + 1j * rng.normal(size=n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    g = rng.normal(size=n) + 1j * rng.normal(size=n)

    def loss(a_, x_):
        return float(np.real(np.vdot(g, orc.fcirc_matvec_c128(f, a_, x_))))

    ga, gx = orc.fcirc_grad_c128(f, a, x, g)
    h = 1e-6
    for which, grad in (("a", ga), ("x", gx)):
        fd = np.zeros(n, complex)
        for k in range(n):
            for unit, w in ((1.0, 1.0), (1j, 1j)):
                e = np.zeros(n, complex)
                e[k] = unit * h
                if which == "a":
                    d = (loss(a + e, x) - loss(a - e, x)) / (2 * h)
                else:
                    d = (loss(a, x + e) - loss(a, x - e)) / (2 * h)
                fd[k] += d * w
        np.testing.assert_allclose(grad, fd, rtol=1e-7, atol=1e-7)


def test_complex_adjoint_dot(orc):
    rng = np.random.default_rng(501)
    n, f = 64, 0.3 + 1.1j
    a = rng.normal(size=n) + 1j * rng.normal(size=n)
    x = rng.normal(size=n) + 1j * rng.normal(size=n)
    g = rng.normal(size=n) + 1j * rng.normal(size=n)
    _, gx = orc.fcirc_grad_c128(f, a, x, g)
    lhs = np.vdot(g, orc.fcirc_matvec_c128(f, a, x))
    rhs = np.vdot(gx, x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs) * n


# -- polynomial and large-integer products (Section 3) -------------------------

@pytest.mark.parametrize("np_,nq", [(1, 1), (1, 9), (8, 8), (13, 70), (512, 300)])
def test_poly_mul_vs_numpy_convolve(orc, np_, nq):
    rng = np.random.default_rng(600 + np_)
    Pp = rng.integers(0, 1 << 16, np_).astype(np.uint16)
    Q = rng.integers(0, 1 << 16, nq).astype(np.uint16)
    want = np.convolve(Pp.astype(np.int64), Q.astype(np.int64))
    got = orc.poly_mul(Pp, Q)
    assert np.array_equal(got, want)
    idx = np.array([0, len(want) - 1, len(want) // 2], np.uint64)
    assert np.array_equal(orc.poly_mul_coeffs(Pp, Q, idx), want[idx.astype(np.int64)])


def test_poly_extreme_coefficients(orc):
    n = 4096
    Pp = np.full(n, 0xFFFF, np.uint16)
    got = orc.poly_mul(Pp, Pp)
    k = np.arange(2 * n - 1)
    want = np.minimum(k + 1, 2 * n - 1 - k).astype(np.int64) * 0xFFFF * 0xFFFF
    assert np.array_equal(got, want)


@pytest.mark.parametrize("na,nb", [(1, 1), (3, 5), (64, 64), (1000, 777)])
def test_bigint_mul_vs_python_int(orc, na, nb):
    A, B = I.bigint_pair(16 * max(na, nb), seed=900 + na)
    A, B = A[:na], B[:nb]
    want = I.limbs_to_int(A) * I.limbs_to_int(B)
    got = orc.bigint_mul(A, B)
    assert got.size == na + nb
    assert I.limbs_to_int(got) == want


def test_bigint_all_ones(orc):
    n = 300
    A = np.full(n, 0xFFFF, np.uint16)
    v = (1 << (16 * n)) - 1
    assert I.limbs_to_int(orc.bigint_mul(A, A)) == v * v


def test_bigint_columns_are_poly_coefficients(orc):
    A, B = I.bigint_pair(16 * 200, seed=5)
    idx = np.arange(399, dtype=np.uint64)
    cols = orc.bigint_columns(A, B, idx)
    assert np.array_equal(cols.astype(np.int64), np.convolve(A.astype(np.int64), B.astype(np.int64)))
    assert sum(int(c) << (16 * k) for k, c in enumerate(cols)) == I.limbs_to_int(A) * I.limbs_to_int(B)


def test_eval_mod_q(orc):
    q = (1 << 61) - 1
    rng = np.random.default_rng(12)
    c16 = rng.integers(0, 1 << 16, 777).astype(np.uint16)
    c64 = rng.integers(0, 1 << 62, 555).astype(np.int64)
    t = int(rng.integers(2, q))
    assert orc.eval_u16_mod(c16, t, q) == sum(int(v) * pow(t, k, q) for k, v in enumerate(c16)) % q
    assert orc.eval_i64_mod(c64, t, q) == sum(int(v) * pow(t, k, q) for k, v in enumerate(c64)) % q
    # P(t) Q(t) = (PQ)(t) for the oracle's product
    Pp, Q = c16[:300], c16[300:700]
    C = orc.poly_mul(Pp, Q)
    assert orc.eval_i64_mod(C, t, q) == orc.eval_u16_mod(Pp, t, q) * orc.eval_u16_mod(Q, t, q) % q
