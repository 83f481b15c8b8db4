"""CPU tests of the library's host side: the shared object loads and exports
every function the public headers declare, and the root chains / twiddle
numbers of the plans satisfy what the recursion needs (no GPU calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P1, P2, P3 = 998244353, 469762049, 167772161


@pytest.fixture(scope="module")
def F():
    from paper_2103_02605_gb300 import build
    build.build()
    import paper_2103_02605_gb300 as F
    F.load()
    return F


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_library_exports_every_declared_symbol(F):
    names = declared_functions()
    assert "fcirc_matvec" in names and "poly_mul_int" in names
    lib = ctypes.CDLL(F.library_path())
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_error_strings(F):
    L = F.load()
    for code in range(6):
        assert L.fcirc_error_string(code).decode().startswith("FCIRC_")


def test_two_adic_limits(F):
    # n may reach 2^(v+1): 2^24, 2^27, 2^26 for the three primes
    for p, v in ((P1, 23), (P2, 26), (P3, 25)):
        assert (p - 1) % (1 << v) == 0 and (p - 1) % (1 << (v + 1)) != 0
        F.node_twiddle(p, 1, 1 << (v + 1), v - 1, 0)
        with pytest.raises(F.FcircError) as e:
            F.node_twiddle(p, 1, 1 << (v + 2), 0, 0)
        assert e.value.status == 2  # ENOROOT


@pytest.mark.parametrize("p", [P1, P2, P3, 17, 97, 7681, 12289])
def test_nth_root_matches_existence_criterion(F, p):
    rng = np.random.default_rng(p)
    v = ((p - 1) & -(p - 1)).bit_length() - 1
    for _ in range(60):
        f = int(rng.integers(1, p))
        k = int(rng.integers(0, v + 3))
        g = np.gcd(1 << k, p - 1)
        exists = pow(f, (p - 1) // int(g), p) == 1
        if exists:
            r = F.nth_root(p, f, k)
            assert pow(r, 1 << k, p) == f
        else:
            with pytest.raises(F.FcircError):
                F.nth_root(p, f, k)
    # perfect powers always have roots
    for _ in range(20):
        r0 = int(rng.integers(1, p))
        k = int(rng.integers(0, min(v, 12) + 1))
        f = pow(r0, 1 << k, p)
        assert pow(F.nth_root(p, f, k), 1 << k, p) == f


def test_nth_root_rejects_bad_input(F):
    for p in (1, 2, 4, 15, 1 << 31, 2147483647):
        with pytest.raises(F.FcircError):
            F.nth_root(p, 1, 1)
    with pytest.raises(F.FcircError):
        F.nth_root(P1, 0, 3)


@pytest.mark.parametrize("p,f,m", [(P1, 1, 6), (P1, 5, 5), (P2, 7, 7), (P3, 1, 4), (97, 3, 4)])
def test_node_twiddles_form_a_square_root_chain(F, p, f, m):
    """s_{0,0}^2 = f, and s_{l,j}^2 = +s_{l-1,j/2} for even j, -s_{l-1,j/2} for
    odd j: the children of an f'-circulant are sqrt(f')- and (-sqrt(f'))-circulant
    (structure preservation in the proof of Theorem 1)."""
    n = 1 << m
    L = m - 1
    try:
        F.nth_root(p, f, L)
    except F.FcircError:
        f = pow(f, 1 << L, p)
    s00, si00 = F.node_twiddle(p, f, n, 0, 0)
    assert s00 * s00 % p == f % p and s00 * si00 % p == 1
    for l in range(1, L):
        for j in range(1 << l):
            s, si = F.node_twiddle(p, f, n, l, j)
            par, _ = F.node_twiddle(p, f, n, l - 1, j >> 1)
            assert s * s % p == (par if j % 2 == 0 else (p - par) % p)
            assert s * si % p == 1
    for j in range(n // 2):
        phi = F.leaf_param(p, f, n, j)
        par, _ = F.node_twiddle(p, f, n, L - 1, j >> 1) if L >= 1 else (f, 0)
        assert phi == (par if j % 2 == 0 else (p - par) % p)


def test_leaf_params_are_the_roots_of_z_n_minus_f(F):
    """The n/2 leaf parameters are the distinct square roots' parents: the
    polynomials z^2 - phi_j multiply to z^n - f, i.e. {phi_j} are the n/2
    distinct (n/2)-th roots of f."""
    p, m = P1, 6
    n = 1 << m
    f = pow(31337, n // 2, p)
    phis = [F.leaf_param(p, f, n, j) for j in range(n // 2)]
    assert len(set(phis)) == n // 2
    for ph in phis:
        assert pow(ph, n // 2, p) == f


def test_inverse_root_identity_of_section_3_1(F):
    """The inverse of the 4th root of i is -i * sqrt(i) * 4th root of i, for the
    chain i = psi_4, sqrt(i) = psi_8, 4th root of i = psi_16 the plans use."""
    for p in (P1, P2, P3):
        n = 32   # levels 0..3 exist; level l uses psi_{2^(l+1)}^brv_l(j)
        i_, _ = F.node_twiddle(p, 1, n, 1, 1)        # psi_4
        r2, _ = F.node_twiddle(p, 1, n, 2, 2)        # psi_8   (brv_2(2) = 1)
        r4, r4inv = F.node_twiddle(p, 1, n, 3, 4)    # psi_16  (brv_3(4) = 1)
        assert i_ * i_ % p == p - 1                  # i = sqrt(-1)
        assert r2 * r2 % p == i_ and r4 * r4 % p == r2
        assert r4inv == (p - i_) * r2 % p * r4 % p


def test_twiddle_from_factor_matches_exact_division(F):
    rng = np.random.default_rng(3)
    for p in (P1, P2, P3, 3, 5, 7681, (1 << 30) - 35):
        if any(p % q == 0 for q in range(2, int(p ** 0.5) + 1)):
            continue
        for _ in range(400):
            u = int(rng.integers(0, p))
            s = int(rng.integers(0, p))
            w, wp = F.twiddle_from_factor(p, u, s)
            assert w == u * s % p
            assert wp == (w << 32) // p
        for u, s in ((0, 0), (p - 1, p - 1), (1, p - 1), (p - 1, 1), (0, p - 1)):
            w, wp = F.twiddle_from_factor(p, u, s)
            assert (w, wp) == (u * s % p, ((u * s % p) << 32) // p)


# -- the paper's field GF(p^2) = Z/pZ[sqrt 3], p = 2^31 - 1 -------------------------

GFP = (1 << 31) - 1


def _gmul(a, b):
    return ((a[0] * b[0] + 3 * a[1] * b[1]) % GFP, (a[0] * b[1] + a[1] * b[0]) % GFP)


def _gpow(a, e):
    r = (1, 0)
    while e:
        if e & 1:
            r = _gmul(r, a)
        a = _gmul(a, a)
        e >>= 1
    return r


def _gf_root(F, f, k):
    import ctypes
    rr, ri = ctypes.c_uint32(), ctypes.c_uint32()
    st = F.load().fcirc_gf_nth_root(f[0], f[1], k, ctypes.byref(rr), ctypes.byref(ri))
    return st, (rr.value, ri.value)


def test_gf_roots(F):
    """Roots in the paper's field: r^(2^k) = f for f that are 2^k-th powers;
    3 is not a square mod p (so sqrt 3 extends Z/pZ); the element of order
    2^32 has no square root; -1 has roots up to order 2^31 (p + 1 = 2^31)."""
    assert pow(3, (GFP - 1) // 2, GFP) == GFP - 1
    rng = np.random.default_rng(5)
    for k in (0, 1, 5, 11, 30):
        for _ in range(4):
            b = tuple(int(v) for v in rng.integers(1, GFP, 2))
            f = _gpow(b, 1 << k)
            st, r = _gf_root(F, f, k)
            assert st == 0 and _gpow(r, 1 << k) == f
    st, r = _gf_root(F, (GFP - 1, 0), 30)
    assert st == 0 and _gpow(r, 1 << 30) == (GFP - 1, 0)
    # a generator g of the 2-Sylow subgroup: g^2 = 2 + sqrt 3 (the paper's generator)
    st, g = _gf_root(F, (2, 1), 1)
    assert st == 0 and _gpow(g, 1 << 31) == (GFP - 1, 0)
    assert _gf_root(F, g, 1)[0] == 2
    assert _gf_root(F, (0, 0), 3)[0] == 2
    assert _gf_root(F, (GFP, 0), 3)[0] == 1


def test_mul_probe_rejects_bad_arguments_before_any_device_call(F):
    import ctypes as C
    L = F.load()
    ms, rate = C.c_double(), C.c_double()
    assert L.fcirc_prof_mul_probe(2, 4, 16, C.byref(ms), C.byref(rate)) == 1     # kind
    assert L.fcirc_prof_mul_probe(0, 0, 16, C.byref(ms), C.byref(rate)) == 1     # no CTAs
    assert L.fcirc_prof_mul_probe(0, 9, 16, C.byref(ms), C.byref(rate)) == 1     # too many
    assert L.fcirc_prof_mul_probe(0, 4, 0, C.byref(ms), C.byref(rate)) == 1      # no work
    assert L.fcirc_prof_mul_probe(0, 4, 16, None, C.byref(rate)) == 1
