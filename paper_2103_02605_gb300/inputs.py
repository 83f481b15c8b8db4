"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds random-number generation only -- no arithmetic of the
circulant method.  Both sides of every parity check (the CUDA library and
the CPU oracle) receive the same arrays from here.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then the
xor-shift-multiply finaliser with constants 0xBF58476D1CE4E5B9 and
0x94D049BB133111EB.  Draws are consumed in order from one stream per seed.

Distributions:
  * uniform residues in [0, p): rejection sampling on the top 32 bits;
  * uniform 16-bit values (polynomial coefficients, integer limbs): top 16
    bits of each draw;
  * standard normals: Box-Muller in float64 on two 53-bit uniforms, then
    rounded to float32.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

SEED_BASE = 2103026050

P1, P2, P3 = 998244353, 469762049, 167772161
PRIMES = (P1, P2, P3)


class SplitMix64:
    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, count: int) -> np.ndarray:
        count = int(count)
        k = np.arange(1, count + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = self.state + k * GOLDEN
            self.state = self.state + np.uint64(count) * GOLDEN
            z = (z ^ (z >> np.uint64(30))) * M1
            z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))

    def uniform_mod(self, p: int, count: int) -> np.ndarray:
        """count values uniform in [0, p) (p <= 2^32), exact by rejection."""
        lim = np.uint64((2 ** 32 // p) * p)
        out = np.empty(count, dtype=np.uint32)
        got = 0
        while got < count:
            # draw exactly as many as are still missing; every draw is
            # consumed in order, accepted or rejected
            v = self.next_u64(count - got) >> np.uint64(32)
            v = v[v < lim]
            out[got:got + v.size] = (v % np.uint64(p)).astype(np.uint32)
            got += v.size
        return out

    def uniform_u16(self, count: int) -> np.ndarray:
        return (self.next_u64(count) >> np.uint64(48)).astype(np.uint16)

    def normal_f32(self, count: int) -> np.ndarray:
        m = (count + 1) // 2
        z = self.next_u64(2 * m)
        u1 = ((z[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
        u2 = (z[1::2] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        r = np.sqrt(-2.0 * np.log(u1))
        out = np.empty(2 * m, dtype=np.float64)
        out[0::2] = r * np.cos(2.0 * np.pi * u2)
        out[1::2] = r * np.sin(2.0 * np.pi * u2)
        return out[:count].astype(np.float32)

    def complex_normal_c64(self, shape) -> np.ndarray:
        count = int(np.prod(shape))
        v = self.normal_f32(2 * count)
        return v.view(np.complex64).reshape(shape)


# -- named workloads ---------------------------------------------------------

def single_mod(n: int, p: int = P1, seed: int = SEED_BASE + 0):
    """Row vector a and vector x, uniform in [0, p)."""
    g = SplitMix64(seed)
    return g.uniform_mod(p, n), g.uniform_mod(p, n)


def poly_pair(n_coeffs: int, seed: int = SEED_BASE + 1, nq: int | None = None):
    """Two integer polynomials with coefficients uniform in [0, 2^16)."""
    g = SplitMix64(seed)
    P = g.uniform_u16(n_coeffs)
    Q = g.uniform_u16(n_coeffs if nq is None else nq)
    return P, Q


def complex_layer(batch: int, n: int, seed: int = SEED_BASE + 2):
    """a, x, g complex64 of shape (batch, n), real/imag i.i.d. N(0, 1)."""
    g = SplitMix64(seed)
    a = g.complex_normal_c64((batch, n))
    x = g.complex_normal_c64((batch, n))
    gr = g.complex_normal_c64((batch, n))
    return a, x, gr


def primitive_2k_root(p: int, k: int) -> int:
    """A primitive 2^k-th root of unity mod p, as 3^((p-1)/2^k) (3 generates
    the unit group of each of the three primes above).  Used only to build
    the f values of the batched workload."""
    assert (p - 1) % (1 << k) == 0
    return pow(3, (p - 1) >> k, p)


def batched_mod(count: int = 10_000, log_lo: int = 6, log_hi: int = 16,
                p: int = P1, seed: int = SEED_BASE + 3):
    """Uneven batch: n_i = 2^e, e uniform in [log_lo, log_hi]; f_i = w^m_i
    with w a primitive 2^23-th root of unity and m_i = (k_i * n_i) mod 2^23,
    k_i uniform in [0, 2^23) (so that each f_i has an n_i-th root, namely
    w^k_i); a and x uniform in [0, p).

    Returns (n, f, offsets, a, x) with a and x packed back to back."""
    g = SplitMix64(seed)
    e = log_lo + (g.next_u64(count) % np.uint64(log_hi - log_lo + 1)).astype(np.int64)
    n = (np.int64(1) << e).astype(np.uint64)
    k = (g.next_u64(count) >> np.uint64(41)).astype(np.int64)  # uniform in [0, 2^23)
    w = primitive_2k_root(p, 23)
    m = (k * n.astype(np.int64)) % (1 << 23)
    f = np.array([pow(w, int(mi), p) for mi in m], dtype=np.uint32)
    offsets = np.zeros(count + 1, dtype=np.uint64)
    np.cumsum(n, out=offsets[1:])
    total = int(offsets[-1])
    a = g.uniform_mod(p, total)
    x = g.uniform_mod(p, total)
    return n, f, offsets, a, x


def bigint_pair(bits: int = 1 << 26, seed: int = SEED_BASE + 4):
    """Two unsigned integers of `bits` uniform random bits, as little-endian
    16-bit limbs."""
    assert bits % 16 == 0
    g = SplitMix64(seed)
    return g.uniform_u16(bits // 16), g.uniform_u16(bits // 16)


def ssa_to_words(values, K: int) -> np.ndarray:
    """Elements of Z/(2^K + 1) (Python ints in [0, 2^K]) in the library's
    layout: K/64 little-endian uint64 words and a top word per element."""
    W = K // 64
    out = np.zeros((len(values), W + 1), np.uint64)
    for i, v in enumerate(values):
        assert 0 <= v <= (1 << K)
        if v == 1 << K:
            out[i, W] = 1
        else:
            for j in range(W):
                out[i, j] = (v >> (64 * j)) & 0xFFFFFFFFFFFFFFFF
    return out


def ssa_from_words(words) -> list:
    w = np.asarray(words, np.uint64)
    W = w.shape[-1] - 1
    return [sum(int(row[j]) << (64 * j) for j in range(W)) + (int(row[W]) << (64 * W)) for row in w.reshape(-1, W + 1)]


def ssa_elements(n: int, K: int, seed: int) -> list:
    """Elements of Z/(2^K + 1) of K random bits each from the seeded
    generator, with the edge values 0, 1, 2^K - 1 and 2^K planted at the
    first positions."""
    W = K // 64
    words = SplitMix64(seed).next_u64(n * W).reshape(n, W)
    vals = [sum(int(words[i, j]) << (64 * j) for j in range(W)) for i in range(n)]
    for i, e in enumerate((0, 1, (1 << K) - 1, 1 << K)):
        if i < n:
            vals[i] = e
    return vals


def limbs_to_int(limbs) -> int:
    """Python int from little-endian 16-bit limbs (exact)."""
    b = np.ascontiguousarray(limbs, dtype="<u2").tobytes()
    return int.from_bytes(b, "little")


def int_to_limbs(v: int, nlimbs: int) -> np.ndarray:
    return np.frombuffer(v.to_bytes(2 * nlimbs, "little"), dtype="<u2").astype(np.uint16)
