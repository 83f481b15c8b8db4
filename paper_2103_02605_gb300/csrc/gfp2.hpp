// gfp2.hpp -- arithmetic in the paper's own field GF(p^2) = Z/pZ[sqrt 3],
// p = 2^31 - 1 (Section 3.1: 3 is not a square mod p, so sqrt 3 generates the
// quadratic extension; p + 1 = 2^31, and 2 + sqrt 3 generates the subgroup
// of order p + 1, so every power-of-two root of unity Algorithm 1 needs up
// to order 2^31 is a power of it).  Shared by the host plan builder and the
// kernels.
//
// An element is (re, im) = re + im sqrt 3 with canonical re, im in [0, p).
// Products reduce with the Mersenne identity 2^31 = 1 (mod p).
#pragma once
#include <stdint.h>

#include "modarith.cuh"   // FCIRC_HD, reduce_min

namespace fcirc {
namespace gf {

constexpr uint32_t P = 0x7FFFFFFFu;   // 2^31 - 1

struct E {
    uint32_t re, im;
};

// x mod p for any 64-bit x (two folds of 2^31 = 1, one subtraction)
// x mod p for x < 2^63, in 32-bit words (2^31 = 1 mod p): with
// x = lo + 2^31 h, h = x >> 31 < 2^32 is first folded to h' = (h & p) +
// (h >> 31) <= 2^31, so that lo + h' <= p + 2^31 = 2^32 - 1 does not
// overflow; one more fold leaves t <= p + 1, and one add-and-min
// (reduce_min) makes it canonical.
FCIRC_HD uint32_t red(uint64_t x)
{
    const uint32_t lo = (uint32_t)x & P;
    uint32_t h = (uint32_t)(x >> 31);
    h = (h & P) + (h >> 31);                    // <= 2^31
    const uint32_t s = lo + h;                  // <= 2^32 - 1
    const uint32_t t = (s & P) + (s >> 31);     // <= p + 1
    return reduce_min(t, P);
}

// a + b for canonical a, b (the sum is below 2p < 2^32)
FCIRC_HD uint32_t add1(uint32_t a, uint32_t b) { return reduce_min(a + b, P); }

FCIRC_HD uint32_t sub1(uint32_t a, uint32_t b) { return add1(a, P - b); }

FCIRC_HD E add(E a, E b) { return E{add1(a.re, b.re), add1(a.im, b.im)}; }
FCIRC_HD E sub(E a, E b) { return E{sub1(a.re, b.re), sub1(a.im, b.im)}; }
// p - a, with p itself (a = 0) reduced to 0
FCIRC_HD E neg(E a) { return E{reduce_min(P - a.re, P), reduce_min(P - a.im, P)}; }

// (a + b s)(c + d s) = (ac + 3 bd) + (ad + bc) s, s = sqrt 3
FCIRC_HD E mul(E a, E b)
{
    const uint32_t bd = red((uint64_t)a.im * b.im);
    const uint64_t re = (uint64_t)a.re * b.re + 3ull * bd;                 // < 2^62 + 2^33
    const uint64_t im = (uint64_t)a.re * b.im + (uint64_t)a.im * b.re;     // < 2^63
    return E{red(re), red(im)};
}

FCIRC_HD E pow(E b, uint64_t e)
{
    E r{1u, 0u};
    while (e) {
        if (e & 1) r = mul(r, b);
        b = mul(b, b);
        e >>= 1;
    }
    return r;
}

FCIRC_HD bool eq(E a, E b) { return a.re == b.re && a.im == b.im; }
FCIRC_HD bool is_zero(E a) { return a.re == 0 && a.im == 0; }

// (a + b s)^-1 = (a - b s) / (a^2 - 3 b^2); the norm is a nonzero element of
// Z/pZ for a nonzero element (3 is not a square), inverted by Fermat.
FCIRC_HD E inv(E a)
{
    const uint32_t nrm = sub1(red((uint64_t)a.re * a.re), red(3ull * red((uint64_t)a.im * a.im)));
    uint64_t e = P - 2;
    uint32_t r = 1, b = nrm;
    while (e) {
        if (e & 1) r = red((uint64_t)r * b);
        b = red((uint64_t)b * b);
        e >>= 1;
    }
    return E{red((uint64_t)a.re * r), red((uint64_t)(a.im ? P - a.im : 0u) * r)};
}

// The multiplicative group has order p^2 - 1 = 2^32 q with q = 2^30 - 1 odd.
constexpr int V = 32;
constexpr uint64_t Q = (1ull << 30) - 1;

// A generator of the 2-Sylow subgroup (order 2^32): g = (1 + sqrt 3) / sqrt 2,
// whose square is 2 + sqrt 3 (p = 7 mod 8, so sqrt 2 = 2^((p+1)/4) is in Z/pZ).
FCIRC_HD E sylow2_generator()
{
    uint64_t e = (P + 1) / 4;
    uint32_t r = 1, b = 2;
    while (e) {
        if (e & 1) r = red((uint64_t)r * b);
        b = red((uint64_t)b * b);
        e >>= 1;
    }
    return mul(E{1u, 1u}, inv(E{r, 0u}));
}

// A primitive 2^k-th root of unity (k <= 32): g^(2^(32-k)).
FCIRC_HD E root_of_unity(int k) { return pow(sylow2_generator(), (uint64_t)1 << (V - k)); }

// A 2^k-th root of f (r^(2^k) = f), k <= 30, or false if none exists.
// y = f^u with u = 2^-k mod q satisfies y^(2^k) = f z, z = f^(q m) in the
// 2-Sylow subgroup <g> for some m; a 2^k-th root of z^-1 there is
// g^(log / 2^k) when 2^k divides the discrete logarithm (found bit by bit).
inline bool root_2k(E f, int k, E &root)
{
    if (is_zero(f) || k < 0 || k > 30) return false;
    // u = 2^-k mod q: 2^30 = 1 (mod q), so 2^-k = 2^(30 - k)
    const uint64_t u = (uint64_t)1 << (30 - k);
    const E y = pow(f, u);
    const E yk = pow(y, (uint64_t)1 << k);
    const E z = mul(yk, inv(f));   // in the 2-Sylow subgroup
    const E zi = inv(z);
    // discrete log of zi to base g
    const E g = sylow2_generator(), gi = inv(g);
    const E minus_one{P - 1, 0u};
    uint64_t L = 0;
    E cur = zi;
    if (!eq(pow(cur, (uint64_t)1 << V), E{1u, 0u})) return false;
    for (int i = 0; i < V; ++i) {
        const E t = pow(cur, (uint64_t)1 << (V - 1 - i));
        if (!eq(t, E{1u, 0u})) {
            if (!eq(t, minus_one)) return false;
            L |= (uint64_t)1 << i;
            cur = mul(cur, pow(gi, (uint64_t)1 << i));
        }
    }
    if (L & (((uint64_t)1 << k) - 1)) return false;
    root = mul(y, pow(g, L >> k));
    return eq(pow(root, (uint64_t)1 << k), f);
}

}  // namespace gf
}  // namespace fcirc
