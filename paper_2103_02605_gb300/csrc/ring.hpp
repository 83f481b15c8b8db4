// ring.hpp -- host-side arithmetic of Z/pZ for the plan builder: primality,
// a generator of the unit group, 2-adic valuation, 2^k-th roots and the
// Shoup quotients the kernels consume.
//
// Theorem 1 (Section 2) asks for an n-th root of f, an n-th root of unity,
// 2^-1 and f^-1 in the ring; for Z/pZ with p prime the roots of unity of
// order 2^k exist iff 2^k | p - 1, and f has a 2^k-th root iff
// f^((p-1)/gcd(2^k, p-1)) = 1.
#pragma once
#include <stdint.h>
#include <vector>

#include "modarith.cuh"   // FCIRC_HD

namespace fcirc {
namespace host {

FCIRC_HD uint64_t umulhi64(uint64_t a, uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Products mod p < 2^31 by Barrett reduction with m = floor((2^64 - 1) / p):
// for x = a b < p^2, q = floor(x m / 2^64) is floor(x / p) or one less
// (x m / 2^64 > x / p - x (1 + 1/p) / 2^64 and x < 2^62), so x - q p lies in
// [0, 2p) and one conditional subtraction finishes.  The reciprocal costs one
// 64-bit division, once; each product is a multiply, a high multiply and a
// subtraction -- on the GPU, much cheaper than a 64-bit remainder.
struct ModP {
    uint32_t p;
    uint64_t m;
    FCIRC_HD explicit ModP(uint32_t p_) : p(p_), m(~(uint64_t)0 / p_) {}
    FCIRC_HD uint32_t mul(uint32_t a, uint32_t b) const
    {
        const uint64_t x = (uint64_t)a * b;
        const uint64_t r = x - umulhi64(x, m) * p;
        return (uint32_t)(r >= p ? r - p : r);
    }
    FCIRC_HD uint32_t pow(uint32_t b, uint64_t e) const
    {
        uint32_t r = 1 % p, x = b % p;
        while (e) {
            if (e & 1) r = mul(r, x);
            x = mul(x, x);
            e >>= 1;
        }
        return r;
    }
    FCIRC_HD uint32_t inv(uint32_t a) const { return pow(a, (uint64_t)p - 2); }   // p prime, a != 0
    // floor(x / p) for x < 2^62: the same estimate, one correction
    FCIRC_HD uint64_t div(uint64_t x) const
    {
        uint64_t q = umulhi64(x, m);
        if (x - q * p >= p) ++q;
        return q;
    }
    // Shoup quotients: floor(w 2^32 / p), and floor(w 2^64 / p) as (hi, lo)
    // (w < p < 2^30 keeps every dividend below 2^62)
    FCIRC_HD uint32_t quot32(uint32_t w) const { return (uint32_t)div((uint64_t)w << 32); }
    FCIRC_HD void quot64(uint32_t w, uint32_t &hi, uint32_t &lo) const
    {
        const uint64_t t = (uint64_t)w << 32;
        const uint64_t q = div(t);
        hi = (uint32_t)q;
        lo = (uint32_t)div((t - q * p) << 32);
    }
};

FCIRC_HD uint32_t mulmod(uint32_t a, uint32_t b, uint32_t p)
{
    return (uint32_t)((uint64_t)a * b % p);
}

FCIRC_HD uint32_t powmod(uint32_t b, uint64_t e, uint32_t p)
{
    uint64_t r = 1 % p, x = b % p;
    while (e) {
        if (e & 1) r = r * x % p;
        x = x * x % p;
        e >>= 1;
    }
    return (uint32_t)r;
}

FCIRC_HD uint32_t invmod(uint32_t a, uint32_t p)  // p prime, a != 0 mod p
{
    return powmod(a, (uint64_t)p - 2, p);
}

// Deterministic Miller-Rabin for 32-bit integers (bases 2, 7, 61).
inline bool is_prime(uint32_t n)
{
    if (n < 2) return false;
    for (uint32_t sp : {2u, 3u, 5u, 7u, 11u, 13u, 61u})
        if (n % sp == 0) return n == sp;
    uint32_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; ++s; }
    for (uint32_t a : {2u, 7u, 61u}) {
        uint32_t x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; ++r) {
            x = mulmod(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

inline int two_adic(uint32_t p)  // v with 2^v || p - 1
{
    uint32_t q = p - 1;
    int v = 0;
    while ((q & 1) == 0) { q >>= 1; ++v; }
    return v;
}

// Smallest generator of (Z/pZ)^*: g^((p-1)/r) != 1 for every prime r | p-1.
inline uint32_t generator(uint32_t p)
{
    std::vector<uint32_t> fac;
    uint32_t m = p - 1;
    for (uint32_t r = 2; (uint64_t)r * r <= m; ++r)
        if (m % r == 0) {
            fac.push_back(r);
            while (m % r == 0) m /= r;
        }
    if (m > 1) fac.push_back(m);
    for (uint32_t g = 2; g < p; ++g) {
        bool ok = true;
        for (uint32_t r : fac)
            if (powmod(g, (p - 1) / r, p) == 1) { ok = false; break; }
        if (ok) return g;
    }
    return 0;
}

// Omega: the fixed primitive 2^v-th root of unity g^((p-1)/2^v) every plan
// of this prime derives its roots of unity from (psi_m = Omega^(2^v/m)).
inline uint32_t omega(uint32_t p)
{
    int v = two_adic(p);
    return powmod(generator(p), (uint64_t)(p - 1) >> v, p);
}

// Discrete log of w in the cyclic group <Om> of order 2^v (Pohlig-Hellman,
// one bit at a time).  Returns false if w is not in the group.
FCIRC_HD bool dlog_2group(uint32_t w, uint32_t Om, int v, const ModP &M, uint64_t &out)
{
    if (M.pow(w, (uint64_t)1 << v) != 1) return false;
    uint32_t step = M.inv(Om);   // Om^-(2^i) at bit i
    uint64_t L = 0;
    uint32_t cur = w;  // w * Om^-L
    for (int i = 0; i < v; ++i) {
        // cur has order dividing 2^(v-i); test bit i
        uint32_t t = cur;
        for (int k = 0; k < v - 1 - i; ++k) t = M.mul(t, t);
        if (t != 1) {
            L |= (uint64_t)1 << i;
            cur = M.mul(cur, step);
        }
        step = M.mul(step, step);
    }
    out = L;
    return true;
}

FCIRC_HD bool dlog_2group(uint32_t w, uint32_t Om, int v, uint32_t p, uint64_t &out)
{
    return dlog_2group(w, Om, v, ModP(p), out);
}

// A 2^k-th root r of f mod p (r^(2^k) = f), or false if none exists.
// Write p - 1 = q 2^v with q odd.  y = f^u with u = 2^-k mod q gives
// y^(2^k) = f * z for z = (f^q)^m in the 2-Sylow subgroup <Omega>; a 2^k-th
// root of z^-1 there is Omega^(log/2^k) when 2^k divides the discrete log.
// Same, with Omega and v supplied (usable on the device).
FCIRC_HD bool nth_root_2k_om(uint32_t f, int k, const ModP &M, uint32_t Om, int v, uint32_t &root)
{
    const uint32_t p = M.p;
    f %= p;
    if (f == 0) return false;
    if (k == 0) { root = f; return true; }
    if (f == 1) { root = 1; return true; }
    uint64_t q = (uint64_t)(p - 1) >> v;
    // u = (2^k)^-1 mod q  (q odd; q == 1 -> u = 0)
    uint64_t u = 0;
    if (q > 1) {
        // the inverse of 2 mod q is (q+1)/2, so (2^k)^-1 = ((q+1)/2)^k mod q
        uint64_t t = 1, h = (q + 1) / 2;
        for (int i = 0; i < k; ++i) t = t * h % q;
        u = t;
    }
    uint32_t y = M.pow(f, u);
    // z = y^(2^k) / f lies in <Omega>
    if (k > 62) return false;
    uint32_t y2k = y;
    for (int i = 0; i < k; ++i) y2k = M.mul(y2k, y2k);
    uint32_t z = M.mul(y2k, M.inv(f));
    uint32_t zi = M.inv(z);
    uint64_t L;
    if (!dlog_2group(zi, Om, v, M, L)) return false;
    uint32_t w;
    if (k <= v) {
        if (L & (((uint64_t)1 << k) - 1)) return false;
        w = M.pow(Om, L >> k);
    } else {
        // x -> x^(2^k) kills <Omega>; a root exists only if z = 1
        if (L != 0) return false;
        w = 1;
    }
    root = M.mul(y, w);
    uint32_t chk = root;
    for (int i = 0; i < k; ++i) chk = M.mul(chk, chk);
    if (chk != f) return false;
    return true;
}

FCIRC_HD bool nth_root_2k_om(uint32_t f, int k, uint32_t p, uint32_t Om, int v, uint32_t &root)
{
    return nth_root_2k_om(f, k, ModP(p), Om, v, root);
}

inline bool nth_root_2k(uint32_t f, int k, uint32_t p, uint32_t &root)
{
    return nth_root_2k_om(f, k, p, omega(p), two_adic(p), root);
}

FCIRC_HD uint32_t shoup_quot(uint32_t w, uint32_t p)  // floor(w 2^32 / p)
{
    return (uint32_t)(((uint64_t)w << 32) / p);
}

// floor(w 2^64 / p) = (hi << 32) | lo for w < p, in two 64-bit divisions:
// w 2^32 = hi p + r, then lo = floor(r 2^32 / p).
FCIRC_HD void shoup_quot64(uint32_t w, uint32_t p, uint32_t &hi, uint32_t &lo)
{
    const uint64_t t = (uint64_t)w << 32;
    const uint64_t q = t / p;
    const uint64_t r = t - q * p;
    hi = (uint32_t)q;
    lo = (uint32_t)((r << 32) / p);
}

FCIRC_HD uint32_t bitrev(uint64_t j, int bits)
{
    uint64_t r = 0;
    for (int i = 0; i < bits; ++i)
        if (j >> i & 1) r |= (uint64_t)1 << (bits - 1 - i);
    return (uint32_t)r;
}

}  // namespace host
}  // namespace fcirc
