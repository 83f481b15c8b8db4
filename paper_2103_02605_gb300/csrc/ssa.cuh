// ssa.cuh -- arithmetic in the ring Z/(2^K + 1), K = 64 W (the ring of
// Schoenhage-Strassen multiplication, which the conclusion of the paper
// names as the place its algorithm could serve).  2 has order 2K there
// (2^K = -1), so every root of unity the recursion of Algorithm 1 needs is a
// power of two: each twiddle product is a shift and a subtraction, with no
// multiplication.  Only the leaf products multiply two elements.
//
// An element is SsaE<W>: W little-endian 64-bit words and a top word, value
// w + top 2^K in [0, 2^K] (top = 1 only for 2^K = -1).  A twiddle 2^e is
// SsaTw<W>{e}, 0 <= e < 2K.
#pragma once
#include <stdint.h>

namespace fcirc {

template <int W>
struct SsaE {
    uint64_t w[W];
    uint64_t top;
};

template <int W>
struct SsaTw {
    int e;
};

template <int W>
__device__ __forceinline__ SsaTw<W> ld_tw(const SsaTw<W> *p)
{
    return SsaTw<W>{__ldg(&p->e)};
}

// -2^e = 2^(e + K)
template <int W>
__device__ __forceinline__ SsaTw<W> cneg(SsaTw<W> t)
{
    constexpr int K = 64 * W;
    return SsaTw<W>{t.e >= K ? t.e - K : t.e + K};
}

// The value t = lo + hi 2^K, lo < 2^K, hi in [-3, 3], reduced into [0, 2^K]:
// first lo - hi as words and a signed top in {-1, 0, 1}, then one correction
// by 2^K + 1 (2^K = -1).
template <int W>
__device__ __forceinline__ SsaE<W> ssa_norm(const uint64_t *lo, int hi)
{
    SsaE<W> r;
    int ext = 0;
    if (hi >= 0) {
        uint64_t b = (uint64_t)hi;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const uint64_t v = lo[i];
            r.w[i] = v - b;
            b = v < b ? 1u : 0u;
        }
        ext = -(int)b;
    } else {
        uint64_t c = (uint64_t)(-hi);
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const uint64_t v = lo[i] + c;
            c = v < c ? 1u : 0u;
            r.w[i] = v;
        }
        ext = (int)c;
    }
    r.top = 0;
    if (ext < 0) {
        // t + 2^K + 1 = words + 1, in [2^K - 2, 2^K]
        uint64_t c = 1;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const uint64_t v = r.w[i] + c;
            c = v < c ? 1u : 0u;
            r.w[i] = v;
        }
        r.top = c;   // words wrapped to 0: the value is 2^K
    } else if (ext > 0) {
        // t = 2^K + words, words <= 2: 2^K itself, or words - 1
        bool zero = true;
#pragma unroll
        for (int i = 0; i < W; ++i) zero = zero && r.w[i] == 0;
        if (zero) {
            r.top = 1;
        } else {
            uint64_t b = 1;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const uint64_t v = r.w[i];
                r.w[i] = v - b;
                b = v < b ? 1u : 0u;
            }
        }
    }
    return r;
}

template <int W>
__device__ __forceinline__ SsaE<W> cadd(SsaE<W> a, SsaE<W> b)
{
    uint64_t s[W], c = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint64_t t = a.w[i] + c;
        const uint64_t c1 = t < c ? 1u : 0u;
        s[i] = t + b.w[i];
        c = c1 + (s[i] < t ? 1u : 0u);
    }
    return ssa_norm<W>(s, (int)(c + a.top + b.top));
}

template <int W>
__device__ __forceinline__ SsaE<W> csub(SsaE<W> a, SsaE<W> b)
{
    uint64_t d[W], br = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint64_t t = a.w[i] - br;
        const uint64_t b1 = a.w[i] < br ? 1u : 0u;
        d[i] = t - b.w[i];
        br = b1 + (t < b.w[i] ? 1u : 0u);
    }
    // a - b = d + (a.top - b.top - br) 2^K
    return ssa_norm<W>(d, (int)a.top - (int)b.top - (int)br);
}

template <int W>
__device__ __forceinline__ SsaE<W> ssa_zero()
{
    SsaE<W> z;
#pragma unroll
    for (int i = 0; i < W; ++i) z.w[i] = 0;
    z.top = 0;
    return z;
}

template <int W>
__device__ __forceinline__ SsaE<W> cneg(SsaE<W> a)
{
    return csub<W>(ssa_zero<W>(), a);
}

// x 2^e for 0 <= e < K, x < 2^K: the 2W-word shift split at bit K into
// lo - hi (2^K = -1).
template <int W>
__device__ __forceinline__ SsaE<W> ssa_shift_low(const SsaE<W> &x, int e)
{
    const int q = e >> 6, s = e & 63;
    uint64_t sh[2 * W];
#pragma unroll
    for (int j = 0; j < 2 * W; ++j) sh[j] = 0;
#pragma unroll
    for (int qq = 0; qq < W; ++qq) {
        if (q == qq) {
#pragma unroll
            for (int i = 0; i < W; ++i) {
                sh[i + qq] |= s ? (x.w[i] << s) : x.w[i];
                if (s && i + qq + 1 < 2 * W) sh[i + qq + 1] |= x.w[i] >> (64 - s);
            }
        }
    }
    SsaE<W> lo, hi;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        lo.w[i] = sh[i];
        hi.w[i] = sh[W + i];
    }
    lo.top = hi.top = 0;
    return csub<W>(lo, hi);
}

// twiddle product x 2^e, 0 <= e < 2K
template <int W>
__device__ __forceinline__ SsaE<W> cmul(SsaTw<W> t, SsaE<W> x)
{
    constexpr int K = 64 * W;
    const bool negate = t.e >= K;
    const int e = negate ? t.e - K : t.e;
    SsaE<W> r;
    if (x.top) {
        // 2^K 2^e = -2^e
        SsaE<W> p = ssa_zero<W>();
#pragma unroll
        for (int i = 0; i < W; ++i) p.w[i] = (e >> 6) == i ? (uint64_t)1 << (e & 63) : 0u;
        r = cneg<W>(p);
    } else {
        r = ssa_shift_low<W>(x, e);
    }
    return negate ? cneg<W>(r) : r;
}

template <int W>
__device__ __forceinline__ SsaE<W> cmul(SsaE<W> x, SsaTw<W> t)
{
    return cmul<W>(t, x);
}

// general product (the leaves): the 2W-word schoolbook product split at bit
// K into lo - hi; an operand 2^K = -1 negates the other
template <int W>
__device__ __forceinline__ SsaE<W> cmul(SsaE<W> a, SsaE<W> b)
{
    if (a.top) return cneg<W>(b);
    if (b.top) return cneg<W>(a);
    uint64_t p[2 * W];
#pragma unroll
    for (int j = 0; j < 2 * W; ++j) p[j] = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        uint64_t carry = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const uint64_t lo = a.w[i] * b.w[j], hi = __umul64hi(a.w[i], b.w[j]);
            uint64_t t = p[i + j] + lo;
            uint64_t c = t < lo ? 1u : 0u;
            t += carry;
            c += t < carry ? 1u : 0u;
            p[i + j] = t;
            carry = hi + c;
        }
        p[i + W] = carry;
    }
    SsaE<W> lo, hi;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        lo.w[i] = p[i];
        hi.w[i] = p[W + i];
    }
    lo.top = hi.top = 0;
    return csub<W>(lo, hi);
}

}  // namespace fcirc
