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

// The value t = lo + hi 2^K, lo < 2^K, hi in [-3, 3], reduced into [0, 2^K],
// without data-dependent branches (the lanes of a warp hold different
// elements, so a branch here would split the warp).  2^K = -1, so
// t = lo - hi: first r = lo - hi as W words and a signed top e in
// {-1, 0, 1}, so t = r - e (mod 2^K + 1); then r - e as W words again, whose
// carry out decides the one case that lands on 2^K itself.
template <int W>
__device__ __forceinline__ SsaE<W> ssa_norm(const uint64_t *lo, int hi)
{
    // r = lo + c with c = -hi sign-extended over W words
    const int64_t c = -(int64_t)hi;
    const uint64_t ext = c < 0 ? ~0ull : 0ull;
    uint64_t r[W], carry = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint64_t add = i == 0 ? (uint64_t)c : ext;
        const uint64_t t = lo[i] + add;
        const uint64_t c1 = t < add ? 1u : 0u;
        r[i] = t + carry;
        carry = c1 + (r[i] < t ? 1u : 0u);
    }
    // the W-word sum with the sign extension: top word e = carry + ext
    const int e = (int)(carry & 1u) - (c < 0 ? 1 : 0);
    // value = r - e; d = -e in {-1, 0, 1} added the same way
    const int64_t d = -(int64_t)e;
    const uint64_t dext = d < 0 ? ~0ull : 0ull;
    SsaE<W> o;
    carry = 0;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint64_t add = i == 0 ? (uint64_t)d : dext;
        const uint64_t t = r[i] + add;
        const uint64_t c1 = t < add ? 1u : 0u;
        o.w[i] = t + carry;
        carry = c1 + (o.w[i] < t ? 1u : 0u);
    }
    carry &= 1u;
    // d = +1: a carry out means r was 2^K - 1 and the words wrapped to 0 --
    //         the value 2^K;
    // d = -1: no carry out means r was 0 (a borrow) -- again 2^K, words 0.
    const bool up = d > 0 && carry;
    const bool down = d < 0 && !carry;
#pragma unroll
    for (int i = 0; i < W; ++i) o.w[i] = down ? 0ull : o.w[i];
    o.top = (up || down) ? 1u : 0u;
    return o;
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

// v >> (64 - s) for 0 <= s < 64, 0 when s = 0, without a branch
__device__ __forceinline__ uint64_t ssa_rsh_c(uint64_t v, int s) { return (v >> 1) >> (63 - s); }

// twiddle product x 2^e, 0 <= e < 2K.  With e = e' + K [e >= K] (2^K = -1),
// x 2^e' is the 2W-word shift of x split at bit K into lo - hi, and the
// factor -1 swaps the operands of that subtraction.  The element 2^K
// (top = 1, words 0) contributes 2^(K + e'): the bit e' of hi.  One
// subtraction, no branch.
template <int W>
__device__ __forceinline__ SsaE<W> cmul(SsaTw<W> t, SsaE<W> x)
{
    constexpr int K = 64 * W;
    const bool negate = t.e >= K;
    const int e = negate ? t.e - K : t.e;
    const int q = e >> 6, s = e & 63;
    uint64_t sh[2 * W];
#pragma unroll
    for (int j = 0; j < 2 * W; ++j) sh[j] = 0;
#pragma unroll
    for (int qq = 0; qq < W; ++qq) {
        const uint64_t m = q == qq ? ~0ull : 0ull;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            sh[i + qq] |= (x.w[i] << s) & m;
            if (i + qq + 1 < 2 * W) sh[i + qq + 1] |= ssa_rsh_c(x.w[i], s) & m;
        }
    }
    SsaE<W> lo, hi;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        lo.w[i] = sh[i];
        hi.w[i] = sh[W + i] | ((x.top && q == i) ? (1ull << s) : 0ull);
    }
    lo.top = hi.top = 0;
    SsaE<W> u, v;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        u.w[i] = negate ? hi.w[i] : lo.w[i];
        v.w[i] = negate ? lo.w[i] : hi.w[i];
    }
    u.top = v.top = 0;
    return csub<W>(u, v);
}

template <int W>
__device__ __forceinline__ SsaE<W> cmul(SsaE<W> x, SsaTw<W> t)
{
    return cmul<W>(t, x);
}

// general product (the leaves): the 2W-word schoolbook product of the words
// split at bit K into lo - hi, then the element 2^K = -1 handled by one more
// subtraction, without a branch: a.top = 1 (a.w = 0) makes the word product
// 0 and the result -b; b.top = 1 alone gives -a; both give -(2^K) = 1.
template <int W>
__device__ __forceinline__ SsaE<W> cmul(SsaE<W> a, SsaE<W> b)
{
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
    const SsaE<W> r = csub<W>(lo, hi);
    // the top terms: -b when a = 2^K, -a when b = 2^K (r is 0 then)
    SsaE<W> m;
#pragma unroll
    for (int i = 0; i < W; ++i) m.w[i] = a.top ? b.w[i] : (b.top ? a.w[i] : 0ull);
    m.top = a.top ? b.top : 0u;
    return csub<W>(r, m);
}

}  // namespace fcirc
