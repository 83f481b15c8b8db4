// modarith.cuh -- 32-bit modular arithmetic for primes p < 2^30, shared by
// the host plan builder and the sm_103a kernels.
//
// Representation: residues are uint32 in a "lazy" range [0, 2p) or [0, 4p)
// (4p < 2^32 because p < 2^30) and made canonical only where results leave
// the library.
//
//  * Multiplication by a known constant w uses Shoup's precomputed quotient
//    w' = floor(w * 2^32 / p) (V. Shoup, NTL; D. Harvey, "Faster arithmetic
//    for number-theoretic transforms", J. Symb. Comp. 2014): for any 32-bit
//    x, x*w - umulhi(x, w')*p lies in [0, 2p).
//  * Multiplication of two variable residues uses Montgomery reduction
//    (P. L. Montgomery, Math. Comp. 1985) with R = 2^32: for x*y < p*R the
//    result x*y*R^-1 mod p lies in (0, 2p).
//  * The butterflies are those of the paper's Algorithm 1 (Section 2):
//      row vector of A_M1 / A_M2:   a_lo + s a_hi,  a_lo - s a_hi
//      vector side:                 s b_lo + b_hi,  s b_lo - b_hi
//      recombination:               (M1 + M2) / (2s),  (M1 + M2)/2 - M2
//    with the factor 1/2 of every recombination level deferred to the leaf
//    product (one multiplication by 2^-L there instead of one per level).
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define FCIRC_HD __host__ __device__ __forceinline__
#else
#define FCIRC_HD inline
#endif

namespace fcirc {

FCIRC_HD uint32_t umulhi32(uint32_t a, uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// Shoup product: x * w mod p in [0, 2p) for any 32-bit x, with w < p and
// wp = floor(w * 2^32 / p).
FCIRC_HD uint32_t shoup_mul(uint32_t x, uint32_t w, uint32_t wp, uint32_t p)
{
    uint32_t q = umulhi32(x, wp);
    return x * w - q * p;
}

// x in [0, 2m) -> [0, m).  Two instruction forms of the same result, chosen
// per kernel by measurement: the select x >= m ? x - m : x, and
// min(x, x - m) in unsigned arithmetic (x - m wraps to a large value when
// x < m), which sm_103a issues as one add-and-min.
FCIRC_HD uint32_t reduce_sel(uint32_t x, uint32_t m) { return x >= m ? x - m : x; }

FCIRC_HD uint32_t reduce_min(uint32_t x, uint32_t m)
{
#if defined(__CUDA_ARCH__)
    return umin(x, x - m);
#else
    return x >= m ? x - m : x;
#endif
}

template <bool UM = true>
FCIRC_HD uint32_t reduce_once(uint32_t x, uint32_t m)
{
    return UM ? reduce_min(x, m) : reduce_sel(x, m);
}

// [0, 4p) -> [0, p)
FCIRC_HD uint32_t canon4(uint32_t x, uint32_t p, uint32_t p2)
{
    return reduce_once(reduce_once(x, p2), p);
}

// Montgomery reduction of a 64-bit T < p 2^32: T 2^-32 mod p in (0, 2p).
// pinv = p^-1 mod 2^32; m p agrees with T in the low word, so the low words
// cancel exactly and only the high words are subtracted.
FCIRC_HD uint32_t redc(uint64_t T, uint32_t p, uint32_t pinv)
{
    const uint32_t m = (uint32_t)T * pinv;
    return (uint32_t)(T >> 32) - umulhi32(m, p) + p;
}

// Montgomery product x*y*2^-32 mod p in (0, 2p), valid when x*y < p*2^32
// (e.g. x, y < 2p).  pinv = p^-1 mod 2^32.
FCIRC_HD uint32_t mont_mul(uint32_t x, uint32_t y, uint32_t p, uint32_t pinv)
{
    uint32_t lo = x * y;
    uint32_t hi = umulhi32(x, y);
    uint32_t m = lo * pinv;                 // m*p = x*y (mod 2^32)
    return hi - umulhi32(m, p) + p;         // (x*y - m*p)/2^32 + p
}

// Twiddle generated from a universal root-of-unity entry u (< p) and a
// per-block factor sigma given with its 64-bit quotient
// floor(sigma * 2^64 / p) = (sp << 32) | spp:
//   w  = u * sigma mod p (canonical),   wp = floor(w * 2^32 / p).
// Derivation: w * 2^32 / p = u*sp - q*2^32 + (u*spp + u*eps) / 2^32 with
// q = floor(u*sigma/p) and 0 <= eps < 1, so wp is lo32(u*sp) + umulhi(u, spp)
// or one more; the remainder w*2^32 - wp*p (mod 2^32) tells which.
struct Tw {
    uint32_t w, wp;
};

FCIRC_HD Tw twiddle_from(uint32_t u, uint32_t sigma, uint32_t sp, uint32_t spp,
                         uint32_t p)
{
    uint32_t q = umulhi32(u, sp);
    uint32_t w = u * sigma - q * p;
    w = reduce_once(w, p);
    uint32_t cand = u * sp + umulhi32(u, spp);
    uint32_t r = 0u - cand * p;
    cand += (r >= p) ? 1u : 0u;
    Tw t;
    t.w = w;
    t.wp = cand;
    return t;
}

// Negated twiddle p - w with its quotient: floor((p-w) 2^32/p) = 2^32-1-wp
// for 0 < w < p.
FCIRC_HD Tw tw_neg(Tw t, uint32_t p)
{
    Tw r;
    r.w = t.w ? p - t.w : 0u;
    r.wp = t.w ? ~t.wp : 0u;
    return r;
}

// -- butterflies of Algorithm 1 ---------------------------------------------
// UM selects the form of the conditional subtraction (see reduce_once).
// Row-vector side (A_M1 / A_M2 rows):  (lo, hi) <- (lo + s hi, lo - s hi)
// in/out range [0, 4p).
template <bool UM = true>
FCIRC_HD void bfly_row(uint32_t &lo, uint32_t &hi, Tw s, uint32_t p, uint32_t p2)
{
    uint32_t t = shoup_mul(hi, s.w, s.wp, p);      // [0, 2p)
    uint32_t l = reduce_once<UM>(lo, p2);          // [0, 2p)
    lo = l + t;                                    // [0, 4p)
    hi = l - t + p2;                               // (0, 4p)
}

// Vector side: (lo, hi) <- (s lo + hi, s lo - hi); in/out range [0, 4p).
template <bool UM = true>
FCIRC_HD void bfly_vec(uint32_t &lo, uint32_t &hi, Tw s, uint32_t p, uint32_t p2)
{
    uint32_t t = shoup_mul(lo, s.w, s.wp, p);      // [0, 2p)
    uint32_t h = reduce_once<UM>(hi, p2);          // [0, 2p)
    lo = t + h;
    hi = t - h + p2;
}

// Recombination with the 1/2 deferred: (M1, M2) <- ((M1 + M2) / s, M1 - M2),
// si = s^-1; in/out range [0, 2p).
FCIRC_HD void bfly_rec(uint32_t &m1, uint32_t &m2, Tw si, uint32_t p, uint32_t p2)
{
    uint32_t s = m1 + m2;                          // [0, 4p)
    uint32_t d = m1 - m2 + p2;                     // (0, 4p)
    m1 = shoup_mul(s, si.w, si.wp, p);             // [0, 2p)
    m2 = reduce_once(d, p2);                       // [0, 2p)
}

// Row vector shifted by one place (a'_k = a_(k-1), indices mod n; at f = 1
// the product's entries move up by one, c'_i = c_(i+1)).  The shift is
// z a(z), so a 2x2 leaf's row (x0, x1) = a mod (z^2 - phi) becomes
// (phi x1, x0), and the leaf gives c'_0 = c1 and c'_1 = phi c0, with (c0, c1)
// what leaf2 gives for the unshifted row.  The factor phi = +-s costs no
// multiplication when it is left to the first recombination level: the
// position-1 entries of sibling leaves, s c0_A and -s c0_B, recombine as
// (c0_A - c0_B, s (c0_A + c0_B)).  bfly_rec_shift is that butterfly; it
// takes the forward twiddle s.  In (0, 2p), out [0, 2p).
FCIRC_HD void bfly_rec_shift(uint32_t &m1, uint32_t &m2, Tw s, uint32_t p, uint32_t p2)
{
    const uint32_t sum = m1 + m2;                  // (0, 4p)
    const uint32_t d = m1 - m2 + p2;               // (0, 4p)
    m1 = reduce_once(d, p2);                       // [0, 2p)
    m2 = shoup_mul(sum, s.w, s.wp, p);             // [0, 2p)
}

// 2x2 leaf: the phi-circulant [[a0, a1], [phi a1, a0]] times (y0, y1) --
// Definition 2 at n = 2, which is what Algorithm 1 gives for 1x1 blocks.
// Each output is one 64-bit sum of two products of canonical residues
// (below 2 p^2 < p 2^32) reduced once by Montgomery; the factor 2^32 2^-L this
// leaves over (2^-L being the deferred halvings of the recombination) is put
// on the row-vector input when it is first loaded.  a*, y* in [0, 4p);
// outputs in (0, 2p).
FCIRC_HD void leaf2(uint32_t &a0, uint32_t &a1, uint32_t y0, uint32_t y1, Tw phi, uint32_t p,
                    uint32_t p2, uint32_t pinv)
{
    const uint32_t x0 = canon4(a0, p, p2), x1 = canon4(a1, p, p2);
    const uint32_t z0 = canon4(y0, p, p2), z1 = canon4(y1, p, p2);
    const uint32_t x1f = reduce_once(shoup_mul(x1, phi.w, phi.wp, p), p);
    const uint64_t t0 = (uint64_t)x0 * z0 + (uint64_t)x1 * z1;
    const uint64_t t1 = (uint64_t)x1f * z0 + (uint64_t)x0 * z1;
    a0 = redc(t0, p, pinv);
    a1 = redc(t1, p, pinv);
}

}  // namespace fcirc
