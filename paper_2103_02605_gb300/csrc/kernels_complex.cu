// kernels_complex.cu -- the f-circulant product over complex numbers in
// FP32 (the closing remark of Section 3.1: real or complex coefficients need
// complex roots), forward and hand-written backward, batched.
//
// Same recursion as the modular path (Algorithm 1): row-vector butterflies
// lo +- s hi, vector butterflies s lo +- hi, 2x2 leaves, recombination
// ((M1 + M2) s^-1, M1 - M2) with the halvings deferred to one exact scaling
// by 2^-L at the end.  Twiddles s_{l,j} = |f|^(1/2^(l+1)) exp(i (arg f +
// 2 pi brv_l(j)) / 2^(l+1)) are formed in FP64 on the host and rounded to
// FP32.
//
// Backward, for L = Re <g, A x> (PyTorch's convention for complex tensors):
//   dL/dx = A^H g = RowCirc_{1/conj(f)}(beta) g,
//           beta = (conj a_0, conj(f) conj a_{n-1}, ..., conj(f) conj a_1),
//   dL/da = RowCirc_{conj(f)}(g) conj(x),
// two more f'-circulant products through the same recursion, computed
// together in one CTA per instance.
//
// Layout: n = 2^M complex numbers per instance, interleaved (re, im) float,
// instances back to back.  A thread owns 8 numbers of a side; the CTA runs
// register stages of up to 3 levels with shared-memory exchanges, the last
// stage on 8 contiguous numbers (bottom two levels, four 2x2 leaves, and
// the first two recombination levels).
#include <cmath>
#include <type_traits>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.hpp"
#include "kernels_complex.hpp"
#include "prof.hpp"
#include "gfp2.hpp"
#include "ssa.cuh"
#include "ring.hpp"

namespace fcirc {

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// Sums and differences as single packed two-lane FP32 instructions (the
// {re, im} pair is one 64-bit register pair); a - b as fma(b, -1, a), the
// exact difference rounded once, as the scalar subtraction rounds it.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float2 ld_tw(const float2 *p) { return __ldg(p); }
__device__ __forceinline__ uint2 ld_tw(const uint2 *p) { return __ldg(p); }

// The same four operations in GF(p^2) = Z/pZ[sqrt 3], p = 2^31 - 1 (the
// paper's own field, Section 3.1), an element (x, y) = x + y sqrt 3.
__device__ __forceinline__ uint2 gf2(gf::E e) { return make_uint2(e.re, e.im); }
__device__ __forceinline__ gf::E gfe(uint2 v) { return gf::E{v.x, v.y}; }
__device__ __forceinline__ uint2 cmul(uint2 a, uint2 b) { return gf2(gf::mul(gfe(a), gfe(b))); }
__device__ __forceinline__ uint2 cadd(uint2 a, uint2 b) { return gf2(gf::add(gfe(a), gfe(b))); }
__device__ __forceinline__ uint2 csub(uint2 a, uint2 b) { return gf2(gf::sub(gfe(a), gfe(b))); }
__device__ __forceinline__ uint2 cneg(uint2 a) { return gf2(gf::neg(gfe(a))); }

template <int M>
struct CShape {
    static constexpr int N = 1 << M;
    static constexpr int L = M - 1;           // halving levels; 2x2 leaves below
    static constexpr int NTI = N / 8;         // threads per instance
    static constexpr int CT = NTI < 128 ? 128 : NTI;   // threads per CTA
    static constexpr int IPC = CT / NTI;      // instances per CTA
    static constexpr int P = L - 2;           // levels before the last stage
    static constexpr int NST = (P + 2) / 3;   // stages of up to 3 levels, remainder first
    static constexpr int nl(int s) { return s == 0 ? P - 3 * (NST - 1) : 3; }
    static constexpr int d0(int s) { return s == 0 ? 0 : (P - 3 * (NST - 1)) + 3 * (s - 1); }
};

// One product's data in shared memory: row-vector side R and vector side X.
// T: the element type -- float2 (complex FP32), uint2 (GF(p^2), gfp2.hpp)
// or SsaE<W> (Z/(2^K + 1), ssa.cuh); TW: the twiddle type (T itself, or a
// shift amount for Z/(2^K + 1)).  The arithmetic comes from the cmul /
// cadd / csub / cneg overloads and ld_tw.
// Shared-memory position of element e of a side.  For complex FP32 the
// low four bits of e are XORed with bits 4-6 of e, and bit 3 also with bit
// 6: a bijection inside every 16-element block that makes each half-warp's
// 64-bit accesses fall in 16 distinct bank pairs in every pattern of the
// kernels -- the loads and stores e = t + (n/8) k, the register stages, and
// the last stage's 8 contiguous numbers per thread -- for n >= 128 (checked
// on the CPU for n = 2^3 .. 2^12).  Only the complex FP32 kernels, which are
// bound by shared-memory bandwidth, use it: the GF(p^2) and Z/(2^K + 1)
// kernels are bound by their ALU work and keep e.
template <class T>
__host__ __device__ __forceinline__ int cpos(int e)
{
    if constexpr (std::is_same<T, float2>::value)
        return e ^ (((e >> 4) & 7) | (((e >> 6) & 1) << 3));
    else
        return e;
}

template <class T, class TW = T>
struct SideT {
    T *R, *X;
    const TW *tw, *itw;   // heap-indexed twiddles and inverses, [N/2]
    __device__ __forceinline__ T &ra(int e) const { return R[cpos<T>(e)]; }
    __device__ __forceinline__ T &xa(int e) const { return X[cpos<T>(e)]; }
};
using Side = SideT<float2>;

// forward stage S (levels d0 .. d0+nl-1) on both sides
template <int M, int S, class T, class TW>
__device__ __forceinline__ void cfwd_stage(SideT<T, TW> &sd, int t)
{
    using Sh = CShape<M>;
    constexpr int NL = Sh::nl(S), D0 = Sh::d0(S), G = 8 >> NL, MM = 1 << NL;
    constexpr int LST = M - D0 - NL, LRB = M - D0;
#pragma unroll
    for (int h = 0; h < G; ++h) {
        const int gg = t + Sh::NTI * h;
        const int blk = gg >> LST, off = gg & ((1 << LST) - 1);
        const int e0 = (blk << LRB) + off;
        T r[MM], x[MM];
#pragma unroll
        for (int i = 0; i < MM; ++i) {
            r[i] = sd.ra(e0 + (i << LST));
            x[i] = sd.xa(e0 + (i << LST));
        }
#pragma unroll
        for (int d = 0; d < NL; ++d) {
            const int hh = MM >> (d + 1);
#pragma unroll
            for (int j = 0; j < (1 << d); ++j) {
                const TW s = ld_tw(&sd.tw[(1 << (D0 + d)) + (blk << d) + j]);
#pragma unroll
                for (int i = 0; i < hh; ++i) {
                    const int lo = (j << (NL - d)) + i, hi = lo + hh;
                    const T tr = cmul(s, r[hi]);
                    const T tx = cmul(s, x[lo]);
                    r[hi] = csub(r[lo], tr);
                    r[lo] = cadd(r[lo], tr);
                    const T xh = x[hi];
                    x[hi] = csub(tx, xh);
                    x[lo] = cadd(tx, xh);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < MM; ++i) {
            sd.ra(e0 + (i << LST)) = r[i];
            sd.xa(e0 + (i << LST)) = x[i];
        }
    }
}

// recombination stage S (levels d0+nl-1 .. d0), result in R
template <int M, int S, class T, class TW>
__device__ __forceinline__ void crec_stage(SideT<T, TW> &sd, int t)
{
    using Sh = CShape<M>;
    constexpr int NL = Sh::nl(S), D0 = Sh::d0(S), G = 8 >> NL, MM = 1 << NL;
    constexpr int LST = M - D0 - NL, LRB = M - D0;
#pragma unroll
    for (int h = 0; h < G; ++h) {
        const int gg = t + Sh::NTI * h;
        const int blk = gg >> LST, off = gg & ((1 << LST) - 1);
        const int e0 = (blk << LRB) + off;
        T r[MM];
#pragma unroll
        for (int i = 0; i < MM; ++i) r[i] = sd.ra(e0 + (i << LST));
#pragma unroll
        for (int d = NL - 1; d >= 0; --d) {
            const int hh = MM >> (d + 1);
#pragma unroll
            for (int j = 0; j < (1 << d); ++j) {
                const TW si = ld_tw(&sd.itw[(1 << (D0 + d)) + (blk << d) + j]);
#pragma unroll
                for (int i = 0; i < hh; ++i) {
                    const int lo = (j << (NL - d)) + i, hi = lo + hh;
                    const T sum = cadd(r[lo], r[hi]);
                    r[hi] = csub(r[lo], r[hi]);
                    r[lo] = cmul(sum, si);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < MM; ++i) sd.ra(e0 + (i << LST)) = r[i];
    }
}

// last stage: 8 contiguous numbers at 8t: levels L-2, L-1, four 2x2
// leaves, recombination L-1, L-2; result in R
template <int M, class T, class TW>
__device__ __forceinline__ void cleaf_stage(SideT<T, TW> &sd, int t)
{
    constexpr int L = M - 1;
    T r[8], x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        r[i] = sd.ra(8 * t + i);
        x[i] = sd.xa(8 * t + i);
    }
    const TW s0 = ld_tw(&sd.tw[(1 << (L - 2)) + t]);
    const TW s1[2] = {ld_tw(&sd.tw[(1 << (L - 1)) + 2 * t]), ld_tw(&sd.tw[(1 << (L - 1)) + 2 * t + 1])};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const T tr = cmul(s0, r[i + 4]), tx = cmul(s0, x[i]);
        r[i + 4] = csub(r[i], tr);
        r[i] = cadd(r[i], tr);
        const T xh = x[i + 4];
        x[i + 4] = csub(tx, xh);
        x[i] = cadd(tx, xh);
    }
#pragma unroll
    for (int hb = 0; hb < 2; ++hb)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int lo = 4 * hb + i, hi = lo + 2;
            const T tr = cmul(s1[hb], r[hi]), tx = cmul(s1[hb], x[lo]);
            r[hi] = csub(r[lo], tr);
            r[lo] = cadd(r[lo], tr);
            const T xh = x[hi];
            x[hi] = csub(tx, xh);
            x[lo] = cadd(tx, xh);
        }
    // leaves (2q, 2q+1): the phi-circulant [[a0, a1], [phi a1, a0]], phi = +-s_{L-1}
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const TW phi = (q & 1) ? cneg(s1[q >> 1]) : s1[q >> 1];
        const T a0 = r[2 * q], a1 = r[2 * q + 1], y0 = x[2 * q], y1 = x[2 * q + 1];
        const T a1f = cmul(phi, a1);
        r[2 * q] = cadd(cmul(a0, y0), cmul(a1, y1));
        r[2 * q + 1] = cadd(cmul(a1f, y0), cmul(a0, y1));
    }
    const TW i1[2] = {ld_tw(&sd.itw[(1 << (L - 1)) + 2 * t]), ld_tw(&sd.itw[(1 << (L - 1)) + 2 * t + 1])};
    const TW i0 = ld_tw(&sd.itw[(1 << (L - 2)) + t]);
#pragma unroll
    for (int hb = 0; hb < 2; ++hb)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int lo = 4 * hb + i, hi = lo + 2;
            const T sum = cadd(r[lo], r[hi]);
            r[hi] = csub(r[lo], r[hi]);
            r[lo] = cmul(sum, i1[hb]);
        }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const T sum = cadd(r[i], r[i + 4]);
        r[i + 4] = csub(r[i], r[i + 4]);
        r[i] = cmul(sum, i0);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) sd.ra(8 * t + i) = r[i];
}

// Stage 0 on the elements a thread loads from global memory: its groups are
// g = h + G i (i < 2^NL) of the numbers t + (n/8) k, k = 0..7, in r[k], x[k]
// (for every n >= 16, stage 0's element set is exactly that load set).  The
// results go to shared memory for stage 1 or the last stage.
template <int M, class T, class TW>
__device__ __forceinline__ void cfwd_stage0_regs(SideT<T, TW> &sd, int t, T *r, T *x)
{
    using Sh = CShape<M>;
    constexpr int NL = Sh::nl(0), G = 8 >> NL, MM = 1 << NL;
#pragma unroll
    for (int d = 0; d < NL; ++d) {
        const int hh = MM >> (d + 1);
#pragma unroll
        for (int j = 0; j < (1 << d); ++j) {
            const TW s = ld_tw(&sd.tw[(1 << d) + j]);
#pragma unroll
            for (int h = 0; h < G; ++h)
#pragma unroll
                for (int i = 0; i < hh; ++i) {
                    const int lo = h + G * ((j << (NL - d)) + i), hi = lo + G * hh;
                    const T tr = cmul(s, r[hi]);
                    const T tx = cmul(s, x[lo]);
                    r[hi] = csub(r[lo], tr);
                    r[lo] = cadd(r[lo], tr);
                    const T xh = x[hi];
                    x[hi] = csub(tx, xh);
                    x[lo] = cadd(tx, xh);
                }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        sd.ra(t + Sh::NTI * k) = r[k];
        sd.xa(t + Sh::NTI * k) = x[k];
    }
}

// The recombination of stage 0, ending in registers: r[k] receives the
// result's number t + (n/8) k.
template <int M, class T, class TW>
__device__ __forceinline__ void crec_stage0_regs(SideT<T, TW> &sd, int t, T *r)
{
    using Sh = CShape<M>;
    constexpr int NL = Sh::nl(0), G = 8 >> NL, MM = 1 << NL;
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = sd.ra(t + Sh::NTI * k);
#pragma unroll
    for (int d = NL - 1; d >= 0; --d) {
        const int hh = MM >> (d + 1);
#pragma unroll
        for (int j = 0; j < (1 << d); ++j) {
            const TW si = ld_tw(&sd.itw[(1 << d) + j]);
#pragma unroll
            for (int h = 0; h < G; ++h)
#pragma unroll
                for (int i = 0; i < hh; ++i) {
                    const int lo = h + G * ((j << (NL - d)) + i), hi = lo + G * hh;
                    const T sum = cadd(r[lo], r[hi]);
                    r[hi] = csub(r[lo], r[hi]);
                    r[lo] = cmul(sum, si);
                }
        }
    }
}

// The last stage (8 contiguous numbers at 8 t) exchanges numbers with the
// last register stage only between threads of one warp: the register
// stage's blocks of 2^(n - d0) numbers are 8 threads', cpos permutes inside
// 16-number blocks, and an instance's n / 8 threads are whole warps or lie
// inside one (checked on the CPU for n = 16 .. 4096).  So the barriers on
// either side of the last stage are warp syncs; the other stages' exchanges
// cross warps.

// whole product for one instance: forward stages, last stage, recombination
template <int M, int S, class T, class TW>
__device__ __forceinline__ void cfwd_all(SideT<T, TW> &sd, int t)
{
    if constexpr (S < CShape<M>::NST) {
        cfwd_stage<M, S, T, TW>(sd, t);
        if constexpr (S == CShape<M>::NST - 1)
            __syncwarp();   // next: the last stage
        else
            __syncthreads();
        cfwd_all<M, S + 1, T, TW>(sd, t);
    }
}

// recombination stages S .. LOW (each followed by a barrier)
template <int M, int S, class T, class TW, int LOW = 0>
__device__ __forceinline__ void crec_all(SideT<T, TW> &sd, int t)
{
    if constexpr (S >= LOW) {
        crec_stage<M, S, T, TW>(sd, t);
        __syncthreads();
        crec_all<M, S - 1, T, TW, LOW>(sd, t);
    }
}

template <int M, class T, class TW>
__device__ __forceinline__ void cproduct(SideT<T, TW> &sd, int t)
{
    cfwd_all<M, 0, T, TW>(sd, t);
    cleaf_stage<M, T, TW>(sd, t);
    __syncwarp();
    crec_all<M, CShape<M>::NST - 1, T, TW>(sd, t);
}

// The same product with stage 0 on registers at both ends (n >= 16): the
// inputs r[k], x[k] are the numbers t + (n/8) k of the row vector and the
// vector, and r[k] receives the same numbers of the result.  Shared memory
// need not hold the inputs; the caller's barriers: none before (each thread
// writes only its own slots first), and every thread must have left the
// product before shared memory is reused.
template <int M, class T, class TW>
__device__ __forceinline__ void cproduct_regs(SideT<T, TW> &sd, int t, T *r, T *x)
{
    static_assert(CShape<M>::NST >= 1, "n >= 16");
    cfwd_stage0_regs<M, T, TW>(sd, t, r, x);
    if constexpr (CShape<M>::NST == 1)
        __syncwarp();   // next: the last stage (n <= 64: the instance is inside one warp)
    else
        __syncthreads();
    cfwd_all<M, 1, T, TW>(sd, t);
    cleaf_stage<M, T, TW>(sd, t);
    __syncwarp();
    crec_all<M, CShape<M>::NST - 1, T, TW, 1>(sd, t);
    crec_stage0_regs<M, T, TW>(sd, t, r);
}

template <int M>
__global__ void __launch_bounds__(CShape<M>::CT, 8) k_cfwd(const __grid_constant__ CParams P)
{
    using Sh = CShape<M>;
    extern __shared__ __align__(16) float2 csm[];
    const int li = threadIdx.x / Sh::NTI, t = threadIdx.x % Sh::NTI;
    const uint64_t inst = (uint64_t)blockIdx.x * Sh::IPC + li;
    const bool live = inst < P.batch;
    Side sd{csm + (size_t)li * 2 * Sh::N, csm + (size_t)li * 2 * Sh::N + Sh::N, P.tw, P.itw};
    const float2 *a = reinterpret_cast<const float2 *>(P.a) + inst * Sh::N;
    const float2 *x = reinterpret_cast<const float2 *>(P.x) + inst * Sh::N;
    if constexpr (Sh::NST >= 1) {
        // stage 0 on the loaded registers at both ends (cproduct_regs)
        float2 r[8], xv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int e = t + Sh::NTI * k;
            r[k] = live ? a[e] : make_float2(0.f, 0.f);
            xv[k] = live ? x[e] : make_float2(0.f, 0.f);
        }
        cproduct_regs<M, float2, float2>(sd, t, r, xv);
        if (live) {
            float2 *c = reinterpret_cast<float2 *>(P.c) + inst * Sh::N;
#pragma unroll
            for (int k = 0; k < 8; ++k) c[t + Sh::NTI * k] = make_float2(r[k].x * P.scale, r[k].y * P.scale);
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int e = t + Sh::NTI * k;
        sd.ra(e) = live ? a[e] : make_float2(0.f, 0.f);
        sd.xa(e) = live ? x[e] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    cproduct<M, float2, float2>(sd, t);
    if (live) {
        float2 *c = reinterpret_cast<float2 *>(P.c) + inst * Sh::N;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int e = t + Sh::NTI * k;
            const float2 v = sd.ra(e);
            c[e] = make_float2(v.x * P.scale, v.y * P.scale);
        }
    }
}

// Products over GF(p^2): the same recursion and layout, uint2 elements; the
// deferred halvings are one multiplication by 2^-L mod p at the end.
template <int M>
__global__ void __launch_bounds__(CShape<M>::CT) k_gfwd(const __grid_constant__ GParams P)
{
    using Sh = CShape<M>;
    extern __shared__ __align__(16) uint2 gsm[];
    const int li = threadIdx.x / Sh::NTI, t = threadIdx.x % Sh::NTI;
    const uint64_t inst = (uint64_t)blockIdx.x * Sh::IPC + li;
    const bool live = inst < P.batch;
    SideT<uint2> sd{gsm + (size_t)li * 2 * Sh::N, gsm + (size_t)li * 2 * Sh::N + Sh::N, P.tw, P.itw};
    const uint2 *a = reinterpret_cast<const uint2 *>(P.a) + inst * Sh::N;
    const uint2 *x = reinterpret_cast<const uint2 *>(P.x) + inst * Sh::N;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int e = t + Sh::NTI * k;
        sd.ra(e) = live ? a[e] : make_uint2(0u, 0u);
        sd.xa(e) = live ? x[e] : make_uint2(0u, 0u);
    }
    __syncthreads();
    cproduct<M, uint2, uint2>(sd, t);
    if (live) {
        uint2 *c = reinterpret_cast<uint2 *>(P.c) + inst * Sh::N;
        const uint2 sc = make_uint2(P.scale, 0u);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int e = t + Sh::NTI * k;
            c[e] = cmul(sd.ra(e), sc);
        }
    }
}

// Products over Z/(2^K + 1), K = 64 W (ssa.cuh): twiddles are shifts; the
// deferred halvings are one shift by 2K - L at the end.
template <int M, int W>
__global__ void __launch_bounds__(CShape<M>::CT) k_sfwd(const __grid_constant__ SParams P)
{
    using Sh = CShape<M>;
    using E = SsaE<W>;
    extern __shared__ __align__(16) unsigned char ssm[];
    E *sbase = reinterpret_cast<E *>(ssm);
    const int li = threadIdx.x / Sh::NTI, t = threadIdx.x % Sh::NTI;
    const uint64_t inst = (uint64_t)blockIdx.x * Sh::IPC + li;
    const bool live = inst < P.batch;
    SideT<E, SsaTw<W>> sd{sbase + (size_t)li * 2 * Sh::N, sbase + (size_t)li * 2 * Sh::N + Sh::N,
                          reinterpret_cast<const SsaTw<W> *>(P.tw), reinterpret_cast<const SsaTw<W> *>(P.itw)};
    const E *a = reinterpret_cast<const E *>(P.a) + inst * Sh::N;
    const E *x = reinterpret_cast<const E *>(P.x) + inst * Sh::N;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int e = t + Sh::NTI * k;
        sd.ra(e) = live ? a[e] : ssa_zero<W>();
        sd.xa(e) = live ? x[e] : ssa_zero<W>();
    }
    __syncthreads();
    cproduct<M, E, SsaTw<W>>(sd, t);
    if (live) {
        E *c = reinterpret_cast<E *>(P.c) + inst * Sh::N;
        const SsaTw<W> sc{P.scale_exp};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int e = t + Sh::NTI * k;
            c[e] = cmul(sc, sd.ra(e));
        }
    }
}

// dL/dx and dL/da of one instance per Sh::NTI threads
template <int M>
__global__ void __launch_bounds__(CShape<M>::CT, 7) k_cbwd(const __grid_constant__ CBwdParams P)
{
    using Sh = CShape<M>;
    extern __shared__ __align__(16) float2 csm[];
    const int li = threadIdx.x / Sh::NTI, t = threadIdx.x % Sh::NTI;
    const uint64_t inst = (uint64_t)blockIdx.x * Sh::IPC + li;
    const bool live = inst < P.batch;
    float2 *base = csm + (size_t)li * 4 * Sh::N;
    Side sx{base, base + Sh::N, P.tw_x, P.itw_x};                // beta(a) and g
    Side sa{base + 2 * Sh::N, base + 3 * Sh::N, P.tw_a, P.itw_a};  // g and conj(x)
    const float2 *a = reinterpret_cast<const float2 *>(P.a) + inst * Sh::N;
    const float2 *x = reinterpret_cast<const float2 *>(P.x) + inst * Sh::N;
    const float2 *g = reinterpret_cast<const float2 *>(P.g) + inst * Sh::N;
    const float2 fc = make_float2(P.fc_re, P.fc_im);   // conj(f)
    if constexpr (Sh::NST >= 1) {
        // stage 0 on the loaded registers at both ends (cproduct_regs); g
        // is read again for the second product instead of kept
        const float2 z = make_float2(0.f, 0.f);
        float2 r[8], xv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int e = t + Sh::NTI * k;
            // beta_e = conj(a_0) for e = 0, conj(f) conj(a_{n-e}) otherwise
            const float2 ae = live ? a[e == 0 ? 0 : Sh::N - e] : z;
            r[k] = e == 0 ? cconj(ae) : cmul(fc, cconj(ae));
            xv[k] = live ? g[e] : z;
        }
        cproduct_regs<M, float2, float2>(sx, t, r, xv);
        if (live) {
            float2 *gx = reinterpret_cast<float2 *>(P.grad_x) + inst * Sh::N;
#pragma unroll
            for (int k = 0; k < 8; ++k) gx[t + Sh::NTI * k] = make_float2(r[k].x * P.scale, r[k].y * P.scale);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int e = t + Sh::NTI * k;
            r[k] = live ? g[e] : z;
            xv[k] = live ? cconj(x[e]) : z;
        }
        cproduct_regs<M, float2, float2>(sa, t, r, xv);
        if (live) {
            float2 *ga = reinterpret_cast<float2 *>(P.grad_a) + inst * Sh::N;
#pragma unroll
            for (int k = 0; k < 8; ++k) ga[t + Sh::NTI * k] = make_float2(r[k].x * P.scale, r[k].y * P.scale);
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int e = t + Sh::NTI * k;
        const float2 z = make_float2(0.f, 0.f);
        // beta_e = conj(a_0) for e = 0, conj(f) conj(a_{n-e}) otherwise
        const float2 ae = live ? a[e == 0 ? 0 : Sh::N - e] : z;
        sx.ra(e) = e == 0 ? cconj(ae) : cmul(fc, cconj(ae));
        const float2 ge = live ? g[e] : z;
        sx.xa(e) = ge;
        sa.ra(e) = ge;
        sa.xa(e) = live ? cconj(x[e]) : z;
    }
    __syncthreads();
    cproduct<M, float2, float2>(sx, t);
    cproduct<M, float2, float2>(sa, t);
    if (live) {
        float2 *gx = reinterpret_cast<float2 *>(P.grad_x) + inst * Sh::N;
        float2 *ga = reinterpret_cast<float2 *>(P.grad_a) + inst * Sh::N;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int e = t + Sh::NTI * k;
            const float2 vx = sx.ra(e), va = sa.ra(e);
            gx[e] = make_float2(vx.x * P.scale, vx.y * P.scale);
            ga[e] = make_float2(va.x * P.scale, va.y * P.scale);
        }
    }
}

// ---------------------------------------------------------------------------
// host: twiddle tables per (f, n), FP64 -> FP32

// Copies a plan's twiddle and inverse-twiddle tables to the device buffers
// d and di; on failure frees both.
int upload_tables(void *d, void *di, const void *h, const void *hi, size_t bytes)
{
    cudaError_t e = cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(di, hi, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        cudaFree(d);
        cudaFree(di);
        return fail(FCIRC_ECUDA, "plan tables: cudaMemcpy: %s", cudaGetErrorString(e));
    }
    return FCIRC_OK;
}

struct CPlanKey {
    int dev;
    double re, im;
    uint64_t n;
    bool operator<(const CPlanKey &o) const { return std::tie(dev, re, im, n) < std::tie(o.dev, o.re, o.im, o.n); }
};
std::mutex g_cmu;
std::map<CPlanKey, std::pair<float2 *, float2 *>> g_cplans;

int get_ctables(double fre, double fim, uint64_t n, const float2 **tw, const float2 **itw)
{
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    const CPlanKey key{dev, fre, fim, n};
    std::lock_guard<std::mutex> lk(g_cmu);
    auto it = g_cplans.find(key);
    if (it == g_cplans.end()) {
        const int m = ilog2(n), L = m - 1;
        const double r = std::hypot(fre, fim), th = std::atan2(fim, fre);
        std::vector<float2> h(n / 2), hi(n / 2);
        h[0] = hi[0] = make_float2(0.f, 0.f);
        for (int l = 0; l < L; ++l) {
            const double mag = std::pow(r, std::ldexp(1.0, -(l + 1)));
            for (uint64_t j = 0; j < ((uint64_t)1 << l); ++j) {
                const double ang = (th + 2.0 * M_PI * (double)host::bitrev(j, l)) / std::ldexp(1.0, l + 1);
                h[((size_t)1 << l) + j] = make_float2((float)(mag * std::cos(ang)), (float)(mag * std::sin(ang)));
                hi[((size_t)1 << l) + j] = make_float2((float)(std::cos(ang) / mag), (float)(-std::sin(ang) / mag));
            }
        }
        float2 *d = nullptr, *di = nullptr;
        if (dev_alloc((void **)&d, n / 2 * sizeof(float2)) != cudaSuccess ||
            dev_alloc((void **)&di, n / 2 * sizeof(float2)) != cudaSuccess) {
            (void)cudaGetLastError();
            cudaFree(d);
            return fail(FCIRC_ENOMEM, "complex plan: cudaMalloc failed");
        }
        FCIRC_TRY(upload_tables(d, di, h.data(), hi.data(), n / 2 * sizeof(float2)));
        it = g_cplans.emplace(key, std::make_pair(d, di)).first;
    }
    *tw = it->second.first;
    *itw = it->second.second;
    return FCIRC_OK;
}

// GF(p^2) twiddles per (f, n): s_{l,j} = rho^(2^(L-l-1)) psi_{2^(l+1)}^brv(j)
// with rho a 2^L-th root of f and psi_m a primitive m-th root of unity
// (gfp2.hpp), and their inverses; exact, cached per device.
struct GPlanKey {
    int dev;
    uint32_t re, im;
    uint64_t n;
    bool operator<(const GPlanKey &o) const { return std::tie(dev, re, im, n) < std::tie(o.dev, o.re, o.im, o.n); }
};
std::map<GPlanKey, std::pair<uint2 *, uint2 *>> g_gplans;

int get_gtables(uint32_t fre, uint32_t fim, uint64_t n, const uint2 **tw, const uint2 **itw)
{
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    const GPlanKey key{dev, fre, fim, n};
    std::lock_guard<std::mutex> lk(g_cmu);
    auto it = g_gplans.find(key);
    if (it == g_gplans.end()) {
        const int m = ilog2(n), L = m - 1;
        gf::E rho;
        if (!gf::root_2k(gf::E{fre, fim}, L, rho))
            return fail(FCIRC_ENOROOT, "GF(p^2) product: f = %u + %u sqrt 3 has no 2^%d-th root", fre, fim, L);
        std::vector<uint2> h(n / 2), hi(n / 2);
        h[0] = hi[0] = make_uint2(0u, 0u);
        for (int l = 0; l < L; ++l) {
            const gf::E r = gf::pow(rho, (uint64_t)1 << (L - l - 1));
            const gf::E psi = gf::root_of_unity(l + 1);
            for (uint64_t j = 0; j < ((uint64_t)1 << l); ++j) {
                const gf::E s = gf::mul(r, gf::pow(psi, host::bitrev(j, l)));
                const gf::E si = gf::inv(s);
                h[((size_t)1 << l) + j] = make_uint2(s.re, s.im);
                hi[((size_t)1 << l) + j] = make_uint2(si.re, si.im);
            }
        }
        uint2 *d = nullptr, *di = nullptr;
        if (dev_alloc((void **)&d, n / 2 * sizeof(uint2)) != cudaSuccess ||
            dev_alloc((void **)&di, n / 2 * sizeof(uint2)) != cudaSuccess) {
            (void)cudaGetLastError();
            cudaFree(d);
            return fail(FCIRC_ENOMEM, "GF(p^2) plan: cudaMalloc failed");
        }
        FCIRC_TRY(upload_tables(d, di, h.data(), hi.data(), n / 2 * sizeof(uint2)));
        it = g_gplans.emplace(key, std::make_pair(d, di)).first;
    }
    *tw = it->second.first;
    *itw = it->second.second;
    return FCIRC_OK;
}

// Z/(2^K + 1) twiddles per (K, f = 2^fe, n): exponents mod 2K of
// s_{l,j} = rho^(2^(L-l-1)) psi_{2^(l+1)}^brv(j), rho = 2^(fe / 2^L),
// psi_m = 2^(2K/m); inverses 2^(2K - e).
struct SPlanKey {
    int dev;
    uint32_t K, fe;
    uint64_t n;
    bool operator<(const SPlanKey &o) const { return std::tie(dev, K, fe, n) < std::tie(o.dev, o.K, o.fe, o.n); }
};
std::map<SPlanKey, std::pair<int *, int *>> g_splans;

int get_stables(uint32_t K, uint32_t fe, uint64_t n, const int **tw, const int **itw)
{
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    const SPlanKey key{dev, K, fe, n};
    std::lock_guard<std::mutex> lk(g_cmu);
    auto it = g_splans.find(key);
    if (it == g_splans.end()) {
        const int m = ilog2(n), L = m - 1;
        const uint64_t twoK = 2ull * K;
        if ((((uint64_t)1 << L) > twoK) || (fe % ((uint64_t)1 << L)) != 0)
            return fail(FCIRC_ENOROOT, "Z/(2^%u + 1): f = 2^%u has no 2^%d-th root that is a power of 2", K, fe, L);
        const uint64_t er = fe >> L;
        std::vector<int> h(n / 2), hi(n / 2);
        h[0] = hi[0] = 0;
        for (int l = 0; l < L; ++l)
            for (uint64_t j = 0; j < ((uint64_t)1 << l); ++j) {
                const uint64_t e = (er * ((uint64_t)1 << (L - l - 1)) + (twoK >> (l + 1)) * host::bitrev(j, l)) % twoK;
                h[((size_t)1 << l) + j] = (int)e;
                hi[((size_t)1 << l) + j] = (int)((twoK - e) % twoK);
            }
        int *d = nullptr, *di = nullptr;
        if (dev_alloc((void **)&d, n / 2 * sizeof(int)) != cudaSuccess ||
            dev_alloc((void **)&di, n / 2 * sizeof(int)) != cudaSuccess) {
            (void)cudaGetLastError();
            cudaFree(d);
            return fail(FCIRC_ENOMEM, "Z/(2^K+1) plan: cudaMalloc failed");
        }
        FCIRC_TRY(upload_tables(d, di, h.data(), hi.data(), n / 2 * sizeof(int)));
        it = g_splans.emplace(key, std::make_pair(d, di)).first;
    }
    *tw = it->second.first;
    *itw = it->second.second;
    return FCIRC_OK;
}

template <class K>
int set_smem(K kernel, int bytes)
{
    FCIRC_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return FCIRC_OK;
}

template <int M>
int launch_cfwd_m(const CParams &P, cudaStream_t s)
{
    using Sh = CShape<M>;
    const int smem = Sh::IPC * 2 * Sh::N * (int)sizeof(float2);
    FCIRC_TRY(set_smem(k_cfwd<M>, smem));
    const uint64_t grid = (P.batch + Sh::IPC - 1) / Sh::IPC;
    ProfScope ps("k_cfwd", s);
    k_cfwd<M><<<(unsigned)grid, Sh::CT, smem, s>>>(P);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

template <int M>
int launch_gfwd_m(const GParams &P, cudaStream_t s)
{
    using Sh = CShape<M>;
    const int smem = Sh::IPC * 2 * Sh::N * (int)sizeof(uint2);
    FCIRC_TRY(set_smem(k_gfwd<M>, smem));
    const uint64_t grid = (P.batch + Sh::IPC - 1) / Sh::IPC;
    ProfScope ps("k_gfwd", s);
    k_gfwd<M><<<(unsigned)grid, Sh::CT, smem, s>>>(P);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

template <int M, int W>
int launch_sfwd_mw(const SParams &P, cudaStream_t s)
{
    using Sh = CShape<M>;
    const int smem = Sh::IPC * 2 * Sh::N * (int)sizeof(SsaE<W>);
    if (smem > 227 * 1024) return fail(FCIRC_EINVAL, "Z/(2^K+1) product: n = %d too large for K = %d", Sh::N, 64 * W);
    FCIRC_TRY(set_smem(k_sfwd<M, W>, smem));
    const uint64_t grid = (P.batch + Sh::IPC - 1) / Sh::IPC;
    ProfScope ps("k_sfwd", s);
    k_sfwd<M, W><<<(unsigned)grid, Sh::CT, smem, s>>>(P);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

template <int W>
int launch_sfwd_w(const SParams &P, int m, cudaStream_t s)
{
    switch (m) {
    case 3: return launch_sfwd_mw<3, W>(P, s);
    case 4: return launch_sfwd_mw<4, W>(P, s);
    case 5: return launch_sfwd_mw<5, W>(P, s);
    case 6: return launch_sfwd_mw<6, W>(P, s);
    case 7: return launch_sfwd_mw<7, W>(P, s);
    case 8: return launch_sfwd_mw<8, W>(P, s);
    case 9: return launch_sfwd_mw<9, W>(P, s);
    default: return fail(FCIRC_EINVAL, "Z/(2^K+1) product: n = 2^%d not supported", m);
    }
}

template <int M>
int launch_cbwd_m(const CBwdParams &P, cudaStream_t s)
{
    using Sh = CShape<M>;
    const int smem = Sh::IPC * 4 * Sh::N * (int)sizeof(float2);
    FCIRC_TRY(set_smem(k_cbwd<M>, smem));
    const uint64_t grid = (P.batch + Sh::IPC - 1) / Sh::IPC;
    ProfScope ps("k_cbwd", s);
    k_cbwd<M><<<(unsigned)grid, Sh::CT, smem, s>>>(P);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

}  // namespace

void release_cplans()
{
    std::lock_guard<std::mutex> lk(g_cmu);
    for (auto &kv : g_cplans) {
        cudaSetDevice(kv.first.dev);
        cudaDeviceSynchronize();
        cudaFree(kv.second.first);
        cudaFree(kv.second.second);
    }
    g_cplans.clear();
    for (auto &kv : g_gplans) {
        cudaSetDevice(kv.first.dev);
        cudaDeviceSynchronize();
        cudaFree(kv.second.first);
        cudaFree(kv.second.second);
    }
    g_gplans.clear();
    for (auto &kv : g_splans) {
        cudaSetDevice(kv.first.dev);
        cudaDeviceSynchronize();
        cudaFree(kv.second.first);
        cudaFree(kv.second.second);
    }
    g_splans.clear();
}

int ssa_tables(uint32_t K, uint32_t fe, uint64_t n, const int **tw, const int **itw)
{
    return get_stables(K, fe, n, tw, itw);
}

int launch_sfwd(const SParams &P, int K, int m, cudaStream_t s)
{
    if (K == 64) return launch_sfwd_w<1>(P, m, s);
    if (K == 128) return launch_sfwd_w<2>(P, m, s);
    return fail(FCIRC_EINVAL, "Z/(2^K+1) product: K = %d not supported (64 or 128)", K);
}

int gf_tables(uint32_t fre, uint32_t fim, uint64_t n, const uint2 **tw, const uint2 **itw)
{
    return get_gtables(fre, fim, n, tw, itw);
}

int launch_gfwd(const GParams &P, int m, cudaStream_t s)
{
    switch (m) {
    case 3: return launch_gfwd_m<3>(P, s);
    case 4: return launch_gfwd_m<4>(P, s);
    case 5: return launch_gfwd_m<5>(P, s);
    case 6: return launch_gfwd_m<6>(P, s);
    case 7: return launch_gfwd_m<7>(P, s);
    case 8: return launch_gfwd_m<8>(P, s);
    case 9: return launch_gfwd_m<9>(P, s);
    case 10: return launch_gfwd_m<10>(P, s);
    case 11: return launch_gfwd_m<11>(P, s);
    case 12: return launch_gfwd_m<12>(P, s);
    default: return fail(FCIRC_EINVAL, "GF(p^2) product: n = 2^%d not supported", m);
    }
}

int complex_tables(double fre, double fim, uint64_t n, const float2 **tw, const float2 **itw)
{
    return get_ctables(fre, fim, n, tw, itw);
}

int launch_cfwd(const CParams &P, int m, cudaStream_t s)
{
    switch (m) {
    case 3: return launch_cfwd_m<3>(P, s);
    case 4: return launch_cfwd_m<4>(P, s);
    case 5: return launch_cfwd_m<5>(P, s);
    case 6: return launch_cfwd_m<6>(P, s);
    case 7: return launch_cfwd_m<7>(P, s);
    case 8: return launch_cfwd_m<8>(P, s);
    case 9: return launch_cfwd_m<9>(P, s);
    case 10: return launch_cfwd_m<10>(P, s);
    case 11: return launch_cfwd_m<11>(P, s);
    case 12: return launch_cfwd_m<12>(P, s);
    default: return fail(FCIRC_EINVAL, "complex product: n = 2^%d not supported", m);
    }
}

int launch_cbwd(const CBwdParams &P, int m, cudaStream_t s)
{
    switch (m) {
    case 3: return launch_cbwd_m<3>(P, s);
    case 4: return launch_cbwd_m<4>(P, s);
    case 5: return launch_cbwd_m<5>(P, s);
    case 6: return launch_cbwd_m<6>(P, s);
    case 7: return launch_cbwd_m<7>(P, s);
    case 8: return launch_cbwd_m<8>(P, s);
    case 9: return launch_cbwd_m<9>(P, s);
    case 10: return launch_cbwd_m<10>(P, s);
    case 11: return launch_cbwd_m<11>(P, s);
    case 12: return launch_cbwd_m<12>(P, s);
    default: return fail(FCIRC_EINVAL, "complex backward: n = 2^%d not supported", m);
    }
}

}  // namespace fcirc
