// tile_dev.cuh -- the tile transforms as device functions, shared by the
// tile kernels and the persistent batched kernel.  A tile is a contiguous
// block of 2^logT residues (a node of the recursion of Algorithm 1) on which
// every remaining halving level of both input sides, the 2x2 leaf products
// and the recombination back to the tile's level run inside one CTA.
#pragma once
#include <stdint.h>

#include "kernels_mod.hpp"
#include "modarith.cuh"
#include "tma.cuh"

namespace fcirc {

__device__ __forceinline__ uint32_t load_src(const Src &s, uint64_t N, uint64_t idx, uint32_t p)
{
    uint32_t v;
    switch (s.kind) {
    case SRC_U32:
        v = static_cast<const uint32_t *>(s.ptr)[idx];
        break;
    case SRC_U16_REV: {
        // a'[idx] = P[N-1-idx] with P zero-padded to N
        uint64_t j = N - 1 - idx;
        v = j < s.len ? static_cast<const uint16_t *>(s.ptr)[j] : 0u;
        break;
    }
    case SRC_U32_REV:
        // a'[idx] = a[N-1-idx]
        v = static_cast<const uint32_t *>(s.ptr)[N - 1 - idx];
        break;
    default:  // SRC_U16
        v = idx < s.len ? static_cast<const uint16_t *>(s.ptr)[idx] : 0u;
    }
    return s.scaled ? shoup_mul(v, s.scale.w, s.scale.wp, p) : v;
}


// Source modes are compile-time so that every load loop is branch-free and
// all of a thread's loads can be in flight together:
//   bits 0-1: SrcKind; bit 2: multiply by Src::scale on load;
//   bits 3-4: zero half of a first pass (1: below N/2, 2: from N/2).
enum : int {
    MODE_U32 = SRC_U32,
    MODE_U32_S = SRC_U32 | 4,
    MODE_REV_S = SRC_U16_REV | 4,
    MODE_U32REV_S = SRC_U32_REV | 4,
    MODE_REV_S_H = SRC_U16_REV | 4 | (1 << 3),
    MODE_U16 = SRC_U16,
    MODE_U16_H = SRC_U16 | (2 << 3),
};

template <int MODE>
__device__ __forceinline__ uint32_t ld_raw(const Src &s, uint32_t N, uint32_t idx)
{
    constexpr int KIND = MODE & 3;
    if constexpr (KIND == SRC_U32) {
        return static_cast<const uint32_t *>(s.ptr)[idx];
    } else if constexpr (KIND == SRC_U32_REV) {
        return static_cast<const uint32_t *>(s.ptr)[N - 1 - idx];   // a'[idx] = a[N-1-idx]
    } else if constexpr (KIND == SRC_U16_REV) {
        const uint32_t j = N - 1 - idx;   // a'[idx] = P[N-1-idx], P zero-padded
        return j < s.len ? (uint32_t) static_cast<const uint16_t *>(s.ptr)[j] : 0u;
    } else {
        return idx < s.len ? (uint32_t) static_cast<const uint16_t *>(s.ptr)[idx] : 0u;
    }
}

template <int MODE>
__device__ __forceinline__ uint32_t ld_scale(uint32_t v, const Src &s, uint32_t p)
{
    if constexpr ((MODE & 4) != 0)
        return shoup_mul(v, s.scale.w, s.scale.wp, p);
    else
        return v;
}

// ---------------------------------------------------------------------------
// register stages.  A group of 2^NL registers v[0..2^NL) is the subtree of one
// node: local level d pairs v[k] with v[k + h], h = 2^(NL-d-1), inside local
// node j = k >> (NL - d); tw(d, j) is that node's twiddle (or its inverse).

template <int NL, int NLEV, class TwFn>
__device__ __forceinline__ void fwd2(uint32_t *a, uint32_t *x, TwFn tw, uint32_t p, uint32_t p2)
{
#pragma unroll
    for (int d = 0; d < NLEV; ++d) {
        const int h = (1 << NL) >> (d + 1);
#pragma unroll
        for (int j = 0; j < (1 << d); ++j) {
            const Tw s = tw(d, j);
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const int lo = (j << (NL - d)) + i;
                bfly_row(a[lo], a[lo + h], s, p, p2);
                bfly_vec(x[lo], x[lo + h], s, p, p2);
            }
        }
    }
}

// forward levels of one side only (VEC: the vector side)
template <int NL, int NLEV, bool VEC, class TwFn>
__device__ __forceinline__ void fwd1(uint32_t *v, TwFn tw, uint32_t p, uint32_t p2)
{
#pragma unroll
    for (int d = 0; d < NLEV; ++d) {
        const int h = (1 << NL) >> (d + 1);
#pragma unroll
        for (int j = 0; j < (1 << d); ++j) {
            const Tw s = tw(d, j);
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const int lo = (j << (NL - d)) + i;
                if (VEC)
                    bfly_vec(v[lo], v[lo + h], s, p, p2);
                else
                    bfly_row(v[lo], v[lo + h], s, p, p2);
            }
        }
    }
}

// recombination, local levels NLEV-1 .. 0
template <int NL, int NLEV, class TwFn>
__device__ __forceinline__ void rec1(uint32_t *v, TwFn tw, uint32_t p, uint32_t p2)
{
#pragma unroll
    for (int d = NLEV - 1; d >= 0; --d) {
        const int h = (1 << NL) >> (d + 1);
#pragma unroll
        for (int j = 0; j < (1 << d); ++j) {
            const Tw s = tw(d, j);
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const int lo = (j << (NL - d)) + i;
                bfly_rec(v[lo], v[lo + h], s, p, p2);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// tile kernel, 4096 residues, 256 threads

// Shared-memory position of tile element e: 128-bit chunks (e >> 2) are
// permuted inside each 128-byte row by an XOR with bits of the row index, so
// that the three access patterns (stride 256, the 16 x 16 transpose and the
// contiguous 16-residue groups read as 128-bit vectors) are conflict-free.
__device__ __forceinline__ int tphi(int e)
{
    const int c = e >> 2, r = c >> 3, col = c & 7;
    const int g = (r & 3) ^ ((r & 8) >> 1);
    return (((r << 3) | (col ^ g)) << 2) | (e & 3);
}

// The three patterns as a per-thread base and terms that are compile-time
// constants in the unrolled loops (so every access is one XOR at most and an
// immediate offset; identities checked for every thread on the CPU):
//   tphi(tid + 256 j)  = (tphi(tid) ^ 16 (j & 1)) + 256 j
//   tphi(eb + 16 m)    = (tphi(eb) ^ (4 ((m >> 1) & 3) | 16 (m & 1))) + 32 (m >> 1)
//   tphi(16 tid + 4 q) = tphi(16 tid) ^ 4 q
__device__ __forceinline__ int tphiA(int tA, int j) { return (tA ^ ((j & 1) << 4)) + (j << 8); }
__device__ __forceinline__ int tphiB(int tB, int m) { return (tB ^ ((((m >> 1) & 3) << 2) | ((m & 1) << 4))) + ((m >> 1) << 5); }
__device__ __forceinline__ int tphiC(int tC, int q) { return tC ^ (q << 2); }

// One tile: J gives the sides, destination, tables and prime; base is the
// tile's first index in arrays of length N; sg its 11 levels of factors
// (6 words each, see plan.cu); SA, SX (4096 words each, 16-byte aligned),
// STW, SITW (256 entries) are this CTA's shared memory.  256 threads.
// ilv (TileParams::ilv): bit 0, the row vector is in the tile-pair
// interleaved layout; bit 1, the vector and the destination are.  Residue
// base + tid + 256 j then sits at ilv_pos(base + tid) + 512 j.
//
// TMA: the interleaved sides arrive as TMA tensor copies (TP->tmap of job jq:
// four boxes of 256 column quads per side) in natural order in SA / SX, and
// the products leave the same way from SX.  Thread 0 issues the copies and
// waits on the mbarrier *bar with at most TP->spin_limit probes; if it gives
// up, it records FCIRC_ETIMEOUT in *TP->status, waits (bounded) for the
// copies still in flight, and the whole CTA returns.  SA, SX 128-byte
// aligned; *flag a shared word.
constexpr uint32_t kTmaDrainProbes = 1u << 24;

template <int MA, int MX, int VAR = TILE_FULL, bool TMA = false>
__device__ __forceinline__ void tile4096_dev(const TileJob &J, uint32_t N, uint32_t base, const uint32_t *sg,
                                             uint32_t *SA, uint32_t *SX, Tw *STW, Tw *SITW, int ilv = 0,
                                             const TileParams *TP = nullptr, int jq = 0, uint64_t *bar = nullptr,
                                             uint32_t *flag = nullptr)
{
    constexpr bool DO_A = VAR != TILE_PLANNED, DO_X = VAR != TILE_ROW;
    const uint32_t p = J.p, p2 = 2 * J.p, pinv = J.pinv;
    const int tid = threadIdx.x;
    // the TMA form: the vector and the destination always through TMA, the
    // row vector too unless it is a plan's transformed one (tile_tma_maps)
    constexpr bool tma_a = TMA && DO_A && VAR != TILE_PLANNED, tma_x = TMA && DO_X;
    const int tp = (int)(base >> 12);   // tile index: pair tp >> 1, parity tp & 1
    if constexpr (TMA) {
        if (tid == 0) {
            mbar_init(bar, 1);
            mbar_arrive_expect_tx(bar, (tma_a ? 16384u : 0u) + (tma_x ? 16384u : 0u));
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (tma_a) tma_load_4d(SA + 1024 * i, &TP->tmap[jq][0], bar, 0, tp & 1, 256 * i, tp >> 1);
                if (tma_x) tma_load_4d(SX + 1024 * i, &TP->tmap[jq][1], bar, 0, tp & 1, 256 * i, tp >> 1);
            }
        }
    }

    // twiddles of tile levels 0..7 (heap index 1..255), one per thread
    if (tid > 0) {
        const int d = 31 - __clz(tid);
        const uint32_t *e = sg + d * 6;
        STW[tid] = twiddle_from(J.U[tid], e[0], e[1], e[2], p);
        if (VAR != TILE_ROW) SITW[tid] = twiddle_from(J.Ui[tid], e[3], e[4], e[5], p);
    }
    uint32_t a[16], x[16];
    const uint32_t ipos = ilv_pos(base + tid);
    const uint32_t ia = (ilv & 1) ? ipos : base + tid, sa = (ilv & 1) ? 512u : 256u;
    const uint32_t ix = (ilv & 2) ? ipos : base + tid, sx = (ilv & 2) ? 512u : 256u;
    if constexpr (TMA) {
        if (tid == 0) {
            const bool ok = mbar_wait_bounded(bar, 0, TP->spin_limit);
            if (!ok) {
                atomicCAS(TP->status, 0u, (uint32_t)FCIRC_ETIMEOUT);
                // the copies still in flight land in this CTA's shared memory
                mbar_wait_bounded(bar, 0, kTmaDrainProbes);
            }
            *flag = ok ? 1u : 0u;
        }
        __syncthreads();
        if (*flag == 0) return;   // the same verdict for every thread
        // the phase has completed: each thread's own probe succeeds at once
        // and makes the copied data visible to it
        mbar_wait_bounded(bar, 0, kTmaDrainProbes);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (DO_A) a[j] = tma_a ? SA[tid + 256 * j] : ld_raw<MA>(J.a, N, ia + sa * j);
        if (DO_X) x[j] = tma_x ? SX[tid + 256 * j] : ld_raw<MX>(J.x, N, ix + sx * j);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (DO_A) a[j] = ld_scale<MA>(a[j], J.a, p);
        if (DO_X) x[j] = ld_scale<MX>(x[j], J.x, p);
    }
    __syncthreads();

    const int tA = tphi(tid);
    // stage A: tile levels 0..3, residues tid + 256 j
    auto twA = [&](int d, int j) { return STW[(1 << d) + j]; };
    if (DO_A && DO_X)
        fwd2<4, 4>(a, x, twA, p, p2);
    else if (DO_A)
        fwd1<4, 4, false>(a, twA, p, p2);
    else
        fwd1<4, 4, true>(x, twA, p, p2);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (DO_A) SA[tphiA(tA, j)] = a[j];
        if (DO_X) SX[tphiA(tA, j)] = x[j];
    }
    __syncthreads();
    // stage B: levels 4..7, residues 256 (tid >> 4) + 16 m + (tid & 15)
    const int eb = ((tid >> 4) << 8) + (tid & 15);
    const int tB = tphi(eb), tC = tphi(16 * tid);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        if (DO_A) a[m] = SA[tphiB(tB, m)];
        if (DO_X) x[m] = SX[tphiB(tB, m)];
    }
    const int nb = tid >> 4;
    auto twB = [&](int d, int j) { return STW[(1 << (4 + d)) + (nb << d) + j]; };
    if (DO_A && DO_X)
        fwd2<4, 4>(a, x, twB, p, p2);
    else if (DO_A)
        fwd1<4, 4, false>(a, twB, p, p2);
    else
        fwd1<4, 4, true>(x, twB, p, p2);
    // Stages B and C work on the same 256-residue block, tid >> 4, held by
    // the 16 threads of one half-warp, and tphi keeps a block inside its own
    // 128-byte rows: the exchanges between them need only the warp's
    // threads to meet (__syncwarp orders their shared-memory accesses).
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        if (DO_A) SA[tphiB(tB, m)] = a[m];
        if (DO_X) SX[tphiB(tB, m)] = x[m];
    }
    __syncwarp();
    // stage C: levels 8..10 and the leaves, residues 16 tid .. 16 tid + 15
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (DO_A) {
            const uint4 va = *reinterpret_cast<const uint4 *>(&SA[tphiC(tC, q)]);
            a[4 * q] = va.x; a[4 * q + 1] = va.y; a[4 * q + 2] = va.z; a[4 * q + 3] = va.w;
        }
        if (DO_X) {
            const uint4 vx = *reinterpret_cast<const uint4 *>(&SX[tphiC(tC, q)]);
            x[4 * q] = vx.x; x[4 * q + 1] = vx.y; x[4 * q + 2] = vx.z; x[4 * q + 3] = vx.w;
        }
    }
    Tw tc[7];   // this thread's nodes: level 8 (tid), 9 (2 tid + r), 10 (4 tid + r)
    {
        const uint32_t *e8 = sg + 8 * 6, *e9 = sg + 9 * 6, *e10 = sg + 10 * 6;
        tc[0] = twiddle_from(J.U[256 + tid], e8[0], e8[1], e8[2], p);
#pragma unroll
        for (int r = 0; r < 2; ++r) tc[1 + r] = twiddle_from(J.U[512 + 2 * tid + r], e9[0], e9[1], e9[2], p);
#pragma unroll
        for (int r = 0; r < 4; ++r) tc[3 + r] = twiddle_from(J.U[1024 + 4 * tid + r], e10[0], e10[1], e10[2], p);
    }
    auto twC = [&](int d, int j) { return tc[(1 << d) - 1 + j]; };
    if (DO_A && DO_X)
        fwd2<4, 3>(a, x, twC, p, p2);
    else if (DO_A)
        fwd1<4, 3, false>(a, twC, p, p2);
    else
        fwd1<4, 3, true>(x, twC, p, p2);
    if constexpr (VAR == TILE_ROW) {
        // the transformed row vector, 16 contiguous residues per thread
        uint4 *d = reinterpret_cast<uint4 *>(J.dst + base + 16 * tid);
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] = make_uint4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
        return;
    }
    if constexpr (VAR == TILE_PLANNED) {
        const uint4 *s = reinterpret_cast<const uint4 *>(static_cast<const uint32_t *>(J.a.ptr) + base + 16 * tid);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 va = __ldg(s + q);
            a[4 * q] = va.x; a[4 * q + 1] = va.y; a[4 * q + 2] = va.z; a[4 * q + 3] = va.w;
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        Tw phi = tc[3 + (q >> 1)];
        if (q & 1) phi = tw_neg(phi, p);
        leaf2(a[2 * q], a[2 * q + 1], x[2 * q], x[2 * q + 1], phi, p, p2, pinv);
        if constexpr (VAR == TILE_SHIFT) {
            // the row vector shifted by one place (bfly_rec_shift): entry 0
            // is c1, entry 1 is phi c0 -- kept as c0 here, the factor phi
            // going into the first recombination level
            const uint32_t c0 = a[2 * q];
            a[2 * q] = a[2 * q + 1];
            a[2 * q + 1] = c0;
        }
    }
    Tw f10[4];   // forward level-10 twiddles, for bfly_rec_shift
    if constexpr (VAR == TILE_SHIFT) {
#pragma unroll
        for (int r = 0; r < 4; ++r) f10[r] = tc[3 + r];
    }
    {
        const uint32_t *e8 = sg + 8 * 6, *e9 = sg + 9 * 6, *e10 = sg + 10 * 6;
        tc[0] = twiddle_from(J.Ui[256 + tid], e8[3], e8[4], e8[5], p);
#pragma unroll
        for (int r = 0; r < 2; ++r) tc[1 + r] = twiddle_from(J.Ui[512 + 2 * tid + r], e9[3], e9[4], e9[5], p);
#pragma unroll
        for (int r = 0; r < 4; ++r) tc[3 + r] = twiddle_from(J.Ui[1024 + 4 * tid + r], e10[3], e10[4], e10[5], p);
    }
    if constexpr (VAR == TILE_SHIFT) {
        // level 10: position-0 pairs as usual, position-1 pairs with the
        // leaves' missing factor phi = +-s
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            bfly_rec(a[4 * j], a[4 * j + 2], tc[3 + j], p, p2);
            bfly_rec_shift(a[4 * j + 1], a[4 * j + 3], f10[j], p, p2);
        }
        rec1<4, 2>(a, [&](int d, int j) { return tc[(1 << d) - 1 + j]; }, p, p2);
    } else {
        rec1<4, 3>(a, [&](int d, int j) { return tc[(1 << d) - 1 + j]; }, p, p2);
    }
    // back from stage C to stage B, and stage B's writes: inside the block
    // of this half-warp (see the forward exchange)
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4 *>(&SA[tphiC(tC, q)]) =
            make_uint4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 16; ++m) a[m] = SA[tphiB(tB, m)];
    rec1<4, 4>(a, [&](int d, int j) { return SITW[(1 << (4 + d)) + (nb << d) + j]; }, p, p2);
    __syncwarp();
#pragma unroll
    for (int m = 0; m < 16; ++m) SA[tphiB(tB, m)] = a[m];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 16; ++j) a[j] = SA[tphiA(tA, j)];
    rec1<4, 4>(a, [&](int d, int j) { return SITW[(1 << d) + j]; }, p, p2);
    if constexpr (TMA) {
        // the products through SX (free since the leaves) and four TMA boxes
#pragma unroll
        for (int j = 0; j < 16; ++j) SX[tid + 256 * j] = J.store_lazy ? a[j] : reduce_once(a[j], p);
        fence_async_shared();
        __syncthreads();
        if (tid == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) tma_store_4d(&TP->tmap[jq][2], SX + 1024 * i, 0, tp & 1, 256 * i, tp >> 1);
            tma_store_commit();
            tma_store_wait_read();   // SX stays valid until the stores have read it
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) J.dst[ix + sx * j] = J.store_lazy ? a[j] : reduce_once(a[j], p);
}

// Any tile size 2 <= T = 2^logT <= 4096 (D = logT - 1 halving levels), with
// the level loops in shared memory (16 T bytes at smem).  sg: the tile's D
// levels of factors; rho_t: the leaf parameter when D = 0.
__device__ __forceinline__ void tile_generic_dev(const TileJob &J, uint64_t N, uint64_t base, int logT, int D,
                                                 const uint32_t *sg, Tw rho_t, uint32_t *smem)
{
    const int T = 1 << logT;
    const uint32_t p = J.p, p2 = 2 * J.p, pinv = J.pinv;
    uint32_t *A = smem;
    uint32_t *X = A + T;
    Tw *tw = reinterpret_cast<Tw *>(X + T);   // [T/2], heap index 2^d + j'
    Tw *itw = tw + (T >> 1);

    for (int i = threadIdx.x; i < T; i += blockDim.x) {
        A[i] = load_src(J.a, N, base + i, p);
        X[i] = load_src(J.x, N, base + i, p);
    }
    if (D > 0) {
        for (int idx = threadIdx.x + 1; idx < (1 << D); idx += blockDim.x) {
            int d = 31 - __clz(idx);
            const uint32_t *e = sg + d * 6;
            tw[idx] = twiddle_from(J.U[idx], e[0], e[1], e[2], p);
            itw[idx] = twiddle_from(J.Ui[idx], e[3], e[4], e[5], p);
        }
    }
    __syncthreads();

    // both input sides, levels k .. L-1 (relative 0 .. D-1)
    for (int d = 0; d < D; ++d) {
        const int lh = logT - d - 1;
        const int half = 1 << lh;
        for (int b = threadIdx.x; b < (T >> 1); b += blockDim.x) {
            const int jn = b >> lh, i = b & (half - 1);
            const int lo = (jn << (lh + 1)) + i, hi = lo + half;
            const Tw s = tw[(1 << d) + jn];
            uint32_t a0 = A[lo], a1 = A[hi];
            bfly_row(a0, a1, s, p, p2);
            A[lo] = a0;
            A[hi] = a1;
            uint32_t x0 = X[lo], x1 = X[hi];
            bfly_vec(x0, x1, s, p, p2);
            X[lo] = x0;
            X[hi] = x1;
        }
        __syncthreads();
    }
    // 2x2 leaves: leaf e has parameter +s or -s of its parent node
    for (int e = threadIdx.x; e < (T >> 1); e += blockDim.x) {
        Tw phi;
        if (D == 0) {
            phi = rho_t;
        } else {
            phi = tw[(1 << (D - 1)) + (e >> 1)];
            if (e & 1) phi = tw_neg(phi, p);
        }
        uint32_t a0 = A[2 * e], a1 = A[2 * e + 1];
        leaf2(a0, a1, X[2 * e], X[2 * e + 1], phi, p, p2, pinv);
        A[2 * e] = a0;
        A[2 * e + 1] = a1;
    }
    __syncthreads();
    // recombination, levels L-1 .. k
    for (int d = D - 1; d >= 0; --d) {
        const int lh = logT - d - 1;
        const int half = 1 << lh;
        for (int b = threadIdx.x; b < (T >> 1); b += blockDim.x) {
            const int jn = b >> lh, i = b & (half - 1);
            const int lo = (jn << (lh + 1)) + i, hi = lo + half;
            uint32_t m1 = A[lo], m2 = A[hi];
            bfly_rec(m1, m2, itw[(1 << d) + jn], p, p2);
            A[lo] = m1;
            A[hi] = m2;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < T; i += blockDim.x) {
        uint32_t v = A[i];
        J.dst[base + i] = J.store_lazy ? v : reduce_once(v, p);
    }
}


}  // namespace fcirc
