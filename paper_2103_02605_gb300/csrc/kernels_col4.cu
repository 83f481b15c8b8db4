// kernels_col4.cu -- column passes of the recursion of Algorithm 1
// (Section 2) with four adjacent columns per thread.
//
// A column pass runs LF (8..12) consecutive halving levels over an array
// viewed as 2^LF rows of 2^logS columns: level d pairs rows r and
// r + 2^(LF-d-1) inside blocks of 2^(LF-d) rows, and every column undergoes
// the same butterflies with the same twiddles.  A CTA of 256 threads owns
// 2^(12-LF) column quads (16-byte row segments) over all 2^LF rows: 16384
// residues per side and prime.  A thread holds 64 of them in registers --
// 16 rows x 4 adjacent columns -- and runs up to four levels on them per
// register stage; the four columns share every twiddle.  Between stages the
// CTA exchanges residues through shared memory, 16-byte words permuted
// within groups of 8 rows (conflict-free for every stage shape, checked
// exhaustively on the CPU).
//
// Results leave through a store phase: the last stage writes shared memory,
// and then each CTA of a two-CTA thread-block cluster (adjacent column
// groups) writes half of the rows of both CTAs' columns, reading the peer's
// words through distributed shared memory.  Every row segment written is
// then 32 bytes -- whole DRAM sectors -- where the CTA alone would write
// half sectors, which the memory system pays for as read-modify-writes.
//
//  * k_colfwd4<LF, M0, M1>: the forward levels of the row-vector and vector
//    trees (one job per side and prime); blockIdx.y selects the side (0: row
//    vector, read in source mode M0; 1: vector, mode M1).
//  * k_colinv4<LF, NP>: the recombination levels; with NP = 3 the three
//    primes of a polynomial product stay in shared memory and a CRT phase
//    writes the int64 coefficients (crt_store4).
//  * k_colinv4x3<LF>: the polynomial product's last pass, one prime per CTA
//    of a three-CTA cluster, the CRT gathered through distributed shared
//    memory.
//
// Inputs need 16-byte (uint32 sources) or 8-byte (uint16 sources) aligned
// pointers; the launchers check that and otherwise leave the pass to the
// one-column kernels of kernels_fast.cu.
#include <atomic>

#include "common.hpp"
#include "kernels_mod.hpp"
#include "prof.hpp"
#include "cluster.cuh"
#include "tile_dev.cuh"
#include "tma.cuh"

namespace fcirc {

namespace {

// log2 rows per thread in a register stage (a thread holds 4 x 2^LR
// residues); the CTA has 16384 / (4 2^LR) threads.
#ifndef FCIRC_C4_LR
#define FCIRC_C4_LR 4
#endif
constexpr int kC4LR = FCIRC_C4_LR;
constexpr int kC4Rows = 1 << kC4LR;
constexpr int kC4Threads = 4096 >> kC4LR;
// Largest cluster, log2: two CTAs (32-byte row segments, whole DRAM sectors)
// measured fastest; larger clusters pay more in cluster-wide waits than the
// wider segments save.
#ifndef FCIRC_C4_MAXLCL
#define FCIRC_C4_MAXLCL 1
#endif
// Whether the jobs of one group (the three primes of one side of a
// polynomial product) get one CTA each; sharing a CTA reads their common
// source from DRAM once instead of three times (64 vs 34 MB) at the same time.
#ifndef FCIRC_C4_SPLITJOBS
#define FCIRC_C4_SPLITJOBS 0
#endif
#ifndef FCIRC_C4_X3
#define FCIRC_C4_X3 1
#endif
#ifndef FCIRC_C4FWD_MINB
#define FCIRC_C4FWD_MINB 2
#endif
#ifndef FCIRC_C4INV_MINB
#define FCIRC_C4INV_MINB 2
#endif

template <int LF>
struct C4 {
    static constexpr int R = 1 << LF;
    static constexpr int LNQ = 12 - LF;            // log2 column quads per CTA
    static constexpr int WORDS = 1 << 14;          // residues per CTA and job
    static constexpr int NST = (LF + kC4LR - 1) / kC4LR;
    static constexpr int NL0 = LF - kC4LR * (NST - 1); // the first stage takes the remainder
    static constexpr int nl(int s) { return s == 0 ? NL0 : kC4LR; }
    static constexpr int d0(int s) { return s == 0 ? 0 : NL0 + kC4LR * (s - 1); }
    // Clusters of CL CTAs over adjacent column groups make every row segment
    // of the coalesced store phase 2^LCQ quads (16 2^LCQ bytes) wide.
    static constexpr int LCL0 = LNQ >= 3 ? 0 : 3 - LNQ;
    static constexpr int LCL = LCL0 < FCIRC_C4_MAXLCL ? LCL0 : FCIRC_C4_MAXLCL;
    static constexpr int CL = 1 << LCL;
    static constexpr int LCQ = LNQ + LCL;            // log2 quads per row segment
    static constexpr int LRW = LF - LCL;             // log2 rows per CTA in that phase
};

// Group slot h of thread tid in a stage running local levels D0 .. D0+NL-1:
// its column quad, first row and level-D0 block; its rows are row0 + i 2^LST.
template <int LF, int D0, int NL>
__device__ __forceinline__ void c4_group(int tid, int h, int &quad, int &row0, int &blk)
{
    constexpr int LST = LF - D0 - NL, LRB = LF - D0, LGQ = LF - NL;
    const int gg = tid + kC4Threads * h;
    quad = gg >> LGQ;
    const int g = gg & ((1 << LGQ) - 1);
    blk = g >> LST;
    row0 = (blk << LRB) + (g & ((1 << LST) - 1));
}

// Shared-memory word of (quad, row, column 0): 16-byte row segments, the row
// permuted inside aligned groups of 8 by bits LR..LR+2 of the row and by the
// quad (its low three bits rotated), so that the 8 lanes of one 128-bit
// access phase hit distinct banks in every stage and in the store phase.
template <int LF>
__device__ __forceinline__ int c4_off(int quad, int row)
{
    const int qs = ((quad & 3) << 1) | ((quad >> 2) & 1);
    return (quad << (LF + 2)) + ((row ^ ((row >> kC4LR) & 7) ^ qs) << 2);
}

// The stage accesses c4_off(quad, row0 + i 2^LST) split into a per-group
// base and terms that are compile-time constants in the unrolled loops (one
// XOR at most and an immediate offset per access).  The stage shapes have
// LST = 0, 4 or >= 7; the identities hold for every thread and group of
// every shape (checked on the CPU).
template <int LF, int LST>
struct C4Addr {
    static_assert(LST == 0 || LST == 4 || LST >= 7, "stage shape");
    int rb, kt;
    __device__ __forceinline__ C4Addr(int quad, int row0)
    {
        const int q = ((quad & 3) << 1) | ((quad >> 2) & 1);
        if constexpr (kC4LR != 4) {
            rb = quad;
            kt = row0;
        } else if constexpr (LST >= 7) {
            rb = (quad << (LF + 2)) + ((row0 ^ ((row0 >> kC4LR) & 7) ^ q) << 2);
            kt = 0;
        } else if constexpr (LST == 4) {
            rb = (quad << (LF + 2)) + ((row0 ^ q) << 2);
            kt = 0;
        } else {
            rb = (quad << (LF + 2)) + (row0 << 2);
            kt = ((row0 >> kC4LR) & 7) ^ q;
        }
    }
    __device__ __forceinline__ int operator()(int i) const
    {
        if constexpr (kC4LR != 4)
            return c4_off<LF>(rb, kt + (i << LST));
        else if constexpr (LST >= 7)
            return rb + (i << (LST + 2));
        else if constexpr (LST == 4)
            return (rb ^ ((i & 7) << 2)) + (i << 6);
        else
            return rb + ((i ^ kt) << 2);
    }
};

// Barrier halves over the CTAs that share row segments (the cluster, or the
// CTA itself when CL = 1).  Every thread alternates arrive and wait.
template <int CL>
__device__ __forceinline__ void grp_arrive()
{
    if constexpr (CL > 1) cl_arrive();
}
// The arrive after a store phase: its only cross-CTA accesses were peer
// shared-memory loads whose values its global stores consumed, so it needs no
// release (which would wait for those stores to drain).
template <int CL>
__device__ __forceinline__ void grp_arrive_done()
{
    if constexpr (CL > 1) cl_arrive_relaxed();
}
template <int CL>
__device__ __forceinline__ void grp_wait()
{
    if constexpr (CL > 1)
        cl_wait();
    else
        __syncthreads();
}

// Shared-memory window of the CTA holding quad cq of a row segment (that CTA
// keeps it as its quad cq & (2^LNQ - 1)); addresses are byte offsets in the
// cluster's shared window, or in the CTA's own when CL = 1.
template <int LF>
__device__ __forceinline__ uint32_t c4_seg_base(const uint32_t *smq, int cq)
{
    using Sh = C4<LF>;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(smq);
    if constexpr (Sh::CL == 1)
        return a;
    else
        return cl_map(a, (uint32_t)(cq >> Sh::LNQ));
}

template <int LF>
__device__ __forceinline__ uint4 c4_seg_ld(uint32_t seg_base, int cq, int row)
{
    using Sh = C4<LF>;
    const uint32_t a = seg_base + 4u * (uint32_t)c4_off<LF>(cq & ((1 << Sh::LNQ) - 1), row);
    if constexpr (Sh::CL == 1) {
        uint4 v;
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];\n"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "r"(a));
        return v;
    } else {
        return cl_ld4(a);
    }
}

// Coalesced store phase: this CTA writes rows [rank 2^LRW, (rank+1) 2^LRW)
// of all 2^LCQ quads of the cluster's columns, 2^LCQ lanes per row segment,
// reading each 16-byte word from the CTA that computed it.  A thread
// keeps one quad cq and steps through rows 256 / 2^LCQ apart.
template <int LF>
__device__ __forceinline__ void c4_store_phase(const uint32_t *smq, uint32_t *dst, uint32_t base0, int logS,
                                               int rank, int tid)
{
    using Sh = C4<LF>;
    constexpr int RSTEP = kC4Threads >> Sh::LCQ;
    const int cq = tid & ((1 << Sh::LCQ) - 1);
    const int row_t = (rank << Sh::LRW) + (tid >> Sh::LCQ);
    const uint32_t sb = c4_seg_base<LF>(smq, cq);
    uint4 *d = reinterpret_cast<uint4 *>(dst + base0 + ((uint32_t)cq << 2) + ((uint32_t)row_t << logS));
    const size_t dstep = (size_t)RSTEP << (logS - 2);   // in uint4
#pragma unroll
    for (int h = 0; h < kC4Rows / 8; ++h) {
        uint4 w[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = c4_seg_ld<LF>(sb, cq, row_t + RSTEP * (8 * h + k));
#pragma unroll
        for (int k = 0; k < 8; ++k) d[dstep * (8 * h + k)] = w[k];
    }
}

// Four residues of columns idx .. idx+3 (idx a multiple of 4) in source mode MODE.
template <int MODE>
__device__ __forceinline__ uint4 ld4_raw(const Src &s, uint32_t N, uint32_t idx)
{
    constexpr int KIND = MODE & 3;
    if constexpr (KIND == SRC_U32) {
        return __ldg(reinterpret_cast<const uint4 *>(static_cast<const uint32_t *>(s.ptr) + idx));
    } else if constexpr (KIND == SRC_U32_REV) {
        // a'[idx + c] = a[N - 1 - idx - c]: the word N - 4 - idx + (3 - c)
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(static_cast<const uint32_t *>(s.ptr) + N - 4 - idx));
        return make_uint4(w.w, w.z, w.y, w.x);
    } else if constexpr (KIND == SRC_U16_REV) {
        // a'[idx + c] = P[N - 1 - idx - c]: P[j0 + 3 - c] with j0 = N - 4 - idx
        const uint16_t *q = static_cast<const uint16_t *>(s.ptr);
        const uint32_t j0 = N - 4 - idx;
        if ((uint64_t)j0 + 4 <= s.len) {
            const uint2 w = __ldg(reinterpret_cast<const uint2 *>(q + j0));
            return make_uint4(w.y >> 16, w.y & 0xFFFFu, w.x >> 16, w.x & 0xFFFFu);
        }
        uint4 r;
        r.x = (uint64_t)j0 + 3 < s.len ? (uint32_t)__ldg(q + j0 + 3) : 0u;
        r.y = (uint64_t)j0 + 2 < s.len ? (uint32_t)__ldg(q + j0 + 2) : 0u;
        r.z = (uint64_t)j0 + 1 < s.len ? (uint32_t)__ldg(q + j0 + 1) : 0u;
        r.w = (uint64_t)j0 < s.len ? (uint32_t)__ldg(q + j0) : 0u;
        return r;
    } else {
        const uint16_t *q = static_cast<const uint16_t *>(s.ptr);
        if ((uint64_t)idx + 4 <= s.len) {
            const uint2 w = __ldg(reinterpret_cast<const uint2 *>(q + idx));
            return make_uint4(w.x & 0xFFFFu, w.x >> 16, w.y & 0xFFFFu, w.y >> 16);
        }
        uint4 r;
        r.x = (uint64_t)idx < s.len ? (uint32_t)__ldg(q + idx) : 0u;
        r.y = (uint64_t)idx + 1 < s.len ? (uint32_t)__ldg(q + idx + 1) : 0u;
        r.z = (uint64_t)idx + 2 < s.len ? (uint32_t)__ldg(q + idx + 2) : 0u;
        r.w = (uint64_t)idx + 3 < s.len ? (uint32_t)__ldg(q + idx + 3) : 0u;
        return r;
    }
}

// Raw-source cache of the forward pass.  The jobs of a CTA that read one
// uint16 source (the three primes of one side of a polynomial product) load
// it from global memory once: the first job packs the 16-bit values of every
// row it loads into shared memory behind the 64 KB exchange area, and the
// others read them back there.  A thread reads only the slots it wrote (slot
// k of thread t at word pair k * threads + t), so no barrier is needed, and the
// cache replaces what would otherwise be re-reads through an L1 that the
// scattered 8-byte row segments thrash.
template <int MODE>
struct C4Cache {
    static constexpr bool ON = (MODE & 3) == SRC_U16 || (MODE & 3) == SRC_U16_REV;
    static constexpr int ROWS = ((MODE >> 3) & 3) ? kC4Rows / 2 : kC4Rows;   // rows a thread loads
    static constexpr int BYTES = ON ? ROWS * kC4Threads * 8 : 0;
};
enum : int { C4_NOCACHE = 0, C4_FILL = 1, C4_USE = 2 };

// Twiddles of local level D of one group (slots 16 - 2^(D+1) .. 16 - 2^D of
// its 16-entry block in the group-ordered table), in 64/128-bit loads.
template <int D>
__device__ __forceinline__ void c4_level_tw(const Tw *g, Tw *t)
{
    if constexpr (D == 0) {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(g + 14));
        t[0] = Tw{w.x, w.y};
    } else {
        const uint4 *q = reinterpret_cast<const uint4 *>(g + 16 - (2 << D));
#pragma unroll
        for (int k = 0; k < (1 << (D - 1)); ++k) {
            const uint4 w = __ldg(q + k);
            t[2 * k] = Tw{w.x, w.y};
            t[2 * k + 1] = Tw{w.z, w.w};
        }
    }
}

// Where a group's twiddles come from.  TwGroup: the group-ordered table,
// 16 consecutive entries per group block (128-bit loads).  TwSlots: the
// copy of a stage ordered by slot pair (ColFwdJob::gtwl), entry
// 2 (q stride + group block) + (slot & 1) for q = slot / 2 -- for the stage in
// which every thread has a group block of its own, so that a warp's 128-bit
// loads of one slot pair are contiguous.
struct TwGroup {
    const Tw *g;
    template <int D>
    __device__ __forceinline__ void level(Tw *t) const { c4_level_tw<D>(g, t); }
};
struct TwSlots {
    const Tw *g;          // the group block's first entry (2 gb)
    uint32_t stride;      // the stage's number of group blocks
    template <int D>
    __device__ __forceinline__ void level(Tw *t) const
    {
        // slot pair q of group block gb at entry 2 (q stride + gb)
        constexpr int Q0 = 8 - (1 << D);
        if constexpr (D == 0) {
            const uint2 w = __ldg(reinterpret_cast<const uint2 *>(g + 2 * Q0 * stride));
            t[0] = Tw{w.x, w.y};
        } else {
#pragma unroll
            for (int k = 0; k < (1 << (D - 1)); ++k) {
                const uint4 w = __ldg(reinterpret_cast<const uint4 *>(g + 2 * (uint32_t)(Q0 + k) * stride));
                t[2 * k] = Tw{w.x, w.y};
                t[2 * k + 1] = Tw{w.z, w.w};
            }
        }
    }
};

// Forward levels D .. NL-1 of one group held as v[4 i + c] (row i, column
// c); `cur` holds level D's twiddles, level D+1's are loaded before level D
// is computed.
template <int NL, int D, bool VEC, class TA>
__device__ __forceinline__ void c4_fwd(uint32_t *v, const TA &g, const Tw *cur, uint32_t p, uint32_t p2)
{
    if constexpr (D < NL) {
        Tw nxt[(D + 1 < NL) ? (2 << D) : 1];
        if constexpr (D + 1 < NL) g.template level<D + 1>(nxt);
        constexpr int h = (1 << NL) >> (D + 1);
#pragma unroll
        for (int j = 0; j < (1 << D); ++j)
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const int lo = (j << (NL - D)) + i;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    // the select form of the reduction measured faster here
                    if (VEC)
                        bfly_vec<false>(v[4 * lo + c], v[4 * (lo + h) + c], cur[j], p, p2);
                    else
                        bfly_row<false>(v[4 * lo + c], v[4 * (lo + h) + c], cur[j], p, p2);
                }
            }
        c4_fwd<NL, D + 1, VEC, TA>(v, g, nxt, p, p2);
    }
}

// Recombination levels D .. 0 of one group (inverse twiddles), with the
// same one-level look-ahead of twiddle loads.
template <int NL, int D, class TA>
__device__ __forceinline__ void c4_rec(uint32_t *v, const TA &g, const Tw *cur, uint32_t p, uint32_t p2)
{
    if constexpr (D >= 0) {
        Tw nxt[D > 0 ? (1 << (D - 1)) : 1];
        if constexpr (D > 0) g.template level<D - 1>(nxt);
        constexpr int h = (1 << NL) >> (D + 1);
#pragma unroll
        for (int j = 0; j < (1 << D); ++j)
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const int lo = (j << (NL - D)) + i;
#pragma unroll
                for (int c = 0; c < 4; ++c) bfly_rec(v[4 * lo + c], v[4 * (lo + h) + c], cur[j], p, p2);
            }
        c4_rec<NL, D - 1, TA>(v, g, nxt, p, p2);
    }
}

// One 32-byte sector: eight consecutive words of the tile-pair interleaved
// layout (a column quad of two adjacent rows), from or to v[0..8).
__device__ __forceinline__ void st_sector(uint32_t *d, const uint32_t *v)
{
    asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};\n" ::"l"(d),
                 "l"((uint64_t)v[0] | ((uint64_t)v[1] << 32)), "l"((uint64_t)v[2] | ((uint64_t)v[3] << 32)),
                 "l"((uint64_t)v[4] | ((uint64_t)v[5] << 32)), "l"((uint64_t)v[6] | ((uint64_t)v[7] << 32))
                 : "memory");
}

__device__ __forceinline__ void ld_sector(const uint32_t *s, uint32_t *v)
{
    uint64_t w0, w1, w2, w3;
    asm volatile("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];\n"
                 : "=l"(w0), "=l"(w1), "=l"(w2), "=l"(w3)
                 : "l"(s));
    v[0] = (uint32_t)w0; v[1] = (uint32_t)(w0 >> 32);
    v[2] = (uint32_t)w1; v[3] = (uint32_t)(w1 >> 32);
    v[4] = (uint32_t)w2; v[5] = (uint32_t)(w2 >> 32);
    v[6] = (uint32_t)w3; v[7] = (uint32_t)(w3 >> 32);
}

__device__ __forceinline__ void put4(uint32_t *v, uint4 w)
{
    v[0] = w.x;
    v[1] = w.y;
    v[2] = w.z;
    v[3] = w.w;
}

__device__ __forceinline__ uint4 get4(const uint32_t *v) { return make_uint4(v[0], v[1], v[2], v[3]); }

// Whether the interleaved output of this pass leaves through TMA tensor
// stores: 12 levels, maps made (fwd_tma_maps), and shared memory on a
// 128-byte boundary (the boxes).  The same for every thread.
template <int LF, bool ILV>
__device__ __forceinline__ bool c4_tma_st(const ColFwdParams &P, const uint32_t *sm)
{
    if constexpr (ILV && LF == 12)
        return P.tma_st && (sm_u32(sm) & 127u) == 0;
    else
        return false;
}

// ILV: the pass writes the tile-pair interleaved layout; its last stage
// stores straight from registers (no shared-memory write, no store phase),
// or, for 12 levels, writes the CTA's 64 KB of shared memory as eight TMA
// boxes and leaves the stores to the TMA unit while the next job starts
// (tm: the job's tensor map).
template <int LF, int S, int MODE, bool VEC, bool ILV>
__device__ __forceinline__ void c4fwd_stage(const ColFwdJob &J, const ColFwdParams &P, uint32_t *sm,
                                            uint32_t base, uint32_t pb, int logS, int tid, bool wait_first,
                                            int cache = C4_NOCACHE, const CUtensorMap *tm = nullptr)
{
    using Sh = C4<LF>;
    constexpr int NL = Sh::nl(S), D0 = Sh::d0(S);
    constexpr int M = 1 << NL, B = kC4Rows >> NL, LST = LF - D0 - NL;
    constexpr bool FIRST = (S == 0);
    constexpr int half = FIRST ? ((MODE >> 3) & 3) : 0;
    const uint32_t p = J.p, p2 = 2 * J.p;
    const Tw *gt = J.gtw + P.stage_off[S];
    uint32_t v[4 * kC4Rows];
    // every load of the stage is issued before any arithmetic
#pragma unroll
    for (int hb = 0; hb < B; ++hb) {
        int quad, row0, blk;
        c4_group<LF, D0, NL>(tid, hb, quad, row0, blk);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            if ((half == 1 && i < M / 2) || (half == 2 && i >= M / 2)) continue;
            const int row = row0 + (i << LST);
            uint4 w;
            if constexpr (FIRST && C4Cache<MODE>::ON) {
                // cache slot: the thread's k-th loaded row
                constexpr int half_m = M / 2;
                const int k = half ? hb * half_m + (i % half_m) : hb * M + i;
                uint2 *rc = reinterpret_cast<uint2 *>(sm + C4<LF>::WORDS) + k * kC4Threads + tid;
                if (cache == C4_USE) {
                    const uint2 r = *rc;
                    w = make_uint4(r.x & 0xFFFFu, r.x >> 16, r.y & 0xFFFFu, r.y >> 16);
                } else {
                    w = ld4_raw<MODE>(J.src, P.N, base + ((uint32_t)quad << 2) + ((uint32_t)row << logS));
                    if (cache == C4_FILL) *rc = make_uint2(w.x | (w.y << 16), w.z | (w.w << 16));
                }
            } else if constexpr (FIRST)
                w = ld4_raw<MODE>(J.src, P.N, base + ((uint32_t)quad << 2) + ((uint32_t)row << logS));
            else
                w = *reinterpret_cast<const uint4 *>(sm + C4Addr<LF, LST>(quad, row0)(i));
            put4(v + 4 * (hb * M + i), w);
        }
    }
#pragma unroll
    for (int hb = 0; hb < B; ++hb) {
        int quad, row0, blk;
        c4_group<LF, D0, NL>(tid, hb, quad, row0, blk);
        const uint32_t gb = (pb << D0) + blk;
        // the last stage gives every thread a group block of its own: its
        // twiddles come from the slot-major copy
        const auto g = [&] {
            if constexpr (S == Sh::NST - 1)
                return TwSlots{J.gtwl + 2 * gb, 1u << (P.l0 + D0)};
            else
                return TwGroup{gt + (gb << 4)};
        }();
        constexpr int DS = (FIRST && half != 0) ? 1 : 0;
        Tw t0[1 << DS];
        g.template level<DS>(t0);
        uint32_t *vg = v + 4 * hb * M;
        if constexpr (FIRST) {
#pragma unroll
            for (int i = 0; i < M; ++i) {
                if ((half == 1 && i < M / 2) || (half == 2 && i >= M / 2)) continue;
#pragma unroll
                for (int c = 0; c < 4; ++c) vg[4 * i + c] = ld_scale<MODE>(vg[4 * i + c], J.src, p);
            }
            if constexpr (half == 1) {
                // row vector zero in rows < R/2; level 0 has s = 1: (0 + hi, 0 - hi)
#pragma unroll
                for (int i = M / 2; i < M; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint32_t x = vg[4 * i + c];
                        vg[4 * (i - M / 2) + c] = x;
                        vg[4 * i + c] = p2 - x;
                    }
            } else if constexpr (half == 2) {
                // vector zero in rows >= R/2; level 0 has s = 1: (lo, lo)
#pragma unroll
                for (int i = 0; i < M / 2; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) vg[4 * (i + M / 2) + c] = vg[4 * i + c];
            }
        }
        c4_fwd<NL, DS, VEC>(vg, g, t0, p, p2);
    }
    if constexpr (ILV && S == Sh::NST - 1) {
        // the last stage holds 16 consecutive rows (tiles) of one column
        // quad; row pair k is one sector of the interleaved layout, and the
        // pass has 2^12 columns (col4_fwd_ilv_ok), so rows are 2^12 apart
        static_assert(B == 1 && M == 16 && LST == 0, "last stage shape");
        int quad, row0, blk;
        c4_group<LF, D0, NL>(tid, 0, quad, row0, blk);
        if constexpr (LF == 12) {
            // (the CTA's 2^11 tile pairs inside the map's N / 8192)
            if (c4_tma_st<LF, ILV>(P, sm) && (base >> 16) + 256u <= (P.N >> 16)) {
                // every thread has read this stage's inputs from shared memory
                __syncthreads();
                // the thread's row pair 8 tid + k (its rows row0 = 16 tid ..
                // row0 + 15, one quad per CTA) is sector tid of box k: byte
                // 8192 k + 32 tid + 16 (row parity) of the 64 KB area
                static_assert(Sh::LNQ == 0, "one column quad per CTA");
#pragma unroll
                for (int k = 0; k < 8; ++k)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        *reinterpret_cast<uint4 *>(sm + 2048 * k + 8 * tid + 4 * h) = get4(v + 8 * k + 4 * h);
                fence_async_shared();
                __syncthreads();
                if (tid == 0) {
                    // the CTA's column quad, and its first tile pair (base is
                    // the natural index of its first element, rows of 4096) as
                    // 8 t0: 2^11 tile pairs per CTA
                    const int q = (int)((base & 4095u) >> 2), t0 = (int)(base >> 16);
#pragma unroll
                    for (int k = 0; k < 8; ++k) tma_store_5d(tm, sm + 2048 * k, 0, 0, q, k, t0);
                    tma_store_commit();
                }
                return;
            }
        }
        uint32_t *d = J.dst + ilv_pos(base + ((uint32_t)quad << 2) + ((uint32_t)row0 << 12));
#pragma unroll
        for (int k = 0; k < 8; ++k) st_sector(d + 8192 * k, v + 8 * k);
        return;
    }
    // the previous job's last stage (or store phase) may still read this
    // CTA's shared memory
    if (FIRST && wait_first) {
        if constexpr (ILV) {
            // and the previous job's TMA stores have read it
            if (tid == 0 && c4_tma_st<LF, ILV>(P, sm)) tma_store_wait_read();
            __syncthreads();
        } else {
            grp_wait<Sh::CL>();
        }
    }
#pragma unroll
    for (int hb = 0; hb < B; ++hb) {
        int quad, row0, blk;
        c4_group<LF, D0, NL>(tid, hb, quad, row0, blk);
        const C4Addr<LF, LST> ad(quad, row0);
#pragma unroll
        for (int i = 0; i < M; ++i) *reinterpret_cast<uint4 *>(sm + ad(i)) = get4(v + 4 * (hb * M + i));
    }
}

// The barrier between register stages S and S + 1 of a pass (either
// direction).  The last two stages exchange residues only between threads
// of one warp (every slot is owned by the same warp in both; checked on the
// CPU for LF = 8 .. 12), so a warp sync orders them; earlier exchanges cross
// warps.
template <int LF, int S>
__device__ __forceinline__ void c4_stage_sync()
{
    if constexpr (S == C4<LF>::NST - 2)
        __syncwarp();
    else
        __syncthreads();
}

template <int LF, int MODE, bool VEC, bool ILV>
__device__ __forceinline__ void c4fwd_jobs(const ColFwdParams &P, uint32_t *sm, int j0, uint32_t base,
                                           uint32_t pb, int logS, int tid)
{
    using Sh = C4<LF>;
    const int rank = (!ILV && Sh::CL > 1) ? (int)cl_rank() : 0;
    const uint32_t base0 = base - ((uint32_t)rank << (2 + Sh::LNQ));
    const bool cached = C4Cache<MODE>::ON && P.share_src && P.jobs_per_cta > 1;
#pragma unroll 1
    for (int jj = 0; jj < P.jobs_per_cta; ++jj) {
        const ColFwdJob &J = P.job[j0 + jj];
        const CUtensorMap *tm = &P.tmap[j0 + jj];
        c4fwd_stage<LF, 0, MODE, VEC, ILV>(J, P, sm, base, pb, logS, tid, jj > 0,
                                           cached ? (jj == 0 ? C4_FILL : C4_USE) : C4_NOCACHE, tm);
        if constexpr (Sh::NST > 1) {
            c4_stage_sync<LF, 0>();
            c4fwd_stage<LF, 1, MODE, VEC, ILV>(J, P, sm, base, pb, logS, tid, false, C4_NOCACHE, tm);
        }
        if constexpr (Sh::NST > 2) {
            c4_stage_sync<LF, 1>();
            c4fwd_stage<LF, 2, MODE, VEC, ILV>(J, P, sm, base, pb, logS, tid, false, C4_NOCACHE, tm);
        }
        if constexpr (Sh::NST > 3) {
            c4_stage_sync<LF, 2>();
            c4fwd_stage<LF, 3, MODE, VEC, ILV>(J, P, sm, base, pb, logS, tid, false, C4_NOCACHE, tm);
        }
        if constexpr (!ILV) {
            grp_arrive<Sh::CL>();
            grp_wait<Sh::CL>();
            c4_store_phase<LF>(sm, J.dst, base0, logS, rank, tid);
            grp_arrive_done<Sh::CL>();
        }
    }
    if constexpr (!ILV) grp_wait<Sh::CL>();   // no CTA leaves while a peer still reads its shared memory
    // nor while its own TMA stores still read it
    if (tid == 0 && c4_tma_st<LF, ILV>(P, sm)) tma_store_wait_read();
}

// CTA origin: node pb of level l0 and the CTA's first column
template <int LF>
__device__ __forceinline__ void c4_origin(int logn, int l0, int l1, uint32_t &pb, uint32_t &base, int &logS,
                                          uint32_t cta = blockIdx.x)
{
    logS = logn - l1;
    const int cg_bits = logS - 2 - C4<LF>::LNQ;
    pb = cta >> cg_bits;
    const uint32_t cg = cta & ((1u << cg_bits) - 1);
    base = (pb << (logn - l0)) + (cg << (2 + C4<LF>::LNQ));
}

template <int LF, int M0, int M1, bool ILV>
__global__ void __cluster_dims__(ILV ? 1 : C4<LF>::CL, 1, 1) __launch_bounds__(kC4Threads, FCIRC_C4FWD_MINB)
    k_colfwd4(const __grid_constant__ ColFwdParams P)
{
    extern __shared__ __align__(128) uint32_t sm[];
    uint32_t pb, base;
    int logS;
    c4_origin<LF>(P.logn, P.l0, P.l1, pb, base, logS);
    const int j0 = blockIdx.y * P.jobs_per_cta;
    // job groups below vec_group0 are the row-vector side, the rest the
    // vector side
    if ((int)blockIdx.y < P.vec_group0)
        c4fwd_jobs<LF, M0, false, ILV>(P, sm, j0, base, pb, logS, threadIdx.x);
    else
        c4fwd_jobs<LF, M1, true, ILV>(P, sm, j0, base, pb, logS, threadIdx.x);
}

// Stage S of the recombination for one prime's job J, its residues in smq.
// ILV: the pass reads the tile-pair interleaved layout; its first stage
// loads whole 32-byte sectors (a column quad of two adjacent rows).
template <int LF, int S, bool ILV>
__device__ __forceinline__ void c4inv_job(const ColInvParams &P, const ColInvJob &J, uint32_t *smq, uint32_t base,
                                          uint32_t pb, int logS, int tid)
{
    using Sh = C4<LF>;
    constexpr int NL = Sh::nl(S), D0 = Sh::d0(S);
    constexpr int M = 1 << NL, B = kC4Rows >> NL, LST = LF - D0 - NL;
    constexpr bool FIRST = (S == Sh::NST - 1), LAST = (S == 0);
    {
        const uint32_t p = J.p, p2 = 2 * J.p;
        const Tw *gt = J.gitw + P.stage_off[S];
        uint32_t v[4 * kC4Rows];
        if constexpr (FIRST && ILV) {
            // 16 consecutive rows (tiles) of one quad, 2^12 columns
            // (col4_inv_ilv_ok): eight sectors of row pairs
            static_assert(B == 1 && M == 16 && LST == 0, "first stage shape");
            int quad, row0, blk;
            c4_group<LF, D0, NL>(tid, 0, quad, row0, blk);
            const uint32_t *src = J.src + ilv_pos(base + ((uint32_t)quad << 2) + ((uint32_t)row0 << 12));
#pragma unroll
            for (int k = 0; k < 8; ++k) ld_sector(src + 8192 * k, v + 8 * k);
        } else {
#pragma unroll
            for (int hb = 0; hb < B; ++hb) {
                int quad, row0, blk;
                c4_group<LF, D0, NL>(tid, hb, quad, row0, blk);
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    const int row = row0 + (i << LST);
                    uint4 w;
                    if constexpr (FIRST)
                        w = __ldg(reinterpret_cast<const uint4 *>(J.src + base + ((uint32_t)quad << 2) +
                                                                  ((uint32_t)row << logS)));
                    else
                        w = *reinterpret_cast<const uint4 *>(smq + C4Addr<LF, LST>(quad, row0)(i));
                    put4(v + 4 * (hb * M + i), w);
                }
            }
        }
#pragma unroll
        for (int hb = 0; hb < B; ++hb) {
            int quad, row0, blk;
            c4_group<LF, D0, NL>(tid, hb, quad, row0, blk);
            const uint32_t gb = (pb << D0) + blk;
            // the first stage gives every thread a group block of its own:
            // its twiddles come from the slot-major copy
            const auto g = [&] {
                if constexpr (FIRST)
                    return TwSlots{J.gitwl + 2 * gb, 1u << (P.l0 + D0)};
                else
                    return TwGroup{gt + (gb << 4)};
            }();
            Tw tl[1 << (NL - 1)];
            g.template level<NL - 1>(tl);
            c4_rec<NL, NL - 1>(v + 4 * hb * M, g, tl, p, p2);
        }
        // the last stage leaves canonical residues unless the output stays lazy
        const bool canon = LAST && P.epi != EPI_LAZY;
#pragma unroll
        for (int hb = 0; hb < B; ++hb) {
            int quad, row0, blk;
            c4_group<LF, D0, NL>(tid, hb, quad, row0, blk);
            const C4Addr<LF, LST> ad(quad, row0);
#pragma unroll
            for (int i = 0; i < M; ++i) {
                uint32_t *e = v + 4 * (hb * M + i);
                const uint4 w = canon ? make_uint4(reduce_once(e[0], p), reduce_once(e[1], p),
                                                   reduce_once(e[2], p), reduce_once(e[3], p))
                                      : get4(e);
                *reinterpret_cast<uint4 *>(smq + ad(i)) = w;
            }
        }
    }
}

template <int LF, int NP, int S, bool ILV>
__device__ __forceinline__ void c4inv_stage(const ColInvParams &P, uint32_t *sm, uint32_t base, uint32_t pb,
                                            int logS, int tid)
{
#pragma unroll 1
    for (int q = 0; q < NP; ++q) c4inv_job<LF, S, ILV>(P, P.job[q], sm + q * C4<LF>::WORDS, base, pb, logS, tid);
}

// The CRT of one quad (circulant entries idx .. idx+3, the three primes'
// canonical residues in r1, r2, r3) into the int64 coefficients.  EPI_CRT:
// entry k is coefficient k, and an in-range quad leaves as one 32-byte store
// (a whole DRAM sector) when the output is 32-byte aligned.  EPI_CRT_ROT:
// coefficient k is circulant entry k + 1, four 8-byte stores.
__device__ __forceinline__ void crt_store4(const ColInvParams &P, uint32_t idx, uint4 r1, uint4 r2, uint4 r3)
{
    const uint64_t e0 = crt3(r1.x, r2.x, r3.x, P.crt), e1 = crt3(r1.y, r2.y, r3.y, P.crt);
    const uint64_t e2 = crt3(r1.z, r2.z, r3.z, P.crt), e3 = crt3(r1.w, r2.w, r3.w, P.crt);
    if (P.epi == EPI_CRT) {
        if ((reinterpret_cast<uintptr_t>(P.dst64) & 31) == 0 && (uint64_t)idx + 3 < P.nout) {
            asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};\n" ::"l"(P.dst64 + idx), "l"(e0), "l"(e1),
                         "l"(e2), "l"(e3)
                         : "memory");
        } else {
            if (idx < P.nout) P.dst64[idx] = e0;
            if (idx + 1 < P.nout) P.dst64[idx + 1] = e1;
            if (idx + 2 < P.nout) P.dst64[idx + 2] = e2;
            if (idx + 3 < P.nout) P.dst64[idx + 3] = e3;
        }
    } else {
        const uint32_t d0 = (idx + P.N - 1) & (P.N - 1);   // coefficient k is circulant entry k + 1
        if (d0 < P.nout) P.dst64[d0] = e0;
        if (idx < P.nout) P.dst64[idx] = e1;
        if (idx + 1 < P.nout) P.dst64[idx + 1] = e2;
        if (idx + 2 < P.nout) P.dst64[idx + 2] = e3;
    }
}

// Whether the quad of circulant entries idx .. idx+3 writes any coefficient.
// The CRT loops load a quad's residues from the peers only when it does, so
// every such load feeds a store before the closing relaxed arrive.
__device__ __forceinline__ bool crt_quad_needed(const ColInvParams &P, uint32_t idx)
{
    if (idx < P.nout) return true;
    return P.epi == EPI_CRT_ROT && ((idx + P.N - 1) & (P.N - 1)) < P.nout;
}

// CRT phase of the polynomial product: the rows of the store phase, the three
// primes' canonical residues from the CTA that computed them, Garner's CRT,
// and the int64 coefficients (crt_store4).
template <int LF>
__device__ __forceinline__ void c4_crt_phase(const ColInvParams &P, const uint32_t *sm, uint32_t base0, int logS,
                                             int rank, int tid)
{
    using Sh = C4<LF>;
    constexpr int RSTEP = kC4Threads >> Sh::LCQ;
    const int cq = tid & ((1 << Sh::LCQ) - 1);
    const int row_t = (rank << Sh::LRW) + (tid >> Sh::LCQ);
    const uint32_t sb = c4_seg_base<LF>(sm, cq);
    constexpr uint32_t PB = 4u * Sh::WORDS;   // bytes per prime region
#pragma unroll 2
    for (int k = 0; k < kC4Rows; ++k) {
        const int row = row_t + RSTEP * k;
        const uint32_t idx = base0 + ((uint32_t)cq << 2) + ((uint32_t)row << logS);
        if (!crt_quad_needed(P, idx)) continue;
        const uint4 r1 = c4_seg_ld<LF>(sb, cq, row);
        const uint4 r2 = c4_seg_ld<LF>(sb + PB, cq, row);
        const uint4 r3 = c4_seg_ld<LF>(sb + 2 * PB, cq, row);
        crt_store4(P, idx, r1, r2, r3);
    }
}

template <int LF, int NP, bool ILV>
__global__ void __cluster_dims__(C4<LF>::CL, 1, 1) __launch_bounds__(kC4Threads, NP == 1 ? FCIRC_C4INV_MINB : 1)
    k_colinv4(const __grid_constant__ ColInvParams P)
{
    extern __shared__ __align__(16) uint32_t sm[];
    using Sh = C4<LF>;
    uint32_t pb, base;
    int logS;
    c4_origin<LF>(P.logn, P.l0, P.l1, pb, base, logS);
    const int tid = threadIdx.x;
    const int rank = Sh::CL > 1 ? (int)cl_rank() : 0;
    const uint32_t base0 = base - ((uint32_t)rank << (2 + Sh::LNQ));
    if constexpr (Sh::NST > 3) {
        c4inv_stage<LF, NP, 3, ILV>(P, sm, base, pb, logS, tid);
        c4_stage_sync<LF, 2>();
    }
    if constexpr (Sh::NST > 2) {
        c4inv_stage<LF, NP, 2, ILV>(P, sm, base, pb, logS, tid);
        c4_stage_sync<LF, 1>();
    }
    if constexpr (Sh::NST > 1) {
        c4inv_stage<LF, NP, 1, ILV>(P, sm, base, pb, logS, tid);
        c4_stage_sync<LF, 0>();
    }
    c4inv_stage<LF, NP, 0, ILV>(P, sm, base, pb, logS, tid);
    grp_arrive<Sh::CL>();
    grp_wait<Sh::CL>();
    if (NP == 3 && epi_crt(P.epi)) {
        c4_crt_phase<LF>(P, sm, base0, logS, rank, tid);
    } else {
#pragma unroll 1
        for (int q = 0; q < NP; ++q) c4_store_phase<LF>(sm + q * Sh::WORDS, P.job[q].dst, base0, logS, rank, tid);
    }
    // no CTA leaves while a peer still reads its shared memory
    grp_arrive_done<Sh::CL>();
    grp_wait<Sh::CL>();
}

// Polynomial product, three primes: a cluster of three CTAs per column
// group, CTA q running prime q's recombination levels in its own 64 KB of
// shared memory (so two clusters' CTAs share an SM and overlap their memory
// and arithmetic phases); then each CTA takes a third of the group's rows,
// gathers the three canonical residues through distributed shared memory,
// and writes the CRT results (crt_store4).
template <int LF, bool ILV>
__global__ void __cluster_dims__(3, 1, 1) __launch_bounds__(kC4Threads, 2)
    k_colinv4x3(const __grid_constant__ ColInvParams P)
{
    extern __shared__ __align__(16) uint32_t sm[];
    using Sh = C4<LF>;
    const int q = (int)cl_rank();
    uint32_t pb, base;
    int logS;
    c4_origin<LF>(P.logn, P.l0, P.l1, pb, base, logS, blockIdx.x / 3);
    const int tid = threadIdx.x;
    const ColInvJob &J = P.job[q];
    if constexpr (Sh::NST > 3) {
        c4inv_job<LF, 3, ILV>(P, J, sm, base, pb, logS, tid);
        c4_stage_sync<LF, 2>();
    }
    if constexpr (Sh::NST > 2) {
        c4inv_job<LF, 2, ILV>(P, J, sm, base, pb, logS, tid);
        c4_stage_sync<LF, 1>();
    }
    if constexpr (Sh::NST > 1) {
        c4inv_job<LF, 1, ILV>(P, J, sm, base, pb, logS, tid);
        c4_stage_sync<LF, 0>();
    }
    c4inv_job<LF, 0, ILV>(P, J, sm, base, pb, logS, tid);
    cl_arrive();
    cl_wait();   // all three primes' residues are in place
    constexpr int W = 1 << 12;                   // 16-byte words (quad, row) per CTA
    constexpr int W3 = (W + 2) / 3;
    const int w0 = q * W3, w1 = (q + 1) * W3 < W ? (q + 1) * W3 : W;
    const uint32_t own = smem_addr(sm);
    const uint32_t s1 = cl_map(own, 0), s2 = cl_map(own, 1), s3 = cl_map(own, 2);
#pragma unroll 4
    for (int w = w0 + tid; w < w1; w += kC4Threads) {
        const int quad = w & ((1 << Sh::LNQ) - 1), row = w >> Sh::LNQ;
        const uint32_t idx = base + ((uint32_t)quad << 2) + ((uint32_t)row << logS);
        if (!crt_quad_needed(P, idx)) continue;
        const uint32_t off = 4u * (uint32_t)c4_off<LF>(quad, row);
        const uint4 r1 = cl_ld4(s1 + off), r2 = cl_ld4(s2 + off), r3 = cl_ld4(s3 + off);
        crt_store4(P, idx, r1, r2, r3);
    }
    // no CTA leaves while a peer still reads its shared memory (every peer
    // load above fed a store: crt_quad_needed)
    cl_arrive_relaxed();
    cl_wait();
}

template <class K>
int c4_smem(K kernel, int bytes, std::atomic<unsigned> &mask)
{
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    const unsigned bit = 1u << (dev & 31);
    if (mask.load() & bit) return FCIRC_OK;
    FCIRC_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    mask.fetch_or(bit);
    return FCIRC_OK;
}

int c4_mode(const Src &s, int half) { return s.kind | (s.scaled ? 4 : 0) | (half << 3); }

bool aligned(const void *ptr, unsigned a) { return (reinterpret_cast<uintptr_t>(ptr) & (a - 1)) == 0; }

bool src_aligned(const Src &s)
{
    return (s.kind == SRC_U32 || s.kind == SRC_U32_REV) ? aligned(s.ptr, 16) : aligned(s.ptr, 8);
}

template <int LF, int M0, int M1, bool ILV>
int launch_c4fwd_m(const ColFwdParams &P, int nctay, cudaStream_t s)
{
    static std::atomic<unsigned> mask{0};
    constexpr int cache_max = C4Cache<M0>::BYTES > C4Cache<M1>::BYTES ? C4Cache<M0>::BYTES : C4Cache<M1>::BYTES;
    FCIRC_TRY(c4_smem(k_colfwd4<LF, M0, M1, ILV>, C4<LF>::WORDS * 4 + cache_max, mask));
    const uint64_t ncta = (uint64_t)1 << (P.l0 + (P.logn - P.l1) - 2 - C4<LF>::LNQ);
    // optionally one job per CTA (more, shorter CTAs)
    ColFwdParams P1 = P;
    // the raw-source cache serves job groups whose jobs all read one source
    P1.share_src = 1;
    for (int k = 0; k < nctay * P.jobs_per_cta; ++k) {
        const Src &a = P.job[k].src, &b = P.job[(k / P.jobs_per_cta) * P.jobs_per_cta].src;
        if (a.ptr != b.ptr || a.len != b.len || a.kind != b.kind) P1.share_src = 0;
    }
    const int smem = C4<LF>::WORDS * 4 + (P1.share_src && P.jobs_per_cta > 1 ? cache_max : 0);
    int ny = nctay;
    if (FCIRC_C4_SPLITJOBS) {
        ny = nctay * P.jobs_per_cta;
        P1.vec_group0 = P.vec_group0 * P.jobs_per_cta;
        P1.jobs_per_cta = 1;
    }
    dim3 grid((unsigned)ncta, ny);
    ProfScope ps("k_colfwd4", s);
    k_colfwd4<LF, M0, M1, ILV><<<grid, kC4Threads, smem, s>>>(P1);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

template <int LF, bool ILV>
int launch_c4fwd_lf(const ColFwdParams &P, int nctay, int m0, int m1, cudaStream_t s)
{
    if (m0 == MODE_U32_S && m1 == MODE_U32) return launch_c4fwd_m<LF, MODE_U32_S, MODE_U32, ILV>(P, nctay, s);
    if (m0 == MODE_U32REV_S && m1 == MODE_U32) return launch_c4fwd_m<LF, MODE_U32REV_S, MODE_U32, ILV>(P, nctay, s);
    if (m0 == MODE_U32 && m1 == MODE_U32) return launch_c4fwd_m<LF, MODE_U32, MODE_U32, ILV>(P, nctay, s);
    if (m0 == MODE_REV_S_H && m1 == MODE_U16_H) return launch_c4fwd_m<LF, MODE_REV_S_H, MODE_U16_H, ILV>(P, nctay, s);
    if (m0 == MODE_REV_S && m1 == MODE_U16) return launch_c4fwd_m<LF, MODE_REV_S, MODE_U16, ILV>(P, nctay, s);
    return fail(FCIRC_EINVAL, "column pass: unsupported source modes %d/%d", m0, m1);
}

template <int LF>
int launch_c4fwd_lf(const ColFwdParams &P, int nctay, int m0, int m1, cudaStream_t s)
{
    return P.ilv ? launch_c4fwd_lf<LF, true>(P, nctay, m0, m1, s) : launch_c4fwd_lf<LF, false>(P, nctay, m0, m1, s);
}

template <int LF, int NP, bool ILV>
int launch_c4inv_lf_(const ColInvParams &P, cudaStream_t s)
{
    static std::atomic<unsigned> mask{0};
    const int smem = NP * C4<LF>::WORDS * 4;
    FCIRC_TRY(c4_smem(k_colinv4<LF, NP, ILV>, smem, mask));
    const uint64_t ncta = (uint64_t)1 << (P.l0 + (P.logn - P.l1) - 2 - C4<LF>::LNQ);
    ProfScope ps("k_colinv4", s);
    k_colinv4<LF, NP, ILV><<<(unsigned)ncta, kC4Threads, smem, s>>>(P);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

template <int LF, int NP>
int launch_c4inv_lf(const ColInvParams &P, cudaStream_t s)
{
    return P.ilv ? launch_c4inv_lf_<LF, NP, true>(P, s) : launch_c4inv_lf_<LF, NP, false>(P, s);
}

template <int LF, bool ILV>
int launch_c4inv_x3_(const ColInvParams &P, cudaStream_t s)
{
    static std::atomic<unsigned> mask{0};
    const int smem = C4<LF>::WORDS * 4;
    FCIRC_TRY(c4_smem(k_colinv4x3<LF, ILV>, smem, mask));
    const uint64_t ncta = (uint64_t)3 << (P.l0 + (P.logn - P.l1) - 2 - C4<LF>::LNQ);
    ProfScope ps("k_colinv4x3", s);
    k_colinv4x3<LF, ILV><<<(unsigned)ncta, kC4Threads, smem, s>>>(P);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

template <int LF>
int launch_c4inv_x3(const ColInvParams &P, cudaStream_t s)
{
    return P.ilv ? launch_c4inv_x3_<LF, true>(P, s) : launch_c4inv_x3_<LF, false>(P, s);
}

}  // namespace

// The pass can run here: LF in 8..12, enough columns for one cluster's
// quads, and 16-byte (uint32) / 8-byte (uint16) aligned sources and
// destinations.
bool col4_fwd_ok(const ColFwdParams &P, int nctay)
{
    const int lf = P.l1 - P.l0, logS = P.logn - P.l1;
    // every cluster's column groups lie in one level-l0 block
    if (lf < 8 || lf > 12 || logS < 2 + ((12 - lf) > 3 ? 12 - lf : 3)) return false;
    // at most one job group per side, the row-vector side first
    if (nctay < 1 || nctay > 2) return false;
    for (int k = 0; k < nctay * P.jobs_per_cta; ++k) {
        const ColFwdJob &J = P.job[k], &J0 = P.job[(k / P.jobs_per_cta) * P.jobs_per_cta];
        if (!src_aligned(J.src) || !aligned(J.dst, 16) || J.vec_side != J0.vec_side) return false;
    }
    if (nctay == 2 && !(P.job[0].vec_side == 0 && P.job[P.jobs_per_cta].vec_side == 1)) return false;
    return true;
}

bool col4_inv_ok(const ColInvParams &P)
{
    const int lf = P.l1 - P.l0, logS = P.logn - P.l1;
    // every cluster's column groups lie in one level-l0 block
    if (lf < 8 || lf > 12 || logS < 2 + ((12 - lf) > 3 ? 12 - lf : 3)) return false;
    // three primes only with the CRT epilogue (the three-CTA cluster kernel)
    if (P.nprime != 1 && !(P.nprime == 3 && epi_crt(P.epi) && FCIRC_C4_X3)) return false;
    for (int q = 0; q < P.nprime; ++q)
        if (!aligned(P.job[q].src, 16) || (!epi_crt(P.epi) && !aligned(P.job[q].dst, 16))) return false;
    return true;
}

bool col4_fwd_ilv_ok(const ColFwdParams &P, int nctay)
{
    if (!col4_fwd_ok(P, nctay) || P.logn - P.l1 != 12) return false;
    for (int k = 0; k < nctay * P.jobs_per_cta; ++k)
        if (!aligned(P.job[k].dst, 32)) return false;
    return true;
}

bool col4_inv_ilv_ok(const ColInvParams &P)
{
    if (!col4_inv_ok(P) || P.logn - P.l1 != 12) return false;
    for (int q = 0; q < P.nprime; ++q)
        if (!aligned(P.job[q].src, 32)) return false;
    return true;
}

int launch_colfwd4(const ColFwdParams &Pin, int nctay, cudaStream_t s)
{
    ColFwdParams P = Pin;
    P.vec_group0 = 0;
    while (P.vec_group0 < nctay && P.job[P.vec_group0 * P.jobs_per_cta].vec_side == 0) ++P.vec_group0;
    // source mode of the row-vector group and of the vector group (when present)
    const int m0 = P.vec_group0 > 0 ? c4_mode(P.job[0].src, P.job[0].half) : MODE_U32;
    const int m1 = P.vec_group0 < nctay
                       ? c4_mode(P.job[P.vec_group0 * P.jobs_per_cta].src, P.job[P.vec_group0 * P.jobs_per_cta].half)
                       : MODE_U32;
    for (int g = 0; g < nctay; ++g)
        for (int k = 0; k < P.jobs_per_cta; ++k) {
            const ColFwdJob &J = P.job[g * P.jobs_per_cta + k];
            if (c4_mode(J.src, J.half) != (g < P.vec_group0 ? m0 : m1))
                return fail(FCIRC_EINVAL, "column pass: mixed source modes in one job group");
        }
    switch (P.l1 - P.l0) {
    case 8: return launch_c4fwd_lf<8>(P, nctay, m0, m1, s);
    case 9: return launch_c4fwd_lf<9>(P, nctay, m0, m1, s);
    case 10: return launch_c4fwd_lf<10>(P, nctay, m0, m1, s);
    case 11: return launch_c4fwd_lf<11>(P, nctay, m0, m1, s);
    case 12: return launch_c4fwd_lf<12>(P, nctay, m0, m1, s);
    default: return fail(FCIRC_EINVAL, "column pass of %d levels", P.l1 - P.l0);
    }
}

int launch_colinv4(const ColInvParams &P, cudaStream_t s)
{
    const int lf = P.l1 - P.l0;
    if (P.nprime == 1) {
        switch (lf) {
        case 8: return launch_c4inv_lf<8, 1>(P, s);
        case 9: return launch_c4inv_lf<9, 1>(P, s);
        case 10: return launch_c4inv_lf<10, 1>(P, s);
        case 11: return launch_c4inv_lf<11, 1>(P, s);
        case 12: return launch_c4inv_lf<12, 1>(P, s);
        }
    } else if (P.nprime == 3 && epi_crt(P.epi)) {
        switch (lf) {
        case 8: return launch_c4inv_x3<8>(P, s);
        case 9: return launch_c4inv_x3<9>(P, s);
        case 10: return launch_c4inv_x3<10>(P, s);
        case 11: return launch_c4inv_x3<11>(P, s);
        case 12: return launch_c4inv_x3<12>(P, s);
        }
    }
    return fail(FCIRC_EINVAL, "column pass of %d levels, %d primes", lf, P.nprime);
}

}  // namespace fcirc
