// kernels_fast.cu -- register-staged sm_103a kernels for the large modular
// path: the recursion of Algorithm 1 (Section 2) run as radix-16 register
// stages with shared-memory transposes in between.
//
// A thread keeps 16 residues of each side in registers and runs up to four
// halving levels on them without moving data (the 16 residues of a group are
// exactly the elements a 4-level subtree of the recursion combines).  Between
// stages the CTA re-distributes residues through shared memory, using
// layouts chosen so that every warp access is free of bank conflicts.
//
//  * k_colfwd<LF> / k_colinv<LF, NP>: LF (8..12) top levels of the whole
//    array, over 4 adjacent columns of 2^LF rows per CTA, one column per
//    thread; the inverse pass can carry all three primes of a polynomial
//    product and finish with the CRT.  The four-column kernels of
//    kernels_col4.cu take the passes they accept; these take the rest.
#include <atomic>

#include "common.hpp"
#include "kernels_mod.hpp"
#include "prof.hpp"
#include "tile_dev.cuh"

namespace fcirc {

// Resident CTAs per SM the column kernels are compiled for (register budgets).
#ifndef FCIRC_COL4
#define FCIRC_COL4 1
#endif
#ifndef FCIRC_COLFWD_MINB
#define FCIRC_COLFWD_MINB 2
#endif
#ifndef FCIRC_COLINV_MINB
#define FCIRC_COLINV_MINB 2
#endif

// ---------------------------------------------------------------------------
// column passes: 2^LF rows x 4 adjacent columns per CTA, 2^LF / 8 threads,
// each thread owning 32 residues of a stage (two batches of 16 registers)

// Shared-memory word of (row r, column c): rows are permuted inside aligned
// groups of 8 by an XOR with bits 4..6 of the row, so that both consecutive
// rows and rows 16 apart fall into distinct banks.
__device__ __forceinline__ int cphi(int r, int c) { return ((r ^ ((r >> 4) & 7)) << 2) | c; }

template <int LF>
struct ColShape {
    static constexpr int R = 1 << LF;
    static constexpr int NT = R / 8;
    static constexpr int NST = (LF + 3) / 4;
    static constexpr int NL0 = LF - 4 * (NST - 1);   // the first stage takes the remainder
    static constexpr int nl(int s) { return s == 0 ? NL0 : 4; }
    static constexpr int d0(int s) { return s == 0 ? 0 : NL0 + 4 * (s - 1); }
};

// Twiddles of local level D of one group (group-ordered table, see
// kernels_mod.hpp), read with 128-bit loads.
template <int D>
__device__ __forceinline__ void load_level(const Tw *g, Tw *tl)
{
    if constexpr (D == 0) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(g + 14));
        tl[0] = Tw{v.x, v.y};
    } else {
        const uint4 *q = reinterpret_cast<const uint4 *>(g + 16 - (2 << D));
#pragma unroll
        for (int k = 0; k < (1 << (D - 1)); ++k) {
            const uint4 v = __ldg(q + k);
            tl[2 * k] = Tw{v.x, v.y};
            tl[2 * k + 1] = Tw{v.z, v.w};
        }
    }
}

// levels D .. NL-1 of one group of 2^NL registers (both input sides)
template <int NL, int D, bool VEC>
__device__ __forceinline__ void fwd_levels(uint32_t *v, const Tw *g, uint32_t p, uint32_t p2)
{
    if constexpr (D < NL) {
        Tw tl[1 << D];
        load_level<D>(g, tl);
        constexpr int h = (1 << NL) >> (D + 1);
#pragma unroll
        for (int j = 0; j < (1 << D); ++j)
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const int lo = (j << (NL - D)) + i;
                if (VEC)
                    bfly_vec(v[lo], v[lo + h], tl[j], p, p2);
                else
                    bfly_row(v[lo], v[lo + h], tl[j], p, p2);
            }
        fwd_levels<NL, D + 1, VEC>(v, g, p, p2);
    }
}

// recombination levels D .. 0 of one group (inverse twiddles)
template <int NL, int D>
__device__ __forceinline__ void rec_levels(uint32_t *v, const Tw *g, uint32_t p, uint32_t p2)
{
    if constexpr (D >= 0) {
        Tw tl[1 << D];
        load_level<D>(g, tl);
        constexpr int h = (1 << NL) >> (D + 1);
#pragma unroll
        for (int j = 0; j < (1 << D); ++j)
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const int lo = (j << (NL - D)) + i;
                bfly_rec(v[lo], v[lo + h], tl[j], p, p2);
            }
        rec_levels<NL, D - 1>(v, g, p, p2);
    }
}

// Group slot h of thread tid in stage (D0, NL): column, first row, and the
// level-D0 block the group lies in; members are row0 + i 2^LST.
template <int LF, int D0, int NL>
__device__ __forceinline__ void col_group(int tid, int h, int &col, int &row0, int &blk)
{
    constexpr int NT = ColShape<LF>::NT;
    constexpr int LST = LF - D0 - NL;
    constexpr int LRB = LF - D0;
    const int gg = tid + NT * h;
    col = gg & 3;
    const int g = gg >> 2;
    blk = g >> LST;
    row0 = (blk << LRB) + (g & ((1 << LST) - 1));
}

template <int LF, int S, int MODE>
__device__ __forceinline__ void colfwd_stage(const ColFwdJob &J, const ColFwdParams &P, uint32_t *sm,
                                             uint32_t base, uint32_t pb, int logS, int tid)
{
    constexpr int half = (S == 0) ? ((MODE >> 3) & 3) : 0;
    using Sh = ColShape<LF>;
    constexpr int NL = Sh::nl(S), D0 = Sh::d0(S);
    constexpr int M = 1 << NL, B = 16 >> NL, LST = LF - D0 - NL;
    constexpr bool FIRST = (S == 0), LAST = (S == Sh::NST - 1);
    const uint32_t p = J.p, p2 = 2 * J.p;
    const Tw *gt = J.gtw + P.stage_off[S];
#pragma unroll 1
    for (int bt = 0; bt < 2; ++bt) {
        uint32_t v[16];
#pragma unroll
        for (int hb = 0; hb < B; ++hb) {
            int col, row0, blk;
            col_group<LF, D0, NL>(tid, bt * B + hb, col, row0, blk);
            uint32_t *vg = v + hb * M;
            if constexpr (FIRST && half == 1) {
                // input zero in rows < R/2, level 0 has s = 1: (0 + hi, 0 - hi)
#pragma unroll
                for (int i = M / 2; i < M; ++i)
                    vg[i] = ld_raw<MODE>(J.src, P.N, base + ((row0 + (i << LST)) << logS) + col);
#pragma unroll
                for (int i = M / 2; i < M; ++i) {
                    const uint32_t t = ld_scale<MODE>(vg[i], J.src, p);
                    vg[i - M / 2] = t;
                    vg[i] = p2 - t;
                }
            } else if constexpr (FIRST && half == 2) {
                // input zero in rows >= R/2, level 0 has s = 1: (lo, lo)
#pragma unroll
                for (int i = 0; i < M / 2; ++i)
                    vg[i] = ld_raw<MODE>(J.src, P.N, base + ((row0 + (i << LST)) << logS) + col);
#pragma unroll
                for (int i = 0; i < M / 2; ++i) {
                    vg[i] = ld_scale<MODE>(vg[i], J.src, p);
                    vg[i + M / 2] = vg[i];
                }
            } else if constexpr (FIRST) {
#pragma unroll
                for (int i = 0; i < M; ++i)
                    vg[i] = ld_raw<MODE>(J.src, P.N, base + ((row0 + (i << LST)) << logS) + col);
#pragma unroll
                for (int i = 0; i < M; ++i) vg[i] = ld_scale<MODE>(vg[i], J.src, p);
            } else {
#pragma unroll
                for (int i = 0; i < M; ++i) vg[i] = sm[cphi(row0 + (i << LST), col)];
            }
        }
#pragma unroll
        for (int hb = 0; hb < B; ++hb) {
            int col, row0, blk;
            col_group<LF, D0, NL>(tid, bt * B + hb, col, row0, blk);
            const Tw *g = gt + (((pb << D0) + blk) << 4);
            uint32_t *vg = v + hb * M;
            if constexpr (FIRST && half != 0) {
                if (J.vec_side)
                    fwd_levels<NL, 1, true>(vg, g, p, p2);
                else
                    fwd_levels<NL, 1, false>(vg, g, p, p2);
            } else {
                if (J.vec_side)
                    fwd_levels<NL, 0, true>(vg, g, p, p2);
                else
                    fwd_levels<NL, 0, false>(vg, g, p, p2);
            }
        }
#pragma unroll
        for (int hb = 0; hb < B; ++hb) {
            int col, row0, blk;
            col_group<LF, D0, NL>(tid, bt * B + hb, col, row0, blk);
#pragma unroll
            for (int i = 0; i < M; ++i) {
                const uint32_t row = row0 + (i << LST);
                if (LAST)
                    J.dst[base + (row << logS) + col] = v[hb * M + i];
                else
                    sm[cphi(row, col)] = v[hb * M + i];
            }
        }
    }
}

template <int LF, int MODE>
__device__ __forceinline__ void colfwd_jobs(const ColFwdParams &P, uint32_t *sm, int j0, uint32_t base,
                                            uint32_t pb, int logS, int tid)
{
    using Sh = ColShape<LF>;
#pragma unroll 1
    for (int jj = 0; jj < P.jobs_per_cta; ++jj) {
        const ColFwdJob &J = P.job[j0 + jj];
        if (jj > 0) __syncthreads();   // the previous job's last reads of sm are done
        colfwd_stage<LF, 0, MODE>(J, P, sm, base, pb, logS, tid);
        if constexpr (Sh::NST > 1) {
            __syncthreads();
            colfwd_stage<LF, 1, MODE>(J, P, sm, base, pb, logS, tid);
        }
        if constexpr (Sh::NST > 2) {
            __syncthreads();
            colfwd_stage<LF, 2, MODE>(J, P, sm, base, pb, logS, tid);
        }
    }
}

// blockIdx.y selects a group of jobs_per_cta jobs; group 0 reads its input
// in mode M0, group 1 in mode M1
template <int LF, int M0, int M1>
__global__ void __launch_bounds__(ColShape<LF>::NT, FCIRC_COLFWD_MINB) k_colfwd(const __grid_constant__ ColFwdParams P)
{
    extern __shared__ __align__(16) uint32_t sm[];
    using Sh = ColShape<LF>;
    const int tid = threadIdx.x;
    const int logS = P.logn - P.l1;
    const int cg_bits = logS - 2;
    const uint32_t pb = blockIdx.x >> cg_bits;
    const uint32_t cg = blockIdx.x & ((1u << cg_bits) - 1);
    const uint32_t base = (pb << (P.logn - P.l0)) + (cg << 2);
    const int j0 = blockIdx.y * P.jobs_per_cta;
    if (blockIdx.y == 0)
        colfwd_jobs<LF, M0>(P, sm, j0, base, pb, logS, tid);
    else
        colfwd_jobs<LF, M1>(P, sm, j0, base, pb, logS, tid);
}

template <int LF, int NP, int S>
__device__ __forceinline__ void colinv_stage(const ColInvParams &P, uint32_t *sm, uint32_t base,
                                             uint32_t pb, int logS, int tid)
{
    using Sh = ColShape<LF>;
    constexpr int NL = Sh::nl(S), D0 = Sh::d0(S);
    constexpr int M = 1 << NL, B = 16 >> NL, LST = LF - D0 - NL;
    constexpr bool FIRST = (S == Sh::NST - 1), LAST = (S == 0);
    constexpr int R = 1 << LF;
#pragma unroll 1
    for (int q = 0; q < NP; ++q) {
        const ColInvJob &J = P.job[q];
        const uint32_t p = J.p, p2 = 2 * J.p;
        uint32_t *smq = sm + q * (R * 4);
        const Tw *gt = J.gitw + P.stage_off[S];
#pragma unroll 1
        for (int bt = 0; bt < 2; ++bt) {
            uint32_t v[16];
#pragma unroll
            for (int hb = 0; hb < B; ++hb) {
                int col, row0, blk;
                col_group<LF, D0, NL>(tid, bt * B + hb, col, row0, blk);
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    const uint32_t row = row0 + (i << LST);
                    v[hb * M + i] = FIRST ? J.src[base + (row << logS) + col] : smq[cphi(row, col)];
                }
            }
#pragma unroll
            for (int hb = 0; hb < B; ++hb) {
                int col, row0, blk;
                col_group<LF, D0, NL>(tid, bt * B + hb, col, row0, blk);
                rec_levels<NL, NL - 1>(v + hb * M, gt + (((pb << D0) + blk) << 4), p, p2);
            }
#pragma unroll
            for (int hb = 0; hb < B; ++hb) {
                int col, row0, blk;
                col_group<LF, D0, NL>(tid, bt * B + hb, col, row0, blk);
#pragma unroll
                for (int i = 0; i < M; ++i) {
                    const uint32_t row = row0 + (i << LST);
                    const uint32_t val = v[hb * M + i];
                    if (!LAST)
                        smq[cphi(row, col)] = val;
                    else if (epi_crt(P.epi))
                        smq[cphi(row, col)] = reduce_once(val, p);   // canonical, for the CRT below
                    else
                        J.dst[base + (row << logS) + col] = P.epi == EPI_CANON ? reduce_once(val, p) : val;
                }
            }
        }
    }
    if (LAST && NP == 3 && epi_crt(P.epi)) {
        // every residue of this thread's groups was written by this thread
        const uint32_t mask = P.N - 1, rot = P.epi == EPI_CRT_ROT ? mask : 0u;
#pragma unroll 1
        for (int h = 0; h < 2 * B; ++h) {
            int col, row0, blk;
            col_group<LF, D0, NL>(tid, h, col, row0, blk);
#pragma unroll 4
            for (int i = 0; i < M; ++i) {
                const uint32_t row = row0 + (i << LST);
                const int w = cphi(row, col);
                const uint32_t idx = base + (row << logS) + col;
                // EPI_CRT_ROT: coefficient k is circulant entry k + 1
                const uint32_t dst = (idx + rot) & mask;
                if (dst < P.nout) P.dst64[dst] = crt3(sm[w], sm[R * 4 + w], sm[2 * R * 4 + w], P.crt);
            }
        }
    }
}

template <int LF, int NP>
__global__ void __launch_bounds__(ColShape<LF>::NT, NP == 1 ? FCIRC_COLINV_MINB : 1) k_colinv(const __grid_constant__ ColInvParams P)
{
    extern __shared__ __align__(16) uint32_t sm[];
    using Sh = ColShape<LF>;
    const int tid = threadIdx.x;
    const int logS = P.logn - P.l1;
    const int cg_bits = logS - 2;
    const uint32_t pb = blockIdx.x >> cg_bits;
    const uint32_t cg = blockIdx.x & ((1u << cg_bits) - 1);
    const uint32_t base = (pb << (P.logn - P.l0)) + (cg << 2);
    static_assert(Sh::NST >= 2 && Sh::NST <= 3, "column pass of 5..12 levels");
    colinv_stage<LF, NP, Sh::NST - 1>(P, sm, base, pb, logS, tid);
    __syncthreads();
    if constexpr (Sh::NST > 2) {
        colinv_stage<LF, NP, 1>(P, sm, base, pb, logS, tid);
        __syncthreads();
    }
    colinv_stage<LF, NP, 0>(P, sm, base, pb, logS, tid);
}

// ---------------------------------------------------------------------------
// launchers

template <class K>
static int ensure_smem_f(K kernel, int bytes, std::atomic<unsigned> &mask)
{
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    const unsigned bit = 1u << (dev & 31);
    if (mask.load() & bit) return FCIRC_OK;
    FCIRC_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    mask.fetch_or(bit);
    return FCIRC_OK;
}

bool fast_col_ok(int lf, int logS) { return lf >= 8 && lf <= 12 && logS >= 2; }

static int src_mode(const Src &s, int half)
{
    return s.kind | (s.scaled ? 4 : 0) | (half << 3);
}

template <int LF, int M0, int M1>
static int launch_colfwd_m(const ColFwdParams &P, int nctay, cudaStream_t s)
{
    static std::atomic<unsigned> mask{0};
    const int smem = (1 << LF) * 4 * 4;
    FCIRC_TRY(ensure_smem_f(k_colfwd<LF, M0, M1>, smem, mask));
    const uint64_t ncta = (uint64_t)1 << (P.l0 + (P.logn - P.l1) - 2);
    dim3 grid((unsigned)ncta, nctay);
    ProfScope ps("k_colfwd", s);
    k_colfwd<LF, M0, M1><<<grid, ColShape<LF>::NT, smem, s>>>(P);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

template <int LF>
static int launch_colfwd_lf(const ColFwdParams &P, int nctay, cudaStream_t s)
{
    const int m0 = src_mode(P.job[0].src, P.job[0].half);
    const int m1 = nctay > 1 ? src_mode(P.job[P.jobs_per_cta].src, P.job[P.jobs_per_cta].half) : MODE_U32;
    for (int g = 0; g < nctay; ++g)
        for (int k = 0; k < P.jobs_per_cta; ++k) {
            const ColFwdJob &J = P.job[g * P.jobs_per_cta + k];
            if (src_mode(J.src, J.half) != (g == 0 ? m0 : m1))
                return fail(FCIRC_EINVAL, "column pass: mixed source modes in one job group");
        }
    if (m0 == MODE_U32_S && m1 == MODE_U32) return launch_colfwd_m<LF, MODE_U32_S, MODE_U32>(P, nctay, s);
    if (m0 == MODE_U32REV_S && m1 == MODE_U32) return launch_colfwd_m<LF, MODE_U32REV_S, MODE_U32>(P, nctay, s);
    if (m0 == MODE_U32 && m1 == MODE_U32) return launch_colfwd_m<LF, MODE_U32, MODE_U32>(P, nctay, s);
    if (m0 == MODE_REV_S_H && m1 == MODE_U16_H) return launch_colfwd_m<LF, MODE_REV_S_H, MODE_U16_H>(P, nctay, s);
    if (m0 == MODE_REV_S && m1 == MODE_U16) return launch_colfwd_m<LF, MODE_REV_S, MODE_U16>(P, nctay, s);
    return fail(FCIRC_EINVAL, "column pass: unsupported source modes %d/%d", m0, m1);
}

int launch_colfwd(const ColFwdParams &P, int nctay, cudaStream_t s)
{
    // only the four-column kernels write the tile-pair interleaved layout
    if (P.ilv) {
        if (!col4_fwd_ilv_ok(P, nctay)) return fail(FCIRC_EINVAL, "column pass: interleaved output not possible here");
        return launch_colfwd4(P, nctay, s);
    }
#if FCIRC_COL4
    if (col4_fwd_ok(P, nctay)) return launch_colfwd4(P, nctay, s);
#endif
    switch (P.l1 - P.l0) {
    case 8: return launch_colfwd_lf<8>(P, nctay, s);
    case 9: return launch_colfwd_lf<9>(P, nctay, s);
    case 10: return launch_colfwd_lf<10>(P, nctay, s);
    case 11: return launch_colfwd_lf<11>(P, nctay, s);
    case 12: return launch_colfwd_lf<12>(P, nctay, s);
    default: return fail(FCIRC_EINVAL, "column pass of %d levels", P.l1 - P.l0);
    }
}

template <int LF, int NP>
static int launch_colinv_lf(const ColInvParams &P, cudaStream_t s)
{
    static std::atomic<unsigned> mask{0};
    const int smem = NP * (1 << LF) * 4 * 4;
    const uint64_t ncta = (uint64_t)1 << (P.l0 + (P.logn - P.l1) - 2);
    FCIRC_TRY(ensure_smem_f(k_colinv<LF, NP>, smem, mask));
    ProfScope ps("k_colinv", s);
    k_colinv<LF, NP><<<(unsigned)ncta, ColShape<LF>::NT, smem, s>>>(P);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

int launch_colinv(const ColInvParams &P, cudaStream_t s)
{
    // only the four-column kernels read the tile-pair interleaved layout
    if (P.ilv) {
        if (!col4_inv_ilv_ok(P)) return fail(FCIRC_EINVAL, "column pass: interleaved input not possible here");
        return launch_colinv4(P, s);
    }
#if FCIRC_COL4
    if (col4_inv_ok(P)) return launch_colinv4(P, s);
#endif
    const int lf = P.l1 - P.l0;
    if (P.nprime == 1) {
        switch (lf) {
        case 8: return launch_colinv_lf<8, 1>(P, s);
        case 9: return launch_colinv_lf<9, 1>(P, s);
        case 10: return launch_colinv_lf<10, 1>(P, s);
        case 11: return launch_colinv_lf<11, 1>(P, s);
        case 12: return launch_colinv_lf<12, 1>(P, s);
        }
    } else if (P.nprime == 3) {
        switch (lf) {
        case 8: return launch_colinv_lf<8, 3>(P, s);
        case 9: return launch_colinv_lf<9, 3>(P, s);
        case 10: return launch_colinv_lf<10, 3>(P, s);
        case 11: return launch_colinv_lf<11, 3>(P, s);
        case 12: return launch_colinv_lf<12, 3>(P, s);
        }
    }
    return fail(FCIRC_EINVAL, "column pass of %d levels, %d primes", lf, P.nprime);
}

}  // namespace fcirc
