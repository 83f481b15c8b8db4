// kernels_tile.cu -- the 4096-residue tile kernel of the large modular path
// (the recursion of Algorithm 1, Section 2, below the column passes).
//
// k_tile4096: one contiguous tile of 4096 residues (a node of level m-12) of
// one prime per CTA of 256 threads; halving levels 0-3 / 4-7 / 8-10 of the
// tile as register stages with shared-memory transposes, the 2x2 leaf
// products, and the recombination back up.  Twiddles of levels 0-7 are
// generated once per CTA into shared memory, those of levels 8-10 by each
// thread for its own subtree (plan.cu explains the factorisation).  The body
// is tile4096_dev (tile_dev.cuh), shared with the batched kernel.
#include "common.hpp"
#include "kernels_mod.hpp"
#include "prof.hpp"
#include "tile_dev.cuh"

namespace fcirc {

// Resident CTAs per SM the kernel is compiled for (register budget).
#ifndef FCIRC_TILE_MINB
#define FCIRC_TILE_MINB 3
#endif

template <int MA, int MX, int VAR = TILE_FULL, bool TMA = false>
__global__ void __launch_bounds__(256, FCIRC_TILE_MINB) k_tile4096(const __grid_constant__ TileParams P)
{
    __shared__ __align__(128) uint32_t SA[4096];
    __shared__ __align__(128) uint32_t SX[4096];
    __shared__ Tw STW[256];
    __shared__ Tw SITW[256];
    __shared__ uint64_t bar;
    __shared__ uint32_t flag;
    const TileJob &J = P.job[blockIdx.y];
    const uint64_t t = blockIdx.x;
    tile4096_dev<MA, MX, VAR, TMA>(J, (uint32_t)P.N, (uint32_t)(t << 12), J.sig + t * (uint64_t)(11 * 6), SA, SX,
                                   STW, SITW, P.ilv, &P, (int)blockIdx.y, &bar, &flag);
}

bool fast_tile_ok(int logT) { return logT == 12; }

int launch_tile_fast(const TileParams &P, uint64_t ntiles, int njobs, cudaStream_t s)
{
    dim3 grid((unsigned)ntiles, njobs);
    const int ma = P.job[0].a.kind | (P.job[0].a.scaled ? 4 : 0);
    const int mx = P.job[0].x.kind | (P.job[0].x.scaled ? 4 : 0);
    if (P.var == TILE_ROW) {
        // the row-vector tree only: writes the transformed row vector
        for (int k = 0; k < njobs; ++k)
            if ((reinterpret_cast<uintptr_t>(P.job[k].dst) & 15) != 0)
                return fail(FCIRC_EINVAL, "tile kernel: unaligned transformed row vector");
        ProfScope ps("k_tile4096_row", s);
        if (ma == MODE_U32)
            k_tile4096<MODE_U32, MODE_U32, TILE_ROW><<<grid, 256, 0, s>>>(P);
        else if (ma == MODE_U32_S)
            k_tile4096<MODE_U32_S, MODE_U32, TILE_ROW><<<grid, 256, 0, s>>>(P);
        else
            return fail(FCIRC_EINVAL, "tile kernel: unsupported row source mode %d", ma);
        FCIRC_CUDA_TRY(cudaGetLastError());
        return FCIRC_OK;
    }
    if (P.tma) {
        // interleaved sides through TMA: plain scratch sources only
        if (ma != MODE_U32 || mx != MODE_U32 || !P.ilv)
            return fail(FCIRC_EINVAL, "tile kernel: TMA copies need interleaved plain sources (%d/%d)", ma, mx);
        if (P.var == TILE_PLANNED)
            for (int k = 0; k < njobs; ++k)
                if ((reinterpret_cast<uintptr_t>(P.job[k].a.ptr) & 15) != 0)
                    return fail(FCIRC_EINVAL, "tile kernel: unaligned transformed row vector");
        ProfScope ps(P.var == TILE_PLANNED ? "k_tile4096_planned" : "k_tile4096", s);
        if (P.var == TILE_SHIFT)
            k_tile4096<MODE_U32, MODE_U32, TILE_SHIFT, true><<<grid, 256, 0, s>>>(P);
        else if (P.var == TILE_PLANNED)
            k_tile4096<MODE_U32, MODE_U32, TILE_PLANNED, true><<<grid, 256, 0, s>>>(P);
        else if (P.var == TILE_FULL)
            k_tile4096<MODE_U32, MODE_U32, TILE_FULL, true><<<grid, 256, 0, s>>>(P);
        else
            return fail(FCIRC_EINVAL, "tile kernel: no TMA form of variant %d", P.var);
        FCIRC_CUDA_TRY(cudaGetLastError());
        return FCIRC_OK;
    }
    if (P.var == TILE_PLANNED) {
        // a transformed row vector (read as it is) with a vector
        for (int k = 0; k < njobs; ++k)
            if ((reinterpret_cast<uintptr_t>(P.job[k].a.ptr) & 15) != 0)
                return fail(FCIRC_EINVAL, "tile kernel: unaligned transformed row vector");
        if (mx != MODE_U32) return fail(FCIRC_EINVAL, "tile kernel: unsupported vector source mode %d", mx);
        ProfScope ps("k_tile4096_planned", s);
        k_tile4096<MODE_U32, MODE_U32, TILE_PLANNED><<<grid, 256, 0, s>>>(P);
        FCIRC_CUDA_TRY(cudaGetLastError());
        return FCIRC_OK;
    }
    ProfScope ps("k_tile4096", s);
    if (P.var == TILE_SHIFT) {
        if (ma != MODE_U32 || mx != MODE_U32)
            return fail(FCIRC_EINVAL, "tile kernel: shifted leaves need plain sources (%d/%d)", ma, mx);
        k_tile4096<MODE_U32, MODE_U32, TILE_SHIFT><<<grid, 256, 0, s>>>(P);
    } else if (ma == MODE_U32 && mx == MODE_U32)
        k_tile4096<MODE_U32, MODE_U32><<<grid, 256, 0, s>>>(P);
    else if (ma == MODE_U32_S && mx == MODE_U32)
        k_tile4096<MODE_U32_S, MODE_U32><<<grid, 256, 0, s>>>(P);
    else if (ma == MODE_U32REV_S && mx == MODE_U32)
        k_tile4096<MODE_U32REV_S, MODE_U32><<<grid, 256, 0, s>>>(P);
    else if (ma == MODE_REV_S && mx == MODE_U16)
        k_tile4096<MODE_REV_S, MODE_U16><<<grid, 256, 0, s>>>(P);
    else
        return fail(FCIRC_EINVAL, "tile kernel: unsupported source modes %d/%d", ma, mx);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

}  // namespace fcirc
