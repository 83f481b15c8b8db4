// tma_host.cu -- host side of the TMA copies of the tile kernel and of the
// forward column pass: tensor maps of the tile-pair interleaved arrays, and
// the limit of the kernels' bounded mbarrier waits.
//
// An interleaved array of N residues (N a multiple of 8192) is described to
// the TMA unit as a 4-D tensor of 32-bit words, innermost first:
//   4 words of a column quad (16 bytes, contiguous),
//   2 tiles of a pair (stride 16 bytes),
//   1024 column quads (stride 32 bytes: one sector per quad and pair),
//   N / 8192 tile pairs (stride 32 KiB).
// One box {4, 1, 256, 1} is 256 column quads of one tile (4 KiB), which lands
// in shared memory in the tile's natural order; four boxes are a tile.
#include <atomic>
#include <mutex>

#include <cudaTypedefs.h>

#include "../../include/fcirc.h"
#include "common.hpp"
#include "kernels_mod.hpp"

namespace fcirc {

namespace {
constexpr uint32_t kDefaultSpinLimit = 1u << 22;
std::atomic<uint32_t> g_spin_limit{kDefaultSpinLimit};

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            (void)cudaGetLastError();
    });
    return fn;
}

bool encode_ilv(PFN_cuTensorMapEncodeTiled_v12000 fn, CUtensorMap *map, const void *ptr, uint64_t N)
{
    const cuuint64_t dims[4] = {4, 2, 1024, N / 8192};
    const cuuint64_t strides[3] = {16, 32, 32768};
    const cuuint32_t box[4] = {4, 1, 256, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 4, const_cast<void *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
// The same array, seen by the forward column pass's stores, with the tile
// pair index split as 8 t + k: a 5-D tensor {4 words, 2 tiles, 1024 quads,
// 8 (k, stride 32 KiB), N / 65536 (t, stride 256 KiB)}.  One box
// {4, 2, 1, 1, 256} is one column quad of the 256 tile pairs 8 t + k of one
// k (8 KiB, 32 bytes per pair, dense in shared memory): the k-th sector of
// each of a CTA's 256 threads, adjacent for adjacent threads.
bool encode_ilv_store(PFN_cuTensorMapEncodeTiled_v12000 fn, CUtensorMap *map, void *ptr, uint64_t N)
{
    const cuuint64_t dims[5] = {4, 2, 1024, 8, N / 65536};
    const cuuint64_t strides[4] = {16, 32, 32768, 262144};
    const cuuint32_t box[5] = {4, 2, 1, 1, 256};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 5, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

int fwd_tma_maps(ColFwdParams &P, int njobs, int lf)
{
    P.tma_st = 0;
    // one column quad per CTA (12 levels over 4096 columns), whole boxes
    if (!P.ilv || lf != 12 || P.N % (8192u * 2048u) != 0) return FCIRC_OK;
    PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
    if (!fn) return FCIRC_OK;   // no encoder: the kernel's direct sector stores
    for (int k = 0; k < njobs; ++k)
        if (!aligned16(P.job[k].dst) || !encode_ilv_store(fn, &P.tmap[k], P.job[k].dst, P.N)) return FCIRC_OK;
    P.tma_st = 1;
    return FCIRC_OK;
}

int tile_tma_maps(TileParams &P, int njobs)
{
    P.tma = 0;
    // the kernel's TMA form moves every side the variant reads plus the
    // destination: all of them must be interleaved
    const int want = P.var == TILE_PLANNED ? 2 : 3;
    if (P.var == TILE_ROW || (P.ilv & want) != want || P.logT != 12 || P.N % 8192 != 0) return FCIRC_OK;
    PFN_cuTensorMapEncodeTiled_v12000 fn = encoder();
    if (!fn) return FCIRC_OK;   // no encoder: the kernel's scalar accesses
    for (int q = 0; q < njobs; ++q) {
        const TileJob &J = P.job[q];
        const void *ptrs[3] = {J.a.ptr, J.x.ptr, J.dst};
        const bool need[3] = {(P.ilv & 1) && P.var != TILE_PLANNED, (P.ilv & 2) != 0, (P.ilv & 2) != 0};
        for (int k = 0; k < 3; ++k) {
            if (!need[k]) continue;
            if (!aligned16(ptrs[k]) || !encode_ilv(fn, &P.tmap[q][k], ptrs[k], P.N)) return FCIRC_OK;
        }
    }
    FCIRC_TRY(device_status_word(&P.status));
    P.spin_limit = g_spin_limit.load();
    P.tma = 1;
    return FCIRC_OK;
}

}  // namespace fcirc

extern "C" int fcirc_debug_spin_limit(long long probes)
{
    fcirc::g_spin_limit.store(probes < 0 ? fcirc::kDefaultSpinLimit
                                         : (uint32_t)(probes > 0xFFFFFFFFll ? 0xFFFFFFFFll : probes));
    return FCIRC_OK;
}
