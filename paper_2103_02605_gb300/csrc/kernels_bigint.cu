// kernels_bigint.cu -- carry propagation for the large-integer product
// (Section 3.2): the circulant product over three primes and the CRT give
// exact 64-bit column sums col_k = sum_{i+j=k} A_i B_j; the product is
// sum_k col_k 2^(16k), written out here in base 2^16.
//
// Carry lookahead without any inter-CTA wait.  A thread owns 16 consecutive
// positions.  Its carry-out as a function of its carry-in c (c < 2^41 here)
// is c -> H + [c >= tau], where X = sum_j col_j 2^(16j) over its positions,
// H = X >> 256 and tau = 2^256 - (X mod 2^256) (saturated: only values below
// 2^48 can ever be reached).  These maps compose in closed form,
//   (H2, tau2) o (H1, tau1) = (H2 + [H1 >= tau2], H1 + 1 == tau2 ? tau1 : INF),
// so three launches suffice: per-chunk maps (a block scan over threads),
// one CTA scanning the chunk maps into chunk carry-ins, and a final pass
// that rebuilds each thread's carry-in and writes its limbs.
#include <stdint.h>

#include "common.hpp"
#include "kernels_bigint.hpp"
#include "prof.hpp"

namespace fcirc {

namespace {

constexpr uint64_t kInf = ~0ull;
constexpr int kCarryThreads = 256;
constexpr int kPerThread = 16;
constexpr int kChunk = kCarryThreads * kPerThread;   // 4096 positions per CTA

struct CMap {
    uint64_t H, tau;
};

// apply f1 first, then f2
__device__ __forceinline__ CMap compose(CMap f1, CMap f2)
{
    CMap r;
    r.H = f2.H + (f1.H >= f2.tau ? 1u : 0u);
    r.tau = (f2.tau != kInf && f1.H + 1 == f2.tau) ? f1.tau : kInf;
    return r;
}

__device__ __forceinline__ uint64_t apply(CMap f, uint64_t c) { return f.H + (c >= f.tau ? 1u : 0u); }

// The 16 column sums of thread position k0 (zero past ncols).
__device__ __forceinline__ void load16(const uint64_t *cols, uint64_t ncols, uint64_t k0, uint64_t *v)
{
    if (k0 + kPerThread <= ncols) {
        const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(cols + k0);
#pragma unroll
        for (int j = 0; j < kPerThread / 2; ++j) {
            const ulonglong2 t = q[j];
            v[2 * j] = t.x;
            v[2 * j + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kPerThread; ++j) v[j] = (k0 + j < ncols) ? cols[k0 + j] : 0;
    }
}

__device__ __forceinline__ CMap thread_map(const uint64_t *v)
{
    uint64_t c = 0, low48 = 0;
    bool ones = true;
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const uint64_t t = v[j] + c;
        const uint64_t limb = t & 0xFFFFu;
        if (j < 3)
            low48 |= limb << (16 * j);
        else
            ones = ones && (limb == 0xFFFFu);
        c = t >> 16;
    }
    CMap m;
    m.H = c;
    m.tau = ones ? ((1ull << 48) - low48) : kInf;
    return m;
}

__device__ __forceinline__ CMap shfl_up_map(CMap m, int d)
{
    CMap o;
    o.H = __shfl_up_sync(0xffffffffu, m.H, d);
    o.tau = __shfl_up_sync(0xffffffffu, m.tau, d);
    return o;
}

// Inclusive block scan (in thread order) of the maps; also returns the
// inclusive map of the previous thread in `prev` (valid for tid > 0).
__device__ __forceinline__ CMap block_scan(CMap m, CMap &prev, CMap *sh)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kCarryThreads / 32;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const CMap o = shfl_up_map(m, d);
        if (lane >= d) m = compose(o, m);
    }
    if (lane == 31) sh[warp] = m;
    __syncthreads();
    if (warp == 0) {
        CMap w = sh[lane < NW ? lane : NW - 1];
#pragma unroll
        for (int d = 1; d < NW; d <<= 1) {
            const CMap o = shfl_up_map(w, d);
            if (lane >= d && lane < NW) w = compose(o, w);
        }
        if (lane < NW) sh[NW + lane] = w;   // inclusive totals of warps 0..lane
    }
    __syncthreads();
    if (warp > 0) m = compose(sh[NW + warp - 1], m);
    const CMap up = shfl_up_map(m, 1);
    prev = (lane > 0) ? up : (warp > 0 ? sh[NW + warp - 1] : m);
    return m;
}

__global__ void __launch_bounds__(kCarryThreads) k_carry_local(const uint64_t *cols, uint64_t ncols,
                                                                CMap *chunk_maps)
{
    __shared__ CMap sh[2 * (kCarryThreads / 32)];
    const uint64_t k0 = ((uint64_t)blockIdx.x * kCarryThreads + threadIdx.x) * kPerThread;
    uint64_t v[kPerThread];
    load16(cols, ncols, k0, v);
    CMap prev;
    const CMap m = block_scan(thread_map(v), prev, sh);
    if (threadIdx.x == kCarryThreads - 1) chunk_maps[blockIdx.x] = m;
}

// One CTA: carry into each chunk, from carry 0 into chunk 0.
__global__ void __launch_bounds__(kCarryThreads) k_carry_scan(const CMap *chunk_maps, uint64_t nchunks,
                                                               uint64_t *chunk_cin)
{
    __shared__ CMap sh[2 * (kCarryThreads / 32)];
    const uint64_t per = (nchunks + kCarryThreads - 1) / kCarryThreads;
    const uint64_t c0 = threadIdx.x * per, c1 = c0 + per < nchunks ? c0 + per : nchunks;
    // this thread's chunks as one map; the maps have no identity element, so
    // a thread without chunks holds c -> 0 -- only trailing threads are
    // empty, and nothing reads their results
    CMap agg{0, kInf};
    bool any = false;
    for (uint64_t c = c0; c < c1; ++c) {
        agg = any ? compose(agg, chunk_maps[c]) : chunk_maps[c];
        any = true;
    }
    CMap prev;
    const CMap incl = block_scan(agg, prev, sh);
    (void)incl;
    uint64_t cin = (threadIdx.x == 0) ? 0 : apply(prev, 0);
    for (uint64_t c = c0; c < c1; ++c) {
        chunk_cin[c] = cin;
        cin = apply(chunk_maps[c], cin);
    }
}

__global__ void __launch_bounds__(kCarryThreads) k_carry_apply(const uint64_t *cols, uint64_t ncols,
                                                                const uint64_t *chunk_cin, uint16_t *out,
                                                                uint64_t nlimbs)
{
    __shared__ CMap sh[2 * (kCarryThreads / 32)];
    const uint64_t k0 = ((uint64_t)blockIdx.x * kCarryThreads + threadIdx.x) * kPerThread;
    uint64_t v[kPerThread];
    load16(cols, ncols, k0, v);
    CMap prev;
    (void)block_scan(thread_map(v), prev, sh);
    const uint64_t cchunk = chunk_cin[blockIdx.x];
    uint64_t c = threadIdx.x == 0 ? cchunk : apply(prev, cchunk);
    uint16_t limb[kPerThread];
#pragma unroll
    for (int j = 0; j < kPerThread; ++j) {
        const uint64_t t = v[j] + c;
        limb[j] = (uint16_t)(t & 0xFFFFu);
        c = t >> 16;
    }
    if (k0 + kPerThread <= nlimbs && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
        uint4 *q = reinterpret_cast<uint4 *>(out + k0);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            uint4 w;
            w.x = limb[8 * j] | ((uint32_t)limb[8 * j + 1] << 16);
            w.y = limb[8 * j + 2] | ((uint32_t)limb[8 * j + 3] << 16);
            w.z = limb[8 * j + 4] | ((uint32_t)limb[8 * j + 5] << 16);
            w.w = limb[8 * j + 6] | ((uint32_t)limb[8 * j + 7] << 16);
            q[j] = w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kPerThread; ++j)
            if (k0 + j < nlimbs) out[k0 + j] = limb[j];
    }
}

}  // namespace

size_t carry_scratch_bytes(uint64_t nlimbs)
{
    const uint64_t nchunks = (nlimbs + kChunk - 1) / kChunk;
    return nchunks * (sizeof(CMap) + sizeof(uint64_t)) + 256;
}

int launch_carry(const uint64_t *cols, uint64_t ncols, uint16_t *out, uint64_t nlimbs, void *scratch,
                 cudaStream_t s)
{
    const uint64_t nchunks = (nlimbs + kChunk - 1) / kChunk;
    if (nchunks > (uint64_t)kCarryThreads * 65536)
        return fail(FCIRC_EINVAL, "carry: %llu limbs exceed the supported size", (unsigned long long)nlimbs);
    CMap *maps = static_cast<CMap *>(scratch);
    uint64_t *cin = reinterpret_cast<uint64_t *>(maps + nchunks);
    {
        ProfScope ps("k_carry_local", s);
        k_carry_local<<<(unsigned)nchunks, kCarryThreads, 0, s>>>(cols, ncols, maps);
        FCIRC_CUDA_TRY(cudaGetLastError());
    }
    {
        ProfScope ps("k_carry_scan", s);
        k_carry_scan<<<1, kCarryThreads, 0, s>>>(maps, nchunks, cin);
        FCIRC_CUDA_TRY(cudaGetLastError());
    }
    {
        ProfScope ps("k_carry_apply", s);
        k_carry_apply<<<(unsigned)nchunks, kCarryThreads, 0, s>>>(cols, ncols, cin, out, nlimbs);
        FCIRC_CUDA_TRY(cudaGetLastError());
    }
    return FCIRC_OK;
}

}  // namespace fcirc
