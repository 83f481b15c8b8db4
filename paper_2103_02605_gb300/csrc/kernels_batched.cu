// kernels_batched.cu -- many independent f-circulant products of uneven
// sizes and distinct f in one persistent launch (the recursion of Algorithm
// 1, Section 2, per instance).
//
// Launch sequence (all on one stream, graph-capturable, no host round trip):
//   1. k_bplan     one thread per instance: n_i from the offsets, a 2^L-th
//                  root of f_i (L = log2 n_i - 1; Theorem 1), its inverse and
//                  the leaf scale 2^32 2^-L; a size bucket for scheduling.
//   2. k_border    bucket starts, largest sizes first (longest processing
//                  time first), and the reset of the work counter.
//   3. k_bscatter  the instance order.
//   4. k_bmain     persistent CTAs that take instances from an atomic
//                  counter in that order.  An instance of up to 2^big_log
//                  residues is one tile in shared memory; a larger one runs
//                  inside the CTA as its top k levels over 2^k-row columns,
//                  its 2^k tiles, and the top k recombination levels.
// Errors of single instances (size not a power of two or above 2^16, no
// root) set the sticky device status word read by fcirc_sync_status and
// leave that instance's output untouched.
#include <stdint.h>

#include "common.hpp"
#include "kernels_batched.hpp"
#include "prof.hpp"
#include "ring.hpp"
#include "tile_dev.cuh"

namespace fcirc {

namespace {

constexpr int kBThreads = 256;
constexpr int kBuckets = 18;   // 17 sizes 2^16 .. 2^0, then invalid instances
constexpr int kBMaxLog = 16;

__device__ __forceinline__ void set_status(uint32_t *st, uint32_t code) { atomicCAS(st, 0u, code); }

__global__ void k_bplan(const BatchParams P)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.count) return;
    BatchMeta md{};
    md.ok = 0;
    md.m = 0;
    const uint64_t o0 = P.offsets[i], o1 = P.offsets[i + 1];
    const uint64_t n = o1 - o0;
    int bucket = kBuckets - 1;
    if (o1 < o0 || o1 > P.total || n == 0 || (n & (n - 1)) != 0 || n > ((uint64_t)1 << kBMaxLog)) {
        set_status(P.status, FCIRC_EINVAL);
    } else {
        const int m = 63 - __clzll(n);
        const int L = m - 1;
        md.m = m;
        uint32_t rho = 1;
        const uint32_t f = P.f[i] % P.p;
        // Barrett products: a 64-bit remainder per product made this kernel
        // take 0.3 ms for 10,000 instances
        const host::ModP M(P.p);
        if (m == 0) {
            md.ok = 1;   // 1x1: c = a x
        } else if (L > P.v || f == 0 || !host::nth_root_2k_om(f, L, M, P.Om, P.v, rho)) {
            set_status(P.status, FCIRC_ENOROOT);
        } else {
            md.ok = 1;
            md.rho = rho;
            md.rhoi = M.inv(rho);
            const uint32_t two32 = (uint32_t)((1ull << 32) % P.p);
            const uint32_t kt = M.mul(two32, M.pow((P.p + 1) / 2, L));
            md.kt = Tw{kt, M.quot32(kt)};
        }
        if (md.ok) bucket = kBMaxLog - m;
    }
    md.bucket = bucket;
    P.meta[i] = md;
    atomicAdd(&P.buckets[bucket], 1u);
}

__global__ void k_border(const BatchParams P)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        uint32_t acc = 0;
        for (int b = 0; b < kBuckets; ++b) {
            P.buckets[kBuckets + b] = acc;       // start
            P.buckets[2 * kBuckets + b] = 0;     // cursor
            acc += P.buckets[b];
        }
        *P.work = 0;
    }
}

__global__ void k_bscatter(const BatchParams P)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.count) return;
    const int b = P.meta[i].bucket;
    const uint32_t pos = P.buckets[kBuckets + b] + atomicAdd(&P.buckets[2 * kBuckets + b], 1u);
    P.order[pos] = i;
}

// sigma_d = r^(2^(D-1-d)) and the same for ri, with their 64-bit Shoup
// quotients, for d < D: the tile factors of plan.cu; thread d does level d.
// (Barrett products and quotients, M: this runs before every tile of a large
// instance while the CTA waits at the next barrier.)
__device__ __forceinline__ void tile_factors(uint32_t r, uint32_t ri, int D, const host::ModP &M, uint32_t *sg)
{
    const int d = threadIdx.x;
    if (d < D) {
        uint32_t s = r, si = ri;
        for (int k = 0; k < D - 1 - d; ++k) {
            s = M.mul(s, s);
            si = M.mul(si, si);
        }
        uint32_t *e = sg + d * 6;
        e[0] = s;
        M.quot64(s, e[1], e[2]);
        e[3] = si;
        M.quot64(si, e[4], e[5]);
    }
}

__device__ __forceinline__ Tw tw_of(uint32_t w, const host::ModP &M) { return Tw{w, M.quot32(w)}; }

// The top K levels of an instance of n = 2^m residues viewed as 2^K rows of
// C = n / 2^K columns: forward on both sides (row vector into c, vector into
// xs) with twiddles FT (heap order), or recombination of c with FIT.
// Several columns per iteration, both sides' loads issued before any
// arithmetic: up to 32 residues in flight per thread (16 when the columns
// are short), so that one DRAM latency serves both sides or several columns
// (CPI columns of 2^K rows each).  C, a
// power of two >= 2048, is a multiple of 256 CPI.
template <int K>
struct ColsShape {
    static constexpr int R = 1 << K;
    static constexpr bool BOTH = 2 * R <= 32;                     // both sides' loads together
    static constexpr int CPI = 2 * R <= 16 ? 16 / (2 * R) : 1;
    static constexpr int CPI_REC = R <= 16 ? 16 / R : 1;
};

template <int K>
__device__ void cols_fwd(const BatchParams &P, uint64_t off, uint32_t C, const Tw *FT, Tw kt)
{
    using Sh = ColsShape<K>;
    constexpr int R = Sh::R, CPI = Sh::CPI;
    const uint32_t p = P.p, p2 = 2 * P.p;
    for (uint32_t col0 = threadIdx.x; col0 < C; col0 += kBThreads * CPI) {
        uint32_t va[CPI][R], vx[Sh::BOTH ? CPI : 1][R];
#pragma unroll
        for (int c = 0; c < CPI; ++c) {
            const uint32_t col = col0 + c * kBThreads;
#pragma unroll
            for (int r = 0; r < R; ++r) va[c][r] = P.a[off + (uint64_t)r * C + col];
            if constexpr (Sh::BOTH) {
#pragma unroll
                for (int r = 0; r < R; ++r) vx[c][r] = P.x[off + (uint64_t)r * C + col];
            }
        }
#pragma unroll
        for (int c = 0; c < CPI; ++c) {
            const uint32_t col = col0 + c * kBThreads;
            uint32_t *v = va[c];
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = shoup_mul(v[r], kt.w, kt.wp, p);
#pragma unroll
            for (int l = 0; l < K; ++l) {
                const int h = R >> (l + 1);
#pragma unroll
                for (int j = 0; j < (1 << l); ++j)
#pragma unroll
                    for (int i = 0; i < h; ++i)
                        bfly_row(v[(j << (K - l)) + i], v[(j << (K - l)) + i + h], FT[(1 << l) + j], p, p2);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) P.c[off + (uint64_t)r * C + col] = v[r];
            uint32_t *w = vx[Sh::BOTH ? c : 0];
            if constexpr (!Sh::BOTH) {
#pragma unroll
                for (int r = 0; r < R; ++r) w[r] = P.x[off + (uint64_t)r * C + col];
            }
#pragma unroll
            for (int l = 0; l < K; ++l) {
                const int h = R >> (l + 1);
#pragma unroll
                for (int j = 0; j < (1 << l); ++j)
#pragma unroll
                    for (int i = 0; i < h; ++i)
                        bfly_vec(w[(j << (K - l)) + i], w[(j << (K - l)) + i + h], FT[(1 << l) + j], p, p2);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) P.xs[off + (uint64_t)r * C + col] = w[r];
        }
    }
}

template <int K>
__device__ void cols_rec(const BatchParams &P, uint64_t off, uint32_t C, const Tw *FIT)
{
    using Sh = ColsShape<K>;
    constexpr int R = Sh::R, CPI = Sh::CPI_REC;
    const uint32_t p = P.p, p2 = 2 * P.p;
    for (uint32_t col0 = threadIdx.x; col0 < C; col0 += kBThreads * CPI) {
        uint32_t v[CPI][R];
#pragma unroll
        for (int c = 0; c < CPI; ++c) {
            const uint32_t col = col0 + c * kBThreads;
#pragma unroll
            for (int r = 0; r < R; ++r) v[c][r] = P.c[off + (uint64_t)r * C + col];
        }
#pragma unroll
        for (int c = 0; c < CPI; ++c) {
            const uint32_t col = col0 + c * kBThreads;
#pragma unroll
            for (int l = K - 1; l >= 0; --l) {
                const int h = R >> (l + 1);
#pragma unroll
                for (int j = 0; j < (1 << l); ++j)
#pragma unroll
                    for (int i = 0; i < h; ++i)
                        bfly_rec(v[c][(j << (K - l)) + i], v[c][(j << (K - l)) + i + h], FIT[(1 << l) + j], p, p2);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) P.c[off + (uint64_t)r * C + col] = reduce_once(v[c][r], p);
        }
    }
}

__device__ void cols_dispatch(const BatchParams &P, int K, bool fwd, uint64_t off, uint32_t C, const Tw *FT,
                              const Tw *FIT, Tw kt)
{
    switch (K) {
    case 1: fwd ? cols_fwd<1>(P, off, C, FT, kt) : cols_rec<1>(P, off, C, FIT); break;
    case 2: fwd ? cols_fwd<2>(P, off, C, FT, kt) : cols_rec<2>(P, off, C, FIT); break;
    case 3: fwd ? cols_fwd<3>(P, off, C, FT, kt) : cols_rec<3>(P, off, C, FIT); break;
    case 4: fwd ? cols_fwd<4>(P, off, C, FT, kt) : cols_rec<4>(P, off, C, FIT); break;
    default: fwd ? cols_fwd<5>(P, off, C, FT, kt) : cols_rec<5>(P, off, C, FIT); break;
    }
}

struct BSmem {
    uint32_t SA[4096];
    uint32_t SX[4096];
    Tw STW[256];
    Tw SITW[256];
    uint32_t sg[12 * 6];
    Tw FT[32], FIT[32];
    uint32_t RT[32], RTi[32];
    uint32_t w;
};

__device__ void run_tile(const BatchParams &P, const TileJob &J, uint64_t N, int logT, const uint32_t *sg, Tw rho_t,
                         BSmem &S)
{
    if (logT == 12) {
        if (J.a.scaled)
            tile4096_dev<MODE_U32_S, MODE_U32>(J, (uint32_t)N, 0, sg, S.SA, S.SX, S.STW, S.SITW);
        else
            tile4096_dev<MODE_U32, MODE_U32>(J, (uint32_t)N, 0, sg, S.SA, S.SX, S.STW, S.SITW);
    } else {
        tile_generic_dev(J, N, 0, logT, logT - 1, sg, rho_t, S.SA);
    }
}

__device__ void process(const BatchParams &P, const host::ModP &M, uint32_t inst, BSmem &S)
{
    const BatchMeta md = P.meta[inst];
    if (!md.ok) return;
    const uint32_t p = P.p;
    const uint64_t off = P.offsets[inst];
    const int m = md.m;
    if (m == 0) {
        if (threadIdx.x == 0) P.c[off] = M.mul(P.a[off] % p, P.x[off] % p);
        return;
    }
    TileJob J;
    J.U = P.U;
    J.Ui = P.Ui;
    J.p = p;
    J.pinv = P.pinv;
    J.sig = nullptr;
    J.rho = nullptr;
    if (m <= P.big_log) {
        // one tile: factors of all L levels, leaf parameter rho when L = 0
        tile_factors(md.rho, md.rhoi, m - 1, M, S.sg);
        __syncthreads();
        J.a = Src{P.a + off, (uint64_t)1 << m, SRC_U32, 1, md.kt};
        J.x = Src{P.x + off, (uint64_t)1 << m, SRC_U32, 0, Tw{0, 0}};
        J.dst = P.c + off;
        J.store_lazy = 0;
        run_tile(P, J, (uint64_t)1 << m, m, S.sg, tw_of(md.rho, M), S);
        __syncthreads();
        return;
    }
    // out of core inside the CTA: top K levels, 2^K tiles, top K recombination
    const int L = m - 1, K = m - P.big_log, logT = P.big_log;
    const uint32_t C = 1u << logT;
    const int tid = threadIdx.x;
    if (tid > 0 && tid < (1 << K)) {
        const int l = 31 - __clz(tid);
        uint32_t r = md.rho, ri = md.rhoi;
        for (int k = 0; k < L - l - 1; ++k) {
            r = M.mul(r, r);
            ri = M.mul(ri, ri);
        }
        S.FT[tid] = tw_of(M.mul(r, P.U[tid]), M);
        S.FIT[tid] = tw_of(M.mul(ri, P.Ui[tid]), M);
    }
    if (tid >= 32 && tid < 32 + (1 << K)) {
        // tile root rho_t = rho Psi^brv_K(t), Psi a primitive 2^L-th root of unity
        const int t = tid - 32;
        const uint32_t Psi = M.pow(P.Om, 1ull << (P.v - L));
        const uint32_t b = host::bitrev(t, K);
        S.RT[t] = M.mul(md.rho, M.pow(Psi, b));
        S.RTi[t] = M.mul(md.rhoi, M.pow(M.inv(Psi), b));
    }
    __syncthreads();
    cols_dispatch(P, K, true, off, C, S.FT, S.FIT, md.kt);
    __syncthreads();
    for (int t = 0; t < (1 << K); ++t) {
        tile_factors(S.RT[t], S.RTi[t], logT - 1, M, S.sg);
        __syncthreads();
        const uint64_t toff = off + (uint64_t)t * C;
        J.a = Src{P.c + toff, C, SRC_U32, 0, Tw{0, 0}};
        J.x = Src{P.xs + toff, C, SRC_U32, 0, Tw{0, 0}};
        J.dst = P.c + toff;
        J.store_lazy = 1;
        run_tile(P, J, C, logT, S.sg, Tw{0, 0}, S);
        __syncthreads();
    }
    cols_dispatch(P, K, false, off, C, S.FT, S.FIT, md.kt);
    __syncthreads();
}

__global__ void __launch_bounds__(kBThreads, 4) k_bmain(const __grid_constant__ BatchParams P)
{
    __shared__ __align__(16) BSmem S;
    const host::ModP M(P.p);
    for (;;) {
        if (threadIdx.x == 0) S.w = atomicAdd(P.work, 1u);
        __syncthreads();
        const uint32_t w = S.w;
        __syncthreads();
        if (w >= P.count) break;
        process(P, M, P.order[w], S);
    }
}

}  // namespace

size_t batch_scratch_bytes(uint32_t count, uint64_t total_n)
{
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return al(total_n * 4) + al((size_t)count * sizeof(BatchMeta)) + al((size_t)count * 4) + al(3 * kBuckets * 4) + 256;
}

void batch_carve(void *scratch, uint32_t count, uint64_t total_n, BatchParams &P)
{
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    char *c = static_cast<char *>(scratch);
    P.xs = reinterpret_cast<uint32_t *>(c);
    c += al(total_n * 4);
    P.meta = reinterpret_cast<BatchMeta *>(c);
    c += al((size_t)count * sizeof(BatchMeta));
    P.order = reinterpret_cast<uint32_t *>(c);
    c += al((size_t)count * 4);
    P.buckets = reinterpret_cast<uint32_t *>(c);
    c += al(3 * kBuckets * 4);
    P.work = reinterpret_cast<uint32_t *>(c);
}

int batch_max_ctas_per_sm()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_bmain, kBThreads, 0) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    return n;
}

int launch_batched(const BatchParams &P, int ctas_per_sm, cudaStream_t s)
{
    if (P.count == 0) return FCIRC_OK;
    int dev = 0, sms = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    FCIRC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned g1 = (P.count + kBThreads - 1) / kBThreads;
    FCIRC_CUDA_TRY(cudaMemsetAsync(P.buckets, 0, kBuckets * 4, s));
    {
        ProfScope ps("k_bplan", s);
        k_bplan<<<g1, kBThreads, 0, s>>>(P);
        FCIRC_CUDA_TRY(cudaGetLastError());
    }
    {
        ProfScope ps("k_border", s);
        k_border<<<1, 32, 0, s>>>(P);
        FCIRC_CUDA_TRY(cudaGetLastError());
    }
    {
        ProfScope ps("k_bscatter", s);
        k_bscatter<<<g1, kBThreads, 0, s>>>(P);
        FCIRC_CUDA_TRY(cudaGetLastError());
    }
    {
        ProfScope ps("k_bmain", s);
        const unsigned grid = (unsigned)(sms * ctas_per_sm);
        k_bmain<<<grid, kBThreads, 0, s>>>(P);
        FCIRC_CUDA_TRY(cudaGetLastError());
    }
    return FCIRC_OK;
}

}  // namespace fcirc
