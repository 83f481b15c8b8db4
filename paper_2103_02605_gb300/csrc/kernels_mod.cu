// kernels_mod.cu -- sm_103a kernels of the modular f-circulant product
// (Algorithm 1, Section 2) and of its polynomial / large-integer uses
// (Section 3).
//
// Data layout: the recursion works IN PLACE in natural order.  Node j of
// level l owns the contiguous block [j n/2^l, (j+1) n/2^l); its halving step
// pairs element i of the first half with element i of the second half.  So
// the top levels pair far-apart elements and the bottom levels near ones:
//
//  * k_strided_fwd / k_strided_inv: levels [l0, l1) of the whole array.
//    The array is viewed, per level-l0 block, as 2^(l1-l0) rows of stride
//    n/2^l1; a CTA stages 2^(l1-l0) rows x W adjacent columns in shared
//    memory (coalesced row segments) and runs all those levels there.
//  * k_tile: a CTA owns one contiguous tile of 2^logT residues (a node of
//    level k = m - logT) and runs every remaining level of both input sides,
//    the 2x2 leaf products and the recombination back up to level k.
//
// Twiddles: the strided passes read the stored s_{l,j}; the tile kernel
// generates its 2^(logT-1) - 1 twiddles (and inverses) from the universal
// root table and two per-tile factors (see plan.cu), so no table of size n
// is ever read.
#include <atomic>

#include <cstdlib>
#include "common.hpp"
#include "kernels_mod.hpp"
#include "prof.hpp"
#include "tile_dev.cuh"

namespace fcirc {

// ---------------------------------------------------------------------------
// tile kernel

__global__ void __launch_bounds__(kTileThreads)
k_tile(const __grid_constant__ TileParams P)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const TileJob &J = P.job[blockIdx.y];
    const uint64_t t = blockIdx.x;
    const Tw rho_t = P.D == 0 ? J.rho[t] : Tw{0, 0};
    tile_generic_dev(J, P.N, t << P.logT, P.logT, P.D, J.sig + t * (uint64_t)(P.D > 0 ? P.D : 1) * 6, rho_t, smem);
}

// ---------------------------------------------------------------------------
// strided passes

__global__ void __launch_bounds__(kStrThreads)
k_strided_fwd(const __grid_constant__ StrFwdParams P)
{
    extern __shared__ __align__(16) uint32_t tile[];
    const StrFwdJob &J = P.job[blockIdx.y];
    const int logR = P.l1 - P.l0, logW = P.logW;
    const int R = 1 << logR, W = 1 << logW, RW = R << logW;
    const int logS = P.logn - P.l1;
    const uint64_t cg_per_blk = (uint64_t)1 << (logS - logW);
    const uint64_t blk = blockIdx.x / cg_per_blk, cg = blockIdx.x % cg_per_blk;
    const uint64_t base = (blk << (P.logn - P.l0)) + (cg << logW);
    const uint32_t p = J.p, p2 = 2 * J.p;

    for (int e = threadIdx.x; e < RW; e += blockDim.x) {
        const int r = e >> logW, w = e & (W - 1);
        tile[e] = load_src(J.src, P.N, base + ((uint64_t)r << logS) + w, p);
    }
    __syncthreads();
    for (int d = 0; d < logR; ++d) {
        const int lh = logR - d - 1;
        const int half = 1 << lh;
        const Tw *lev = J.ftw + ((uint64_t)1 << (P.l0 + d)) + (blk << d);
        for (int bb = threadIdx.x; bb < (RW >> 1); bb += blockDim.x) {
            const int w = bb & (W - 1), rb = bb >> logW;
            const int jn = rb >> lh, i = rb & (half - 1);
            const int rlo = (jn << (lh + 1)) + i, rhi = rlo + half;
            const Tw s = lev[jn];
            uint32_t u = tile[(rlo << logW) + w], v = tile[(rhi << logW) + w];
            if (J.vec_side)
                bfly_vec(u, v, s, p, p2);
            else
                bfly_row(u, v, s, p, p2);
            tile[(rlo << logW) + w] = u;
            tile[(rhi << logW) + w] = v;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < RW; e += blockDim.x) {
        const int r = e >> logW, w = e & (W - 1);
        J.dst[base + ((uint64_t)r << logS) + w] = tile[e];
    }
}


__global__ void __launch_bounds__(kStrThreads)
k_strided_inv(const __grid_constant__ StrInvParams P)
{
    extern __shared__ __align__(16) uint32_t tile[];
    const int logR = P.l1 - P.l0, logW = P.logW;
    const int R = 1 << logR, W = 1 << logW, RW = R << logW;
    const int logS = P.logn - P.l1;
    const uint64_t cg_per_blk = (uint64_t)1 << (logS - logW);
    const uint64_t blk = blockIdx.x / cg_per_blk, cg = blockIdx.x % cg_per_blk;
    const uint64_t base = (blk << (P.logn - P.l0)) + (cg << logW);

    for (int q = 0; q < P.nprime; ++q) {
        const StrInvJob &J = P.job[q];
        uint32_t *tq = tile + q * RW;
        for (int e = threadIdx.x; e < RW; e += blockDim.x) {
            const int r = e >> logW, w = e & (W - 1);
            tq[e] = J.src[base + ((uint64_t)r << logS) + w];
        }
    }
    __syncthreads();
    for (int d = logR - 1; d >= 0; --d) {
        const int lh = logR - d - 1;
        const int half = 1 << lh;
        for (int q = 0; q < P.nprime; ++q) {
            const StrInvJob &J = P.job[q];
            const uint32_t p = J.p, p2 = 2 * J.p;
            uint32_t *tq = tile + q * RW;
            const Tw *lev = J.fitw + ((uint64_t)1 << (P.l0 + d)) + (blk << d);
            for (int bb = threadIdx.x; bb < (RW >> 1); bb += blockDim.x) {
                const int w = bb & (W - 1), rb = bb >> logW;
                const int jn = rb >> lh, i = rb & (half - 1);
                const int rlo = (jn << (lh + 1)) + i, rhi = rlo + half;
                uint32_t m1 = tq[(rlo << logW) + w], m2 = tq[(rhi << logW) + w];
                bfly_rec(m1, m2, lev[jn], p, p2);
                tq[(rlo << logW) + w] = m1;
                tq[(rhi << logW) + w] = m2;
            }
        }
        __syncthreads();
    }
    if (epi_crt(P.epi)) {
        const uint64_t mask = P.N - 1, rot = P.epi == EPI_CRT_ROT ? mask : 0u;
        for (int e = threadIdx.x; e < RW; e += blockDim.x) {
            const int r = e >> logW, w = e & (W - 1);
            const uint64_t idx = base + ((uint64_t)r << logS) + w;
            const uint64_t dst = (idx + rot) & mask;   // EPI_CRT_ROT: coefficient k is circulant entry k + 1
            if (dst < P.nout) {
                const uint32_t r1 = reduce_once(tile[e], P.job[0].p);
                const uint32_t r2 = reduce_once(tile[RW + e], P.job[1].p);
                const uint32_t r3 = reduce_once(tile[2 * RW + e], P.job[2].p);
                P.dst64[dst] = crt3(r1, r2, r3, P.crt);
            }
        }
    } else {
        for (int q = 0; q < P.nprime; ++q) {
            const StrInvJob &J = P.job[q];
            const uint32_t *tq = tile + q * RW;
            for (int e = threadIdx.x; e < RW; e += blockDim.x) {
                const int r = e >> logW, w = e & (W - 1);
                uint32_t v = tq[e];
                J.dst[base + ((uint64_t)r << logS) + w] =
                    P.epi == EPI_CANON ? reduce_once(v, J.p) : v;
            }
        }
    }
}

// CRT of three canonical residue arrays of length N into out[(i-1) mod N]
// (the product with the reversed-row embedding is rotated by one).
__global__ void k_crt_rot(const uint32_t *r1, const uint32_t *r2, const uint32_t *r3, uint64_t N,
                          uint64_t *out, uint64_t nout, CrtConsts C)
{
    const uint64_t mask = N - 1;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t dst = (i + mask) & mask;
        if (dst < nout) out[dst] = crt3(r1[i], r2[i], r3[i], C);
    }
}

// n = 1: c_0 = a_0 x_0 (the 1x1 f-circulant is the scalar a_0).
__global__ void k_scalar(const uint32_t *a, const uint32_t *x, uint32_t *c, uint32_t p)
{
    if (threadIdx.x == 0 && blockIdx.x == 0)
        c[0] = (uint32_t)((uint64_t)a[0] * x[0] % p);
}

// ---------------------------------------------------------------------------
// launchers

// Opt a kernel into more than 48 KB of dynamic shared memory, once per device.
template <class K>
static int ensure_smem(K kernel, int bytes, std::atomic<unsigned> &mask)
{
    int dev = 0;
    FCIRC_CUDA_TRY(cudaGetDevice(&dev));
    const unsigned bit = 1u << (dev & 31);
    if (mask.load() & bit) return FCIRC_OK;
    FCIRC_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    mask.fetch_or(bit);
    return FCIRC_OK;
}

int launch_tile(const TileParams &P, uint64_t ntiles, int njobs, cudaStream_t s)
{
    const size_t smem = (size_t)16 << P.logT;
    static std::atomic<unsigned> mask{0};
    FCIRC_TRY(ensure_smem(k_tile, 16 << kTileLogMax, mask));
    dim3 grid((unsigned)ntiles, njobs);
    ProfScope ps("k_tile", s);
    k_tile<<<grid, kTileThreads, smem, s>>>(P);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

static uint64_t str_grid(int logn, int l0, int l1, int logW)
{
    return (uint64_t)1 << (l0 + (logn - l1) - logW);
}

int launch_strided_fwd(const StrFwdParams &P, int njobs, cudaStream_t s)
{
    const size_t smem = (size_t)4 << (P.l1 - P.l0 + P.logW);
    static std::atomic<unsigned> mask{0};
    FCIRC_TRY(ensure_smem(k_strided_fwd, kStrSmemMax, mask));
    dim3 grid((unsigned)str_grid(P.logn, P.l0, P.l1, P.logW), njobs);
    ProfScope ps("k_strided_fwd", s);
    k_strided_fwd<<<grid, kStrThreads, smem, s>>>(P);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

int launch_strided_inv(const StrInvParams &P, cudaStream_t s)
{
    const size_t smem = (size_t)P.nprime * ((size_t)4 << (P.l1 - P.l0 + P.logW));
    static std::atomic<unsigned> mask{0};
    FCIRC_TRY(ensure_smem(k_strided_inv, kStrSmemMax, mask));
    dim3 grid((unsigned)str_grid(P.logn, P.l0, P.l1, P.logW));
    ProfScope ps("k_strided_inv", s);
    k_strided_inv<<<grid, kStrThreads, smem, s>>>(P);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

int launch_crt_rot(const uint32_t *r1, const uint32_t *r2, const uint32_t *r3, uint64_t N,
                   uint64_t *out, uint64_t nout, const CrtConsts &C, cudaStream_t s)
{
    unsigned blocks = (unsigned)((N + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    ProfScope ps("k_crt_rot", s);
    k_crt_rot<<<blocks, 256, 0, s>>>(r1, r2, r3, N, out, nout, C);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

// Transposed product from the row product of the reversed row vector with
// parameter f^-1: d[n-1] = c'[0], d[j] = f c'[j+1] (canonical in and out).
__global__ void k_rot_scale(const uint32_t *src, uint32_t *dst, uint64_t n, Tw f, uint32_t p)
{
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x)
        dst[j] = j + 1 < n ? reduce_once(shoup_mul(src[j + 1], f.w, f.wp, p), p) : src[0];
}

// Corollary 1 embedding of an n x n product into a power-of-two circulant of
// size N >= 2n - 1 (parameter 1): a'[k] = u[k] for k < n, a'[N - m] = the
// wrapped entry m (1 <= m < n), zero elsewhere; b' = x followed by zeros.
// Wrapped entry m: f u[n - m] (f-circulant, toeplitz = 0) or t[n - 1 - m],
// t the 2n - 1 diagonals of a Toeplitz matrix (toeplitz = 1, u = t + n - 1).
__global__ void k_embed(const uint32_t *u, const uint32_t *t, const uint32_t *x, uint64_t n, uint64_t N, Tw f,
                        uint32_t p, int toeplitz, uint32_t *ap, uint32_t *bp)
{
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < N; k += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t av = 0;
        if (k < n) {
            av = u[k];
        } else if (k > N - n) {
            const uint64_t m = N - k;   // 1 <= m < n
            av = toeplitz ? t[n - 1 - m] : reduce_once(shoup_mul(u[n - m], f.w, f.wp, p), p);
        }
        ap[k] = av;
        bp[k] = k < n ? x[k] : 0u;
    }
}

int launch_embed(const uint32_t *u, const uint32_t *t, const uint32_t *x, uint64_t n, uint64_t N, Tw f, uint32_t p,
                 int toeplitz, uint32_t *ap, uint32_t *bp, cudaStream_t s)
{
    unsigned blocks = (unsigned)((N + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    ProfScope ps("k_embed", s);
    k_embed<<<blocks, 256, 0, s>>>(u, t, x, n, N, f, p, toeplitz, ap, bp);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

int launch_rot_scale(const uint32_t *src, uint32_t *dst, uint64_t n, Tw f, uint32_t p, cudaStream_t s)
{
    unsigned blocks = (unsigned)((n + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    ProfScope ps("k_rot_scale", s);
    k_rot_scale<<<blocks, 256, 0, s>>>(src, dst, n, f, p);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

// Input check (fcirc_set_checks): any word >= bound sets the status word.
__global__ void k_check_lt(const uint32_t *v, uint64_t n, uint32_t bound, uint32_t *status)
{
    bool bad = false;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        bad = bad || v[i] >= bound;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicCAS(status, 0u, (uint32_t)FCIRC_EINVAL);
}

namespace {
std::atomic<int> g_checks{-1};   // -1: not yet read from the environment
}

bool checks_on()
{
    int c = g_checks.load();
    if (c < 0) {
        const char *e = std::getenv("FCIRC_CHECKS");
        c = (e && e[0] && e[0] != '0') ? 1 : 0;
        int expect = -1;
        g_checks.compare_exchange_strong(expect, c);
        c = g_checks.load();
    }
    return c == 1;
}

void set_checks(bool on) { g_checks.store(on ? 1 : 0); }

int check_lt(const uint32_t *v, uint64_t n, uint32_t bound, cudaStream_t s)
{
    if (!checks_on() || n == 0) return FCIRC_OK;
    uint32_t *status;
    FCIRC_TRY(device_status_word(&status));
    unsigned blocks = (unsigned)((n + 255) / 256);
    if (blocks > 152 * 4) blocks = 152 * 4;
    ProfScope ps("k_check_lt", s);
    k_check_lt<<<blocks, 256, 0, s>>>(v, n, bound, status);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

int launch_scalar(const uint32_t *a, const uint32_t *x, uint32_t *c, uint32_t p, cudaStream_t s)
{
    ProfScope ps("k_scalar", s);
    k_scalar<<<1, 32, 0, s>>>(a, x, c, p);
    FCIRC_CUDA_TRY(cudaGetLastError());
    return FCIRC_OK;
}

}  // namespace fcirc
