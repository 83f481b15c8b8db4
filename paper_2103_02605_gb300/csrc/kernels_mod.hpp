// kernels_mod.hpp -- parameter blocks and launchers of the modular kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "modarith.cuh"

namespace fcirc {

constexpr int kTileThreads = 256;
constexpr int kStrThreads = 256;
constexpr int kStrSmemMax = 200 * 1024;

enum SrcKind { SRC_U32 = 0, SRC_U16_REV = 1, SRC_U16 = 2, SRC_U32_REV = 3 };

// Where a pass reads its input: a uint32 array (residues), or 16-bit
// coefficients zero-padded to the transform length, optionally reversed
// (a'[i] = P[N-1-i]) for the row vector of a polynomial product.  The first
// load of the row vector multiplies it by `scale` (2^32 2^-L, see leaf2).
struct Src {
    const void *ptr;
    uint64_t len;
    int kind;
    int scaled;
    Tw scale;
};

struct TileJob {
    Src a, x;
    uint32_t *dst;
    const uint32_t *sig;   // plan tile factors [tiles][D][6]
    const Tw *rho;         // plan tile roots
    const uint32_t *U, *Ui;
    uint32_t p, pinv;
    int store_lazy;
};

// What a 4096-residue tile computes.  TILE_FULL: both trees, the leaves and
// the recombination.  TILE_ROW: the row-vector tree only; J.dst receives the
// transformed row vector (the leaf operands of Algorithm 1's row side, lazy
// in [0, 4p)) for reuse with many vectors.  TILE_PLANNED: J.a is such a
// transformed row vector (read as it is); the vector tree, the leaves and
// the recombination.  TILE_SHIFT: TILE_FULL with the row vector shifted by
// one place in the leaves (bfly_rec_shift), which moves the product up by one
// entry when f = 1: the polynomial product's reversed-row embedding then
// needs no rotation of its output.
enum : int { TILE_FULL = 0, TILE_ROW = 1, TILE_PLANNED = 2, TILE_SHIFT = 3 };

// The tile-pair interleaved layout of the arrays between the column passes
// and the 4096-residue tile kernel.  Seen by the column passes, such an array
// is rows of 4096 residues, one row per tile.  Interleaved, rows 2t and
// 2t + 1 share one 8192-word block in which every 32-byte sector holds one
// column quad of both: residue i sits at ilv_pos(i), a permutation of bits
// 2..12 of i (bit 12, the tile's parity, moves to bit 2).  A column pass
// thread holding two adjacent rows of a quad then writes or reads whole
// 32-byte sectors; a tile reads and writes only the positions of its own
// residues, so it can work in place.
__host__ __device__ __forceinline__ uint32_t ilv_pos(uint32_t i)
{
    return (i & ~0x1FFFu) | (((i >> 12) & 1u) << 2) | ((i & 0xFFCu) << 1) | (i & 3u);
}

struct TileParams {
    TileJob job[3];
    uint64_t N;
    int logT, D;
    int var = 0;           // TILE_FULL / ROW / PLANNED / SHIFT (tile_dev.cuh); logT = 12 only
    // bit 0: the row-vector source, bit 1: the vector source and the
    // destination, are in the tile-pair interleaved layout (logT = 12 only)
    int ilv = 0;
    // With tma = 1 the interleaved sides and the destination move through
    // TMA tensor copies (tmap[job][0]: row vector, [1]: vector, [2]:
    // destination, tile_tma_maps); the loads' mbarrier wait gives up after
    // spin_limit probes and then reports FCIRC_ETIMEOUT in *status.
    int tma = 0;
    uint32_t spin_limit = 0;
    uint32_t *status = nullptr;
    CUtensorMap tmap[3][3];
};

// Fills P.tmap for the interleaved arrays of P's first njobs jobs and sets
// P.tma, P.spin_limit and P.status; leaves P.tma = 0 (scalar accesses) when
// the driver offers no tensor-map encoder.  tma_host.cu.
int tile_tma_maps(TileParams &P, int njobs);

struct StrFwdJob {
    Src src;
    uint32_t *dst;
    const Tw *ftw;
    uint32_t p;
    int vec_side;
};

struct StrFwdParams {
    StrFwdJob job[6];
    uint64_t N;
    int logn, l0, l1, logW;
};

struct StrInvJob {
    const uint32_t *src;
    uint32_t *dst;
    const Tw *fitw;
    uint32_t p;
};

// EPI_CRT_ROT: CRT of three primes, coefficient k taken from circulant entry
// k + 1 (the reversed-row embedding); EPI_CRT: CRT with entry k to
// coefficient k (the leaves already shifted the product, TILE_SHIFT).
enum Epilogue { EPI_CANON = 0, EPI_LAZY = 1, EPI_CRT_ROT = 2, EPI_CRT = 3 };

__host__ __device__ inline bool epi_crt(int e) { return e == EPI_CRT_ROT || e == EPI_CRT; }

// Garner constants for (p1, p2, p3).
struct CrtConsts {
    uint32_t p1, p2, p3;
    uint32_t m2, m3;       // floor(2^32 / p2), floor(2^32 / p3)
    Tw inv12;              // p1^-1 mod p2
    Tw p1m3;               // p1 mod p3
    Tw inv123;             // (p1 p2)^-1 mod p3
    uint64_t p1p2;
};

struct StrInvParams {
    StrInvJob job[3];
    int nprime;
    uint64_t N;
    int logn, l0, l1, logW;
    int epi;
    uint64_t *dst64;
    uint64_t nout;
    CrtConsts crt;
};

#if defined(__CUDACC__)
// Garner recombination of canonical residues r_i mod p_i into the integer
// x < p1 p2 p3 with x = r_i (mod p_i); returned modulo 2^64 (exact whenever
// x < 2^64, which holds for every coefficient the library produces).
__device__ __forceinline__ uint64_t crt3(uint32_t r1, uint32_t r2, uint32_t r3, const CrtConsts &C)
{
    // Garner: x = r1 + p1 t2 + p1 p2 t3 with x = r_i (mod p_i), all r_i canonical
    const uint32_t r1m2 = reduce_once(shoup_mul(r1, 1u, C.m2, C.p2), C.p2);
    const uint32_t t2 = reduce_once(shoup_mul(r2 + C.p2 - r1m2, C.inv12.w, C.inv12.wp, C.p2), C.p2);
    const uint32_t r1m3 = reduce_once(shoup_mul(r1, 1u, C.m3, C.p3), C.p3);
    uint32_t u = r1m3 + reduce_once(shoup_mul(t2, C.p1m3.w, C.p1m3.wp, C.p3), C.p3);
    u = reduce_once(u, C.p3);
    const uint32_t t3 = reduce_once(shoup_mul(r3 + C.p3 - u, C.inv123.w, C.inv123.wp, C.p3), C.p3);
    return (uint64_t)r1 + (uint64_t)C.p1 * t2 + C.p1p2 * (uint64_t)t3;
}
#endif

// Register-staged column passes (kernels_fast.cu).  gtw: this pass's
// twiddles in group order -- for stage s, group block gb (the level-d0 node
// the group lies in), 16 entries at gtw[stage_off[s] + 16 gb]: local level
// d node j at slot 16 - 2^(d+1) + j (levels 3, 2, 1, 0 at slots 0-7, 8-11,
// 12-13, 14), so that each level is read with 128-bit loads.
struct ColFwdJob {
    Src src;
    uint32_t *dst;
    const Tw *gtw;
    uint32_t p;
    int vec_side;
    int half;              // 0; 1: input zero below N/2; 2: input zero from N/2 (and s = 1 at level 0)
    // the pass's last stage ordered by slot pair (Plan::d_gtwl): entry
    // 2 ((slot / 2) ngb + gb) + slot % 2 for the ngb = 2^(l0 + d0) group
    // blocks of that stage; the four-column kernels read that stage from here
    const Tw *gtwl;
};

struct ColFwdParams {
    ColFwdJob job[6];
    int jobs_per_cta;      // 1, or 3 for the three primes of one side of a product
    int vec_group0;        // job groups [0, vec_group0) are row-vector side (set by the launcher)
    int share_src;         // every job group reads one source (set by the launcher)
    uint32_t N;
    int logn, l0, l1;
    int stage_off[3];
    int ilv;               // write the tile-pair interleaved layout (ilv_pos); col4_fwd_ilv_ok
    // the interleaved output of a 12-level pass through TMA tensor stores
    // (fwd_tma_maps): one map per job over its destination, boxes of one
    // column quad of 256 row pairs 8 t + k, dense in shared memory
    int tma_st;
    CUtensorMap tmap[6];
};

// Tensor maps of the forward pass's interleaved destinations; sets
// P.tma_st when every job's map could be made (tma_host.cu).
int fwd_tma_maps(ColFwdParams &P, int njobs, int lf);

struct ColInvJob {
    const uint32_t *src;
    uint32_t *dst;
    const Tw *gitw;
    uint32_t p;
    const Tw *gitwl;       // the last stage by slot pair (see ColFwdJob::gtwl)
};

struct ColInvParams {
    ColInvJob job[3];
    int nprime;
    uint32_t N;
    int logn, l0, l1;
    int stage_off[3];
    int ilv;               // read the tile-pair interleaved layout (ilv_pos); col4_inv_ilv_ok
    int epi;
    uint64_t *dst64;
    uint64_t nout;
    CrtConsts crt;
};

int launch_tile(const TileParams &P, uint64_t ntiles, int njobs, cudaStream_t s);
int launch_strided_fwd(const StrFwdParams &P, int njobs, cudaStream_t s);
int launch_strided_inv(const StrInvParams &P, cudaStream_t s);
int launch_embed(const uint32_t *u, const uint32_t *t, const uint32_t *x, uint64_t n, uint64_t N, Tw f, uint32_t p,
                 int toeplitz, uint32_t *ap, uint32_t *bp, cudaStream_t s);
int launch_rot_scale(const uint32_t *src, uint32_t *dst, uint64_t n, Tw f, uint32_t p, cudaStream_t s);
int launch_crt_rot(const uint32_t *r1, const uint32_t *r2, const uint32_t *r3, uint64_t N,
                   uint64_t *out, uint64_t nout, const CrtConsts &C, cudaStream_t s);
// register-staged kernels (kernels_fast.cu) for the shapes they cover
bool fast_tile_ok(int logT);
bool fast_col_ok(int lf, int logS);
int launch_tile_fast(const TileParams &P, uint64_t ntiles, int njobs, cudaStream_t s);
int launch_colfwd(const ColFwdParams &P, int nctay, cudaStream_t s);
int launch_colinv(const ColInvParams &P, cudaStream_t s);
// four columns per thread (kernels_col4.cu); used when these accept the pass
bool col4_fwd_ok(const ColFwdParams &P, int nctay);
bool col4_inv_ok(const ColInvParams &P);
// whether the four-column kernels can write (forward) / read (inverse) the
// tile-pair interleaved layout for this pass: the pass borders the tiles
// (2^12 columns) and its arrays are 32-byte aligned
bool col4_fwd_ilv_ok(const ColFwdParams &P, int nctay);
bool col4_inv_ilv_ok(const ColInvParams &P);
int launch_colfwd4(const ColFwdParams &P, int nctay, cudaStream_t s);
int launch_colinv4(const ColInvParams &P, cudaStream_t s);
// stage split of a column pass of lf levels: the first stage takes lf mod 4
// (or 4), the others 4 levels each
inline int col_nstage(int lf) { return (lf + 3) / 4; }
inline int col_nl(int lf, int s) { return s == 0 ? lf - 4 * (col_nstage(lf) - 1) : 4; }
inline int col_d0(int lf, int s) { return s == 0 ? 0 : col_nl(lf, 0) + 4 * (s - 1); }
int launch_scalar(const uint32_t *a, const uint32_t *x, uint32_t *c, uint32_t p, cudaStream_t s);

}  // namespace fcirc
