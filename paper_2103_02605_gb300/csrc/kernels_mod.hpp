// kernels_mod.hpp -- parameter blocks and launchers of the modular kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "modarith.cuh"

namespace fcirc {

constexpr int kTileThreads = 256;
constexpr int kStrThreads = 256;
constexpr int kStrSmemMax = 200 * 1024;

enum SrcKind { SRC_U32 = 0, SRC_U16_REV = 1, SRC_U16 = 2 };

// Where a pass reads its input: a uint32 array (residues), or 16-bit
// coefficients zero-padded to the transform length, optionally reversed
// (a'[i] = P[N-1-i]) for the row vector of a polynomial product.
struct Src {
    const void *ptr;
    uint64_t len;
    int kind;
};

struct TileJob {
    Src a, x;
    uint32_t *dst;
    const uint32_t *sig;   // plan tile factors [tiles][D][6]
    const Tw *rho;         // plan tile roots
    const uint32_t *U, *Ui;
    uint32_t p, pinv;
    Tw kt;
    int store_lazy;
};

struct TileParams {
    TileJob job[3];
    uint64_t N;
    int logT, D;
};

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

enum Epilogue { EPI_CANON = 0, EPI_LAZY = 1, EPI_CRT_ROT = 2 };

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

int launch_tile(const TileParams &P, uint64_t ntiles, int njobs, cudaStream_t s);
int launch_strided_fwd(const StrFwdParams &P, int njobs, cudaStream_t s);
int launch_strided_inv(const StrInvParams &P, cudaStream_t s);
int launch_crt_rot(const uint32_t *r1, const uint32_t *r2, const uint32_t *r3, uint64_t N,
                   uint64_t *out, uint64_t nout, const CrtConsts &C, cudaStream_t s);
int launch_scalar(const uint32_t *a, const uint32_t *x, uint32_t *c, uint32_t p, cudaStream_t s);

}  // namespace fcirc
