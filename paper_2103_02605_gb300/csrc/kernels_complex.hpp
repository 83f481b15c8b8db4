// kernels_complex.hpp -- parameter blocks of the complex FP32 kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fcirc {

struct CParams {
    const float *a, *x;
    float *c;
    const float2 *tw, *itw;
    uint64_t batch;
    float scale;   // 2^-L, the deferred halvings
};

struct CBwdParams {
    const float *a, *x, *g;
    float *grad_a, *grad_x;
    const float2 *tw_x, *itw_x;   // twiddles for 1/conj(f) (dL/dx)
    const float2 *tw_a, *itw_a;   // twiddles for conj(f) (dL/da)
    float fc_re, fc_im;           // conj(f)
    uint64_t batch;
    float scale;
};

// GF(p^2), p = 2^31 - 1 (gfp2.hpp): elements as (re, im) uint32 pairs.
struct GParams {
    const uint32_t *a, *x;
    uint32_t *c;
    const uint2 *tw, *itw;
    uint64_t batch;
    uint32_t scale;   // 2^-L mod p
};

int gf_tables(uint32_t fre, uint32_t fim, uint64_t n, const uint2 **tw, const uint2 **itw);

// Z/(2^K + 1), K = 64 W (ssa.cuh): elements of W + 1 uint64 words.
struct SParams {
    const uint64_t *a, *x;
    uint64_t *c;
    const int *tw, *itw;   // twiddle exponents mod 2K
    uint64_t batch;
    int scale_exp;         // 2^-L = 2^(2K - L)
};

int ssa_tables(uint32_t K, uint32_t fe, uint64_t n, const int **tw, const int **itw);
int launch_sfwd(const SParams &P, int K, int m, cudaStream_t s);
int launch_gfwd(const GParams &P, int m, cudaStream_t s);

// Twiddles s_{l,j} of the product with parameter f and size n (FP64
// rounded to FP32), cached per device.
int complex_tables(double fre, double fim, uint64_t n, const float2 **tw, const float2 **itw);
int launch_cfwd(const CParams &P, int m, cudaStream_t s);
int launch_cbwd(const CBwdParams &P, int m, cudaStream_t s);
void release_cplans();

}  // namespace fcirc
