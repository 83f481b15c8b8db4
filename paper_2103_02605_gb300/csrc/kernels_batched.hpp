// kernels_batched.hpp -- the persistent batched product (kernels_batched.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "modarith.cuh"

namespace fcirc {

// Per-instance plan written by the plan kernel.
struct BatchMeta {
    uint32_t ok, m, bucket;
    uint32_t rho, rhoi;   // 2^L-th root of f and its inverse
    Tw kt;                // 2^32 2^-L, the row vector's load scale (see leaf2)
    uint32_t pad;
};

struct BatchParams {
    uint32_t p, pinv, Om;
    int v;
    const uint32_t *U, *Ui;
    const uint32_t *f;
    const uint64_t *offsets;
    const uint32_t *a, *x;
    uint32_t *c;
    uint32_t count;
    uint64_t total;       // offsets[count]: every instance must lie in [0, total)
    int big_log;          // instances above 2^big_log run as 2^big_log tiles (11 or 12)
    // scratch (batch_carve)
    uint32_t *xs;
    BatchMeta *meta;
    uint32_t *order, *buckets, *work;
    uint32_t *status;
};

size_t batch_scratch_bytes(uint32_t count, uint64_t total_n);
void batch_carve(void *scratch, uint32_t count, uint64_t total_n, BatchParams &P);
// resident CTAs per SM of the persistent kernel (-1 on error)
int batch_max_ctas_per_sm();
int launch_batched(const BatchParams &P, int ctas_per_sm, cudaStream_t s);

}  // namespace fcirc
