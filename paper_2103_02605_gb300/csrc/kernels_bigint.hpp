// kernels_bigint.hpp -- carry propagation of the large-integer product.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fcirc {

// Scratch bytes launch_carry needs for nlimbs output limbs.
size_t carry_scratch_bytes(uint64_t nlimbs);

// out[0..nlimbs) = base-2^16 digits of sum_k cols[k] 2^(16k), k < ncols
// (cols[k] < 2^56, ncols < nlimbs; the value must fit in nlimbs limbs).
int launch_carry(const uint64_t *cols, uint64_t ncols, uint16_t *out, uint64_t nlimbs, void *scratch,
                 cudaStream_t s);

}  // namespace fcirc
