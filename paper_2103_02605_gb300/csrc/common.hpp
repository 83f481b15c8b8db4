// common.hpp -- internal declarations shared by the library's translation
// units: status handling, the per-(device, stream) scratch pool and the
// plan cache.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/fcirc.h"
#include "modarith.cuh"

namespace fcirc {

// Thread-local detail string for fcirc_last_error().
void set_error(const char *fmt, ...);
int fail(int status, const char *fmt, ...);

#define FCIRC_CUDA_TRY(expr)                                                   \
    do {                                                                       \
        cudaError_t e_ = (expr);                                               \
        if (e_ != cudaSuccess)                                                 \
            return ::fcirc::fail(FCIRC_ECUDA, "%s: %s (%s:%d)", #expr,         \
                                 cudaGetErrorString(e_), __FILE__, __LINE__);  \
    } while (0)

#define FCIRC_TRY(expr)                                                        \
    do {                                                                       \
        int s_ = (expr);                                                       \
        if (s_ != FCIRC_OK) return s_;                                         \
    } while (0)

inline bool is_pow2(uint64_t n) { return n && !(n & (n - 1)); }
inline int ilog2(uint64_t n)
{
    int r = 0;
    while ((1ull << r) < n) ++r;
    return r;
}

// Scratch memory for one stream on the current device.  Returns a device
// pointer to at least `bytes` bytes, 256-byte aligned; valid until the next
// acquire on the same (device, stream) or fcirc_release().  Growth
// synchronises the device.
int scratch_acquire(cudaStream_t s, size_t bytes, void **out);

// Sticky device status word of the current device (one uint32 in device
// memory, 0 = OK), written by kernels whose bounded waits give up.
int device_status_word(uint32_t **out);

// Every device allocation of the library goes through dev_alloc, so that a
// test can make one of them fail (fcirc_debug_fail_alloc).
cudaError_t dev_alloc(void **ptr, size_t bytes);
void debug_fail_alloc(int k);

// Input checks (fcirc_set_checks): when on, check_lt launches a kernel that
// sets the device status word to FCIRC_EINVAL if any of the n words at v is
// >= bound; a no-op when off.
bool checks_on();
int check_lt(const uint32_t *v, uint64_t n, uint32_t bound, cudaStream_t s);
void set_checks(bool on);

// ---------------------------------------------------------------------------
// Plans.

// Per-prime constants and universal root-of-unity tables, cached per device.
// U[2^d + j] = psi_{2^(d+1)}^brv_d(j) (heap order), Ui its inverse, for
// d < kUnivLog; psi_m = Omega^(2^v / m) with Omega the fixed primitive
// 2^v-th root of unity of p.
constexpr int kUnivLog = 13;

struct PrimeTables {
    uint32_t p = 0, pinv = 0, omega = 0;
    int v = 0;                      // 2^v || p - 1
    uint32_t *d_U = nullptr, *d_Ui = nullptr;
};

int prime_tables(uint32_t p, const PrimeTables **out);

// Limits of the kernels.
constexpr int kTileLogMax = 12;     // tiles of up to 4096 residues in shared memory
constexpr int kPassLogMax = 12;     // strided passes of up to 12 levels
constexpr int kMaxLogN = 28;

// A plan for c = A x with A f-circulant of size n = 2^m over Z/pZ:
// L = m - 1 halving levels, then 2x2 leaves.  The top k levels run as
// strided passes over the whole array (passes[i] = [l0, l1)), the rest
// inside tiles of 2^logT contiguous residues (D = logT - 1 levels each).
struct Plan {
    uint32_t p = 0, f = 0;
    uint64_t n = 0;
    int m = 0, L = 0, k = 0, logT = 0, D = 0;
    int npass = 0;
    int pass_l0[4] = {0}, pass_l1[4] = {0};
    uint32_t rho = 0;               // 2^L-th root of f
    Tw kt{};                        // 2^32 * 2^-L mod p, for the leaf
    const PrimeTables *pt = nullptr;
    Tw *d_ftw = nullptr;            // [2^k] heap order s_{l,j}, l < k
    Tw *d_fitw = nullptr;           // [2^k] their inverses
    uint32_t *d_sig = nullptr;      // [2^k][D][6]: sigma, quotient hi, lo, and the same for sigma^-1
    Tw *d_rho = nullptr;            // [2^k] tile roots rho_t (used when D == 0)
    // the same top-level twiddles in group order, per strided pass (see
    // ColFwdJob in kernels_mod.hpp); offsets in entries
    Tw *d_gtw = nullptr, *d_gitw = nullptr;
    int pass_goff[4] = {0};
    int stage_off[4][3] = {{0}};
    // each pass's last stage again, ordered by slot pair (entry
    // 2 ((slot / 2) ngb + group block) + slot % 2), for the four-column
    // kernels: in that stage every thread has a group block of its own, and
    // this layout makes a warp's 128-bit loads of one slot pair contiguous;
    // offsets in entries
    Tw *d_gtwl = nullptr, *d_gitwl = nullptr;
    int pass_loff[4] = {0};
};

int get_plan(uint32_t p, uint32_t f, uint64_t n, const Plan **out);

// Host-side versions of the plan numbers (used by fcirc_plan.h).
int plan_node_twiddle_host(uint32_t p, uint32_t f, uint64_t n, int level,
                           uint64_t j, uint32_t *s, uint32_t *si);

void release_plans();
void release_scratch();

}  // namespace fcirc
