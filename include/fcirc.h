/*
 * fcirc.h -- C ABI of the GB300 (sm_103a) f-circulant library.
 *
 * The library multiplies an f-circulant matrix by a vector without an FFT,
 * by the recursive halving of Rosowski, "On Fast Computation of a Circulant
 * Matrix-Vector Product" (arXiv 2103.02605), Algorithm 1 and Theorem 1
 * (Section 2), and uses that product for the two applications of Section 3:
 * integer polynomial multiplication (Section 3.1) and large-integer
 * multiplication (Section 3.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Matrix layout (Definition 2, Section 1.2, and the 3x3 example after it):
 *    an f-circulant n x n matrix A is given by its ROW vector a[0..n-1]
 *    (Section 1.2, last paragraph): A[i][j] = a[j-i] for j >= i and
 *    A[i][j] = f * a[n+j-i] for j < i, so c = A x is
 *        c[i] = sum_k a[k] * x[(i+k) mod n] * f^[i+k >= n].
 *  * Memory: every array argument may be a DEVICE pointer (any CUDA
 *    allocation on the current device) or a HOST pointer (pageable or
 *    pinned).  The caller allocates and owns all of them; the library never
 *    frees or keeps them.  With device pointers only, the call enqueues its
 *    kernels on `stream` and returns without waiting.  Host arrays are
 *    staged through device memory on `stream`.  If any of them is pageable,
 *    the call returns after the results are back in the caller's buffers.
 *    If all of them are page-locked (cudaHostAlloc / cudaHostRegister), the
 *    call is asynchronous like cudaMemcpyAsync: it returns at once, host
 *    inputs must stay unchanged and host outputs are valid only once
 *    `stream` has passed the call (so independent products on two streams
 *    overlap one's copies with the other's kernels).
 *  * stream: a cudaStream_t passed as void* (NULL = the legacy default
 *    stream) on the current device.
 *  * Scratch: kept in a per-device pool inside the library, grown on demand
 *    (growth synchronises the device) and released by fcirc_release().
 *    Plans (root chains and twiddle tables) are cached per (device, p, f, n).
 *    The first call for a new size or f builds its plan synchronously, so
 *    make it before capturing a stream into a CUDA graph.
 *  * Return value: an fcirc_status code.  No C++ exception crosses the ABI.
 *    fcirc_error_string() names a code; fcirc_last_error() gives a one-line
 *    detail for the calling thread's last failure.
 *  * Outputs never alias inputs.
 */
#ifndef FCIRC_H
#define FCIRC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum fcirc_status {
    FCIRC_OK = 0,
    FCIRC_EINVAL = 1,   /* bad size, null pointer, p not an odd prime < 2^30 */
    FCIRC_ENOROOT = 2,  /* a root required by Theorem 1 does not exist mod p */
    FCIRC_ENOMEM = 3,   /* device allocation failed */
    FCIRC_ECUDA = 4,    /* a CUDA runtime call failed (see fcirc_last_error) */
    FCIRC_ETIMEOUT = 5  /* a bounded device-side wait gave up */
};

/*
 * fcirc_matvec -- c = A x for the f-circulant A with row vector a, over
 * Z/pZ (Section 2: Theorem 1, Algorithm 1; Definition 2 for the layout).
 *
 *   p     odd prime, 3 <= p < 2^30.
 *   f     the circulant parameter, 1 <= f < p (f = 1: ordinary circulant).
 *   a, x  n residues each, in [0, p) (row vector and vector).
 *   c     n residues out, canonical in [0, p).
 *   n     1 <= n.  A power of two runs Algorithm 1 directly: then
 *         n <= 2^(v+1) where 2^v is the largest power of two dividing p-1
 *         (the recursion halves down to 2x2 blocks, so it needs
 *         2^(log2 n - 1)-th roots of unity), and n <= 2^28.  Any other n
 *         goes through Corollary 1 (below).
 *
 * Errors: FCIRC_EINVAL for a null pointer, n = 0 or too large, or p out of
 * range / not prime; FCIRC_ENOROOT when n is a power of two and f = 0 or f
 * has no (n/2)-th root mod p (Theorem 1 needs a root of f at every level).
 * Results for entries outside [0, p) are unspecified (never out of bounds).
 */
int fcirc_matvec(uint32_t p, uint32_t f, const uint32_t *a, const uint32_t *x,
                 uint32_t *c, uint64_t n, void *stream);

/*
 * (fcirc_matvec, continued) n that is not a power of two (Corollary 1):
 * the product is the first n entries of an ordinary circulant (f = 1)
 * product of size N, the power of two with N >= 2n - 1, whose row vector is
 * a[0..n) | zeros | f a[1..n) and whose vector is x | zeros (the corollary
 * takes N = 2^(d+1) with 2^d > n; any N >= 2n - 1 leaves the gap it needs).
 * It needs only the roots of unity of N and no root of f, so every
 * 0 <= f < p is accepted; n is limited by N <= 2^28 and by the 2-adic
 * order of p - 1 (FCIRC_ENOROOT).  Scratch: 16 N bytes.
 */

/*
 * fcirc_toeplitz_matvec -- c = T x over Z/pZ for the n x n Toeplitz matrix
 * T[i][j] = t[j - i + n - 1] (t holds the 2n - 1 diagonals, from the lowest
 * t[0] = T[n-1][0] to the highest t[2n-2] = T[0][n-1]), any n >= 1.  The
 * paper's introduction recalls that Toeplitz products reduce to circulant
 * ones; this is Corollary 1's embedding with the wrapped part of the row
 * vector taken from the lower diagonals.  Memory, errors and
 * synchronisation as for fcirc_matvec.
 */
int fcirc_toeplitz_matvec(uint32_t p, const uint32_t *t, const uint32_t *x, uint32_t *c, uint64_t n,
                          void *stream);

/*
 * fcirc_matvec_t -- c = A^T x for the same f-circulant A (row vector a):
 * the column convention, c[j] = sum_i A[i][j] x[i], which is the product
 * a(z) x(z) mod (z^n - f) of the two vectors read as polynomials (Section
 * 1.2 relates the two conventions; Section 3.1 uses this one).  Arguments,
 * memory, errors and synchronisation as for fcirc_matvec.
 *
 * It runs the row-convention product of Algorithm 1 with parameter f^-1 on
 * the reversed row vector (a[n-1-k], read reversed by the first pass, no
 * copy) and stores that result rotated by one and scaled by f:
 * c[n-1] = c'[0], c[j] = f c'[j+1].
 */
int fcirc_matvec_t(uint32_t p, uint32_t f, const uint32_t *a, const uint32_t *x,
                   uint32_t *c, uint64_t n, void *stream);

/*
 * fcirc_matvec_noalloc -- the same product as fcirc_matvec for callers that
 * cannot let the library allocate device memory (a process that reserved
 * its GPU memory in fixed pools up front, or that must not see the
 * device-wide synchronisation an allocation can cause while its streams
 * run).  The paper has no counterpart; this is an interface variant only.
 *
 * Arguments and results are those of fcirc_matvec, with three limits:
 *   * a, x, c must be device pointers on the current device (FCIRC_EINVAL
 *     otherwise: host buffers would need staging memory);
 *   * 2 <= n <= 2^20 (FCIRC_EINVAL beyond, with a message naming the limit);
 *   * the call never allocates: its scratch (the vector side's intermediate)
 *     and its plan tables live in one 5 MiB array inside the library that
 *     every GPU loading the library holds until the process exits.
 *
 * All calls on a device share that array, and it keeps the last call's
 * tables and intermediate: calls whose work overlaps on the GPU (two streams,
 * or two host threads) race with each other and must be serialised by the
 * caller.  A call for a new (p, f, n) writes its tables with a host-to-device
 * copy on `stream` before its kernels; nothing else needs clearing, since
 * every scratch word is written before it is read.  The first call on each
 * device also looks up the array's device address (once per device, with
 * that device current); make that first call before capturing any stream
 * into a CUDA graph.
 *
 * Which tables the array holds is remembered on the host, so a call made
 * while `stream` is being captured into a graph returns FCIRC_EINVAL and
 * enqueues nothing.  Unlike the other entry points it runs no input range
 * check under fcirc_set_checks(1): that check reports through a status word
 * the library would have to allocate.  Inputs must be < p.
 */
int fcirc_matvec_noalloc(uint32_t p, uint32_t f, const uint32_t *a, const uint32_t *x,
                         uint32_t *c, uint64_t n, void *stream);

/*
 * Fixed-matrix plans -- many products c = A x with the same f-circulant A.
 *
 * In Algorithm 1 (Section 2) the row vector's halvings (a_lo +- s a_hi down
 * to the 2x2 leaves) do not depend on the vector: they are one of the three
 * trees of the product.  A plan runs that tree once and keeps its result
 * (n residues on the device), so each product with the plan runs only the
 * vector tree, the leaf products and the recombination.  The paper has no
 * plan object; this is the reuse its structure allows.
 *
 * fcirc_aplan_create
 *   p, f, n   as for fcirc_matvec (the same errors for bad p, f, n).
 *   a         uint32[n], the row vector, values < p; device or host memory.
 *   stream    the row tree is computed on this stream; the plan is ready
 *             once the stream has passed the call (use it on the same
 *             stream, or synchronise first).
 *   plan      receives the handle.  The plan owns n * 4 bytes of device
 *             memory on the current device (FCIRC_ENOMEM if that fails).
 *             For n < 4096 the plan keeps a itself and each product runs
 *             in full.
 * fcirc_matvec_aplan
 *   c = A x for the plan's A: x, c uint32[n] as for fcirc_matvec (device
 *   or host memory, same synchronisation rules), on `stream`, with the
 *   plan's device current.  The result equals fcirc_matvec's exactly.
 *   Calls with one plan may run concurrently (the plan is read only).
 * fcirc_aplan_destroy
 *   frees the plan (cudaFree, which waits for the device); NULL is a
 *   no-op.  The caller makes sure no call using the plan is still running.
 */
typedef struct fcirc_aplan *fcirc_aplan_t;
int fcirc_aplan_create(uint32_t p, uint32_t f, const uint32_t *a, uint64_t n, void *stream,
                       fcirc_aplan_t *plan);
int fcirc_matvec_aplan(fcirc_aplan_t plan, const uint32_t *x, uint32_t *c, void *stream);
int fcirc_aplan_destroy(fcirc_aplan_t plan);

/*
 * fcirc_matvec_batched -- many independent products c_i = A_i x_i over
 * Z/pZ (Algorithm 1 per instance), each with its own size and f, in one
 * persistent launch.
 *
 *   p        odd prime < 2^30, common to all instances.
 *   f        count parameters f_i (uint32).
 *   offsets  count + 1 uint64 offsets: instance i occupies
 *            [offsets[i], offsets[i+1]) of a, x and c; its size
 *            n_i = offsets[i+1] - offsets[i] must be a power of two with
 *            1 <= n_i <= 2^16 and f_i must have an (n_i/2)-th root mod p.
 *   a, x, c  packed row vectors, vectors and results (residues).
 *
 * The plan of every instance (its root chain, Theorem 1) is computed on the
 * device, so f and offsets may change between calls without any host work.
 * The call reads offsets[count] once to size its scratch (a stream
 * synchronisation when offsets is device memory).  An instance with a bad
 * size or no root is skipped and reported by fcirc_sync_status
 * (FCIRC_EINVAL / FCIRC_ENOROOT); the others are computed.
 * Launch shape: the configuration fcirc_batched_autotune chose for the same
 * (device, p, count, total size), else a default.
 */
int fcirc_matvec_batched(uint32_t p, const uint32_t *f, const uint64_t *offsets,
                         const uint32_t *a, const uint32_t *x, uint32_t *c,
                         uint32_t count, void *stream);

/*
 * fcirc_batched_autotune -- times every launch configuration of the batched
 * product (persistent CTAs per SM, and the tile size -- hence the levels per
 * in-CTA pass -- used for instances above it) on these exact arguments (device
 * pointers), keeps the fastest for the (device, p, count, total size) of this
 * batch, and returns its index in *chosen.  With FCIRC_TUNE_CACHE set to a
 * file path the choices persist across processes.  Writes c.
 */
int fcirc_batched_autotune(uint32_t p, const uint32_t *f, const uint64_t *offsets,
                           const uint32_t *a, const uint32_t *x, uint32_t *c,
                           uint32_t count, void *stream, int *chosen);

/* Launch configuration `index` of the batched product (for reporting). */
int fcirc_batched_config(int index, int *ctas_per_sm, int *tile_log);

/*
 * fcirc_matvec_batched_graph -- captures the batched launch sequence for
 * these device pointers (and the total size offsets[count] = total_n) into a
 * CUDA graph with its own scratch; fcirc_graph_launch replays it on any
 * stream of the same device, reading f, offsets, a, x as they are at replay
 * time (the sizes must keep the same total).  fcirc_graph_destroy frees it.
 * Capture this before any other capture of the calling thread.
 */
typedef struct fcirc_graph_s *fcirc_graph_t;
int fcirc_matvec_batched_graph(uint32_t p, const uint32_t *f, const uint64_t *offsets,
                               const uint32_t *a, const uint32_t *x, uint32_t *c,
                               uint32_t count, uint64_t total_n, void *stream,
                               fcirc_graph_t *graph);
int fcirc_graph_launch(fcirc_graph_t graph, void *stream);
int fcirc_graph_destroy(fcirc_graph_t graph);

/*
 * fcirc_batched_partition -- splits a batch over `nranks` processes (one
 * GPU each) for fcirc_matvec_batched.  The instances of a batch are
 * independent products, just as the two halves of one product are after a
 * halving step (the structure argument in the proof of Theorem 1), so a
 * batch shards with no exchange between ranks: each rank runs its own
 * instances and keeps their results.
 *
 * Host-only (no GPU call), deterministic: every rank computes the same
 * partition from the same offsets, so no rank has to send it.  Longest
 * processing time first: instances sorted by the cost n_i * max(log2 n_i, 1)
 * of Algorithm 1 (largest first, ties by index), each given to the rank
 * with the least cost so far (ties to the lowest rank).
 *
 *   offsets   HOST uint64[count + 1], as for fcirc_matvec_batched
 *             (non-decreasing; sizes need not be powers of two here).
 *   nranks    1 .. 65536; rank < nranks.
 *   members   caller's uint32[count]: receives the indices of the
 *             instances of `rank`, ascending, in members[0 .. *nmembers).
 *   loads     NULL, or the caller's double[nranks]: every rank's total cost.
 *
 * Returns FCIRC_OK, or FCIRC_EINVAL (null pointer, decreasing offsets, bad
 * nranks or rank), or FCIRC_ENOMEM (host memory).
 */
int fcirc_batched_partition(const uint64_t *offsets, uint32_t count, uint32_t nranks, uint32_t rank,
                            uint32_t *members, uint32_t *nmembers, double *loads);

/*
 * poly_mul_int -- exact product of two polynomials with 16-bit unsigned
 * integer coefficients (Section 3.1): out[k] = sum_{i+j=k} P[i] Q[j] for
 * k < np + nq - 1.
 *
 * The product is one circulant product per prime of size N = next power of
 * two >= np + nq - 1 (Section 3.1: zero-padding to a power-of-two circulant),
 * computed modulo the three primes 998244353, 469762049 and 167772161 and
 * recombined by the Chinese remainder theorem (Garner's method).
 *
 *   P    np coefficients (uint16), Q  nq coefficients (uint16), little
 *        degree first;  1 <= np, nq  and  np + nq - 1 <= 2^24.
 *   out  np + nq - 1 int64 coefficients (exact: every coefficient is below
 *        min(np, nq) * 2^32 < 2^57).
 *
 * Errors: FCIRC_EINVAL for null pointers, zero or too large sizes.
 */
int poly_mul_int(const uint16_t *P, uint64_t np, const uint16_t *Q,
                 uint64_t nq, int64_t *out, void *stream);

/*
 * bigint_mul -- product of two unsigned integers given as little-endian
 * base-2^16 limbs (Section 3.2: the integers are split into parts that are
 * read as polynomial coefficients, the polynomials are multiplied through
 * the circulant product, and the carries are propagated).
 *
 *   A    na limbs (uint16, least significant first), B  nb limbs;
 *        1 <= na, nb and na + nb - 1 <= 2^24.
 *   out  na + nb limbs of A * B (the top limb may be zero).
 *
 * The column sums come from the same three-prime circulant products and CRT
 * as poly_mul_int; the carries are resolved by a parallel carry-lookahead
 * (three launches, no device-side waiting).
 * Errors: FCIRC_EINVAL for null pointers, zero or too large sizes.
 */
int bigint_mul(const uint16_t *A, uint64_t na, const uint16_t *B, uint64_t nb,
               uint16_t *out, void *stream);

/*
 * fcirc_matvec_c64 -- c = A x for a batch of complex f-circulant products in
 * FP32 (Definition 2's layout; the same recursion as fcirc_matvec, Algorithm
 * 1, over the complex numbers as the closing remark of Section 3.1 notes
 * real or complex coefficients need).  Roots and twiddles are formed in FP64
 * and rounded to FP32.
 *
 *   a, x, c  batch instances of n complex numbers, each an interleaved
 *            (re, im) float pair; instance b at offset 2 n b floats.
 *   f        the parameter, f_re + i f_im != 0 (the same for every instance).
 *   n        a power of two, 8 <= n <= 4096;  batch >= 0.
 *
 * Accuracy: relative L2 error of order 1e-7 log2(n) against exact arithmetic
 * for |f| = 1 and inputs of comparable magnitude.
 * Errors: FCIRC_EINVAL for null pointers or an unsupported n, FCIRC_ENOROOT
 * for f = 0.
 */
int fcirc_matvec_c64(const float *a, const float *x, float *c, double f_re, double f_im,
                     uint64_t n, uint64_t batch, void *stream);

/*
 * fcirc_matvec_gf -- a batch of f-circulant products over the paper's own
 * field GF(p^2) = Z/pZ[sqrt 3], p = 2^31 - 1 (Section 3.1: p + 1 = 2^31, and
 * 2 + sqrt 3 generates the elements of order dividing p + 1, so the
 * power-of-two roots of unity Algorithm 1 needs exist up to order 2^31).
 * Same recursion and batch layout as fcirc_matvec_c64, exact arithmetic
 * with Mersenne reduction.
 *
 *   a, x, c  batch instances of n elements, each an interleaved (re, im)
 *            uint32 pair meaning re + im sqrt 3, canonical in [0, p);
 *            instance b at offset 2 n b words.  Results canonical.
 *   f        f_re + f_im sqrt 3, canonical, with a 2^(log2 n - 1)-th root
 *            (Theorem 1); f = 1 gives ordinary circulants, the paper's
 *            polynomial products.
 *   n        a power of two, 8 <= n <= 4096;  batch >= 0.
 * Errors: FCIRC_EINVAL for null pointers, an unsupported n or a
 * non-canonical f; FCIRC_ENOROOT for f = 0 or f without the root.
 */
int fcirc_matvec_gf(const uint32_t *a, const uint32_t *x, uint32_t *c, uint32_t f_re, uint32_t f_im,
                    uint64_t n, uint64_t batch, void *stream);

/*
 * fcirc_matvec_ssa -- a batch of f-circulant products over the ring
 * Z/(2^K + 1), the ring of Schoenhage-Strassen multiplication (the
 * conclusion of the paper proposes Algorithm 1 there).  2 has order 2K in
 * that ring, so every root Algorithm 1 needs is a power of two and every
 * twiddle product is a shift; only the leaf products multiply elements.
 *
 *   K        64 or 128.
 *   a, x, c  batch instances of n elements; an element is K/64 + 1 uint64
 *            words: K/64 little-endian words w and a top word t in {0, 1},
 *            the value w + t 2^K in [0, 2^K] (t = 1 only with w = 0).
 *            Results come back in the same form.
 *   f        2^f_exp, 0 <= f_exp < 2K; Theorem 1's root must be a power of
 *            two, i.e. 2^(log2 n - 1) divides f_exp (f_exp = 0: ordinary
 *            circulants; f_exp = K: f = -1, negacyclic).
 *   n        a power of two, 8 <= n <= min(512, 4K);  batch >= 0.
 * Errors: FCIRC_EINVAL for null pointers, an unsupported K or n, or
 * f_exp >= 2K; FCIRC_ENOROOT when 2^(log2 n - 1) does not divide f_exp.
 */
int fcirc_matvec_ssa(const uint64_t *a, const uint64_t *x, uint64_t *c, uint32_t K, uint32_t f_exp,
                     uint64_t n, uint64_t batch, void *stream);

/*
 * fcirc_matvec_backward -- gradients of the real loss L = Re <g, A x> (the
 * convention PyTorch uses for complex tensors: the gradient of z is
 * dL/dRe z + i dL/dIm z), for the same batch layout as fcirc_matvec_c64:
 *
 *   grad_x = A^H g = the (1/conj f)-circulant with row
 *            (conj a_0, conj(f) conj a_{n-1}, ..., conj(f) conj a_1), times g;
 *   grad_a = the conj(f)-circulant with row g, times conj(x).
 *
 * Both are computed with the same halving recursion (two more f'-circulant
 * products), in one pass over a, x and g.  The paper does not treat
 * gradients; they follow from Definition 2 by differentiation.
 * Errors: as fcirc_matvec_c64.
 */
int fcirc_matvec_backward(const float *a, const float *x, const float *g, double f_re, double f_im,
                          float *grad_a, float *grad_x, uint64_t n, uint64_t batch, void *stream);

/*
 * fcirc_sync_status -- waits for `stream`, then returns and clears the
 * library's sticky device status word for the current device: FCIRC_OK;
 * FCIRC_EINVAL / FCIRC_ENOROOT if an instance of a batched call had a bad
 * size or no root; FCIRC_ETIMEOUT if a bounded device-side wait gave up;
 * FCIRC_ECUDA if the stream reported an error.
 */
int fcirc_sync_status(void *stream);

/* Name of a status code (static string). */
const char *fcirc_error_string(int status);

/* One-line detail of the calling thread's last failing call (static per
 * thread; valid until the thread's next library call). */
const char *fcirc_last_error(void);

/* Frees the scratch pool and the cached plans of every device the library
 * has touched (synchronises those devices first).  Safe to call at any
 * time outside stream capture; later calls rebuild what they need. */
int fcirc_release(void);

/*
 * fcirc_set_checks -- input checks on (1) or off (0; the default unless the
 * environment variable FCIRC_CHECKS is set to a non-zero value when the
 * library first needs it).  With checks on, every entry point that takes
 * residues launches a kernel that compares them with p (2^31 - 1 for the
 * GF(p^2) product) before the product runs; a value out of range sets the
 * sticky device status word to FCIRC_EINVAL, which fcirc_sync_status then
 * returns.  Nothing traps and the product still runs (its result for such
 * inputs is unspecified, never out of bounds).  Always FCIRC_OK.
 */
int fcirc_set_checks(int on);

/*
 * fcirc_debug_fail_alloc -- fault injection for tests: the k-th next device
 * allocation the library makes (k = 0: the next one) fails as if the device
 * were out of memory, so the entry point that asked returns FCIRC_ENOMEM
 * with the library's caches left consistent.  k < 0 switches it off.  Always
 * FCIRC_OK.
 */
int fcirc_debug_fail_alloc(int k);

/*
 * fcirc_debug_spin_limit -- the bound of the library's device-side waits:
 * the tile kernel's thread 0 probes the mbarrier its TMA loads complete on
 * at most `probes` times (mbarrier.try_wait, each probe itself time
 * limited).  A CTA whose wait gives up records FCIRC_ETIMEOUT in the sticky
 * device status word (fcirc_sync_status returns it), waits for the copies it
 * started, and leaves its tile unfinished; the call's result is then
 * unspecified but nothing faults.  probes = 0 makes every such wait give up
 * at once (for tests); probes < 0 restores the default (2^22).  Applies to
 * calls made afterwards.  Always FCIRC_OK.
 */
int fcirc_debug_spin_limit(long long probes);

#ifdef __cplusplus
}
#endif

#endif /* FCIRC_H */
