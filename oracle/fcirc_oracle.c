/*
 * fcirc_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU restatement of what the f-circulant
 * matrix-vector product and its applications compute (Rosowski, "On Fast
 * Computation of a Circulant Matrix-Vector Product", arXiv 2103.02605).
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file.  It shares no code, header, table or
 * constant with the CUDA library, and it does NOT implement the paper's
 * recursive halving: every routine below is the dense O(n^2) definition.
 *
 * Matrix layout (Definition 2, Section 1.2, pinned by the 3x3 example
 * printed right after it): an f-circulant n x n matrix A is identified by
 * its ROW vector a (Section 1.2, last paragraph), with 0-based entries
 *
 *      A[i][j] = a[j-i]          for j >= i
 *      A[i][j] = f * a[n+j-i]    for j <  i
 *
 * so the product c = A x is
 *
 *      c[i] = sum_{j>=i} a[j-i] x[j]  +  f * sum_{j<i} a[n+j-i] x[j].
 *
 * Arithmetic: integers mod p with 64-bit intermediates (p < 2^32), and
 * complex numbers in IEEE double precision.  Loops over independent output
 * entries are spread over OpenMP threads; each single sum is evaluated in
 * the plain index order given above.
 *
 * Functions whose parity is pinned by the tests in tests/test_oracle_pins.py:
 * every exported function below has at least one pin there.
 */
#include <stdint.h>
#include <stddef.h>
#include <complex.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

static inline uint64_t mulmod_u64(uint64_t a, uint64_t b, uint64_t p)
{
    /* a, b < p < 2^32, so a*b < 2^64 */
    return (a * b) % p;
}

static inline uint64_t mulmod_u128(uint64_t a, uint64_t b, uint64_t q)
{
    return (uint64_t)(((unsigned __int128)a * b) % q);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* One output entry c[i] of the f-circulant product mod p (Definition 2). */
static uint64_t fcirc_row_mod(uint64_t p, uint64_t f, const uint32_t *a,
                              const uint32_t *x, uint64_t n, uint64_t i)
{
    uint64_t upper = 0, lower = 0;
    for (uint64_t j = i; j < n; ++j)
        upper = (upper + mulmod_u64(a[j - i], x[j], p)) % p;
    for (uint64_t j = 0; j < i; ++j)
        lower = (lower + mulmod_u64(a[n + j - i], x[j], p)) % p;
    return (upper + mulmod_u64(f % p, lower, p)) % p;
}

/* c = A x over Z/pZ, A the f-circulant matrix with row vector a. */
void oracle_fcirc_matvec_mod(uint32_t p, uint32_t f, const uint32_t *a,
                             const uint32_t *x, uint32_t *c, uint64_t n)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < (int64_t)n; ++i)
        c[i] = (uint32_t)fcirc_row_mod(p, f, a, x, n, (uint64_t)i);
}

/* Selected entries out[m] = c[rows[m]] of the same product (for sizes where
 * the full O(n^2) product is out of reach). */
void oracle_fcirc_matvec_mod_rows(uint32_t p, uint32_t f, const uint32_t *a,
                                  const uint32_t *x, uint64_t n,
                                  const uint64_t *rows, uint64_t m,
                                  uint32_t *out)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < (int64_t)m; ++k)
        out[k] = (uint32_t)fcirc_row_mod(p, f, a, x, n, rows[k]);
}

/* Column convention: c[j] = sum_i A[i][j] x[i], which is coefficient j of
 * a(z) x(z) reduced modulo z^n - f: the terms a[m] x[t] with m + t = j
 * count once, those with m + t = j + n count f times (Section 1.2 relates
 * the row and column conventions). */
void oracle_fcirc_matvec_t_mod(uint32_t p, uint32_t f, const uint32_t *a,
                               const uint32_t *x, uint32_t *c, uint64_t n)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t jj = 0; jj < (int64_t)n; ++jj) {
        const uint64_t j = (uint64_t)jj;
        uint64_t direct = 0, wrapped = 0;
        for (uint64_t m = 0; m <= j; ++m)
            direct = (direct + mulmod_u64(a[m], x[j - m], p)) % p;
        for (uint64_t m = j + 1; m < n; ++m)
            wrapped = (wrapped + mulmod_u64(a[m], x[j + n - m], p)) % p;
        c[j] = (uint32_t)((direct + mulmod_u64(f % p, wrapped, p)) % p);
    }
}

/* The product over the paper's field GF(p^2) = Z/pZ[sqrt 3], p = 2^31 - 1
 * (Section 3.1): elements (re, im) = re + im sqrt 3 stored as uint32 pairs,
 * c[i] = sum_k a[k] x[(i+k) mod n] f^[i+k >= n] (Definition 2). */
#define GFP 2147483647ull
static void gf_mul(uint64_t ar, uint64_t ai, uint64_t br, uint64_t bi, uint64_t *cr, uint64_t *ci)
{
    *cr = (ar * br % GFP + 3 * (ai * bi % GFP)) % GFP;
    *ci = (ar * bi % GFP + ai * br % GFP) % GFP;
}

void oracle_fcirc_matvec_gf(uint32_t f_re, uint32_t f_im, const uint32_t *a, const uint32_t *x, uint32_t *c,
                            uint64_t n)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t ii = 0; ii < (int64_t)n; ++ii) {
        const uint64_t i = (uint64_t)ii;
        uint64_t ur = 0, ui = 0, lr = 0, li = 0, pr, pi;
        for (uint64_t k = 0; k < n; ++k) {
            const uint64_t j = i + k;
            if (j < n) {
                gf_mul(a[2 * k], a[2 * k + 1], x[2 * j], x[2 * j + 1], &pr, &pi);
                ur = (ur + pr) % GFP;
                ui = (ui + pi) % GFP;
            } else {
                gf_mul(a[2 * k], a[2 * k + 1], x[2 * (j - n)], x[2 * (j - n) + 1], &pr, &pi);
                lr = (lr + pr) % GFP;
                li = (li + pi) % GFP;
            }
        }
        gf_mul(f_re, f_im, lr, li, &pr, &pi);
        c[2 * i] = (uint32_t)((ur + pr) % GFP);
        c[2 * i + 1] = (uint32_t)((ui + pi) % GFP);
    }
}

/* Toeplitz product c = T x, T[i][j] = t[j - i + n - 1] (t: the 2n - 1
 * diagonals, lowest first), straight from the definition. */
void oracle_toeplitz_matvec_mod(uint32_t p, const uint32_t *t, const uint32_t *x, uint32_t *c, uint64_t n)
{
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t ii = 0; ii < (int64_t)n; ++ii) {
        const uint64_t i = (uint64_t)ii;
        uint64_t acc = 0;
        for (uint64_t j = 0; j < n; ++j)
            acc = (acc + mulmod_u64(t[j + n - 1 - i], x[j], p)) % p;
        c[i] = (uint32_t)acc;
    }
}

/* A batch of independent products with per-instance f and length
 * n_i = offsets[i+1] - offsets[i]; a, x, c are packed back to back. */
void oracle_fcirc_matvec_mod_batched(uint32_t p, const uint32_t *f,
                                     const uint64_t *offsets,
                                     const uint32_t *a, const uint32_t *x,
                                     uint32_t *c, uint32_t count)
{
    for (uint32_t b = 0; b < count; ++b) {
        uint64_t off = offsets[b], n = offsets[b + 1] - offsets[b];
        oracle_fcirc_matvec_mod(p, f[b], a + off, x + off, c + off, n);
    }
}

/* ---------------------------------------------------------------------- */
/* Complex double precision (the real/complex remark closing Section 3.1). */
/* a, x, c hold `batch` instances of n complex numbers as (re, im) pairs.  */

static cplx ld(const double *v, uint64_t k) { return v[2 * k] + I * v[2 * k + 1]; }
static void st(double *v, uint64_t k, cplx z) { v[2 * k] = creal(z); v[2 * k + 1] = cimag(z); }

/* Entry A[i][j] of the f-circulant with row vector a (Definition 2). */
static cplx fcirc_entry_c(cplx f, const double *a, uint64_t n, uint64_t i, uint64_t j)
{
    return j >= i ? ld(a, j - i) : f * ld(a, n + j - i);
}

void oracle_fcirc_matvec_c128(double f_re, double f_im, const double *a,
                              const double *x, double *c, uint64_t n,
                              uint64_t batch)
{
    const cplx f = f_re + I * f_im;
    #pragma omp parallel for schedule(static) collapse(2)
    for (int64_t b = 0; b < (int64_t)batch; ++b)
        for (int64_t i = 0; i < (int64_t)n; ++i) {
            const double *ab = a + 2 * n * b, *xb = x + 2 * n * b;
            cplx s = 0;
            for (uint64_t j = 0; j < n; ++j)
                s += fcirc_entry_c(f, ab, n, (uint64_t)i, j) * ld(xb, j);
            st(c + 2 * n * b, (uint64_t)i, s);
        }
}

/*
 * Gradients of the real loss L = Re <g, c> = Re sum_i conj(g_i) c_i with
 * c = A x, in the convention PyTorch uses for complex tensors (the returned
 * gradient of z is dL/dRe z + i dL/dIm z):
 *
 *   grad_x = A^H g,            (A^H)[j][i] = conj(A[i][j])
 *   grad_a = X^H g,            X[i][k]     = d c_i / d a_k
 *                                          = x[(i+k) mod n] * f^[i+k >= n]
 *
 * both written out entry by entry from the definition of A above.
 */
void oracle_fcirc_grad_c128(double f_re, double f_im, const double *a,
                            const double *x, const double *g,
                            double *grad_a, double *grad_x, uint64_t n,
                            uint64_t batch)
{
    const cplx f = f_re + I * f_im;
    #pragma omp parallel for schedule(static) collapse(2)
    for (int64_t b = 0; b < (int64_t)batch; ++b)
        for (int64_t k = 0; k < (int64_t)n; ++k) {
            const double *ab = a + 2 * n * b, *xb = x + 2 * n * b, *gb = g + 2 * n * b;
            cplx sx = 0, sa = 0;
            for (uint64_t i = 0; i < n; ++i) {
                /* grad_x[k] += conj(A[i][k]) g[i] */
                sx += conj(fcirc_entry_c(f, ab, n, i, (uint64_t)k)) * ld(gb, i);
                /* grad_a[k] += conj(X[i][k]) g[i] */
                uint64_t idx = i + (uint64_t)k;
                cplx xik = idx >= n ? f * ld(xb, idx - n) : ld(xb, idx);
                sa += conj(xik) * ld(gb, i);
            }
            st(grad_x + 2 * n * b, (uint64_t)k, sx);
            st(grad_a + 2 * n * b, (uint64_t)k, sa);
        }
}

/* ---------------------------------------------------------------------- */
/* Polynomial product (Section 3.1): schoolbook linear convolution.        */
/* out[k] = sum_{i+j=k} P[i] Q[j],  k < np + nq - 1.  Exact in 64 bits for  */
/* min(np, nq) < 2^32 because each term is below 2^32.                     */

static int64_t poly_coeff(const uint16_t *P, uint64_t np, const uint16_t *Q,
                          uint64_t nq, uint64_t k)
{
    uint64_t lo = k + 1 > nq ? k + 1 - nq : 0;
    uint64_t hi = k < np - 1 ? k : np - 1;
    uint64_t s = 0;
    for (uint64_t i = lo; i <= hi; ++i)
        s += (uint64_t)P[i] * (uint64_t)Q[k - i];
    return (int64_t)s;
}

void oracle_poly_mul(const uint16_t *P, uint64_t np, const uint16_t *Q,
                     uint64_t nq, int64_t *out)
{
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < (int64_t)(np + nq - 1); ++k)
        out[k] = poly_coeff(P, np, Q, nq, (uint64_t)k);
}

void oracle_poly_mul_coeffs(const uint16_t *P, uint64_t np, const uint16_t *Q,
                            uint64_t nq, const uint64_t *idx, uint64_t m,
                            int64_t *out)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < (int64_t)m; ++k)
        out[k] = poly_coeff(P, np, Q, nq, idx[k]);
}

/* ---------------------------------------------------------------------- */
/* Large-integer product (Section 3.2): little-endian base-2^16 limbs.     */
/* Column sums by schoolbook, then one sequential carry pass.              */

void oracle_bigint_mul(const uint16_t *A, uint64_t na, const uint16_t *B,
                       uint64_t nb, uint16_t *out)
{
    const uint64_t nout = na + nb;
    uint64_t carry = 0;
    for (uint64_t k = 0; k < nout; ++k) {
        uint64_t col = 0;
        if (k < na + nb - 1) {
            uint64_t lo = k + 1 > nb ? k + 1 - nb : 0;
            uint64_t hi = k < na - 1 ? k : na - 1;
            for (uint64_t i = lo; i <= hi; ++i)
                col += (uint64_t)A[i] * (uint64_t)B[k - i];
        }
        /* col < 2^32 * min(na, nb) and carry < col / 2^15, no overflow for
         * min(na, nb) < 2^31 */
        uint64_t t = col + carry;
        out[k] = (uint16_t)(t & 0xFFFFu);
        carry = t >> 16;
    }
}

/* Column sums alone (the step before the carry), used for sampled checks. */
void oracle_bigint_columns(const uint16_t *A, uint64_t na, const uint16_t *B,
                           uint64_t nb, const uint64_t *idx, uint64_t m,
                           uint64_t *out)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < (int64_t)m; ++k)
        out[k] = (uint64_t)poly_coeff(A, na, B, nb, idx[k]);
}

/* ---------------------------------------------------------------------- */
/* Evaluation at a point modulo an independent modulus q < 2^63 (Horner).  */
/* Used to check full-size products: P(t) Q(t) = C(t) (mod q).             */

uint64_t oracle_eval_u16_mod(const uint16_t *coef, uint64_t len, uint64_t t,
                             uint64_t q)
{
    uint64_t acc = 0;
    for (uint64_t k = len; k-- > 0;)
        acc = (mulmod_u128(acc, t, q) + coef[k]) % q;
    return acc;
}

uint64_t oracle_eval_i64_mod(const int64_t *coef, uint64_t len, uint64_t t,
                             uint64_t q)
{
    uint64_t acc = 0;
    for (uint64_t k = len; k-- > 0;) {
        int64_t v = coef[k] % (int64_t)q;
        uint64_t u = v < 0 ? (uint64_t)(v + (int64_t)q) : (uint64_t)v;
        acc = (mulmod_u128(acc, t, q) + u) % q;
    }
    return acc;
}
