/*
 * fcirc_plan.h -- host-side root chains and twiddles of the f-circulant
 * recursion.  These functions run on the CPU only (no GPU needed) and expose
 * the numbers the kernels use, so that they can be inspected and checked.
 *
 * The recursion (Section 2, Algorithm 1 and the structure argument in the
 * proof of Theorem 1): an f-circulant of size B splits into a sqrt(f)- and a
 * (-sqrt(f))-circulant of size B/2.  Node j of level l (block size n/2^l,
 * 0 <= j < 2^l) has parameter f_{l,j}; its two children get +s_{l,j} and
 * -s_{l,j}, where s_{l,j} is the square root of f_{l,j} the library uses:
 *
 *     s_{l,j} = rho^(2^(L-l-1)) * psi_{2^(l+1)}^brv_l(j)
 *
 * with L = log2(n) - 1 halving levels (the recursion stops at 2x2 blocks),
 * rho a 2^L-th root of f, psi_m = Omega^(2^v / m) for a fixed primitive
 * 2^v-th root of unity Omega mod p (2^v || p-1), and brv_l the reversal of
 * l bits.  Theorem 1 is why rho and the roots of unity must exist.  The
 * inverses the recombination needs (c_1 = (M_1 + M_2) / (2 sqrt f), Algorithm
 * 1) come from the same closed form with rho^-1 and psi^-1, as the text of
 * Section 3.1 notes that inverse roots are products of roots already known.
 *
 * All functions return an fcirc_status code (see fcirc.h).
 */
#ifndef FCIRC_PLAN_H
#define FCIRC_PLAN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A 2^log2k-th root of f mod the odd prime p (p < 2^30): *root^(2^log2k)
 * = f.  FCIRC_ENOROOT if f = 0 or none exists, FCIRC_EINVAL for a bad p. */
int fcirc_nth_root(uint32_t p, uint32_t f, uint32_t log2k, uint32_t *root);

/* The same in the paper's field GF(p^2) = Z/pZ[sqrt 3], p = 2^31 - 1
 * (Section 3.1): a 2^log2k-th root (r_re + r_im sqrt 3) of f_re + f_im sqrt 3,
 * log2k <= 30.  FCIRC_ENOROOT if f = 0 or none exists, FCIRC_EINVAL for a
 * non-canonical f or log2k > 30. */
int fcirc_gf_nth_root(uint32_t f_re, uint32_t f_im, uint32_t log2k, uint32_t *r_re, uint32_t *r_im);

/* The twiddle s_{l,j} (and its inverse) used at node j of level l of the
 * plan for (p, f, n); requires 0 <= l < log2(n) - 1 and j < 2^l. */
int fcirc_node_twiddle(uint32_t p, uint32_t f, uint64_t n, uint32_t level,
                       uint64_t j, uint32_t *s, uint32_t *s_inv);

/* The parameter f_{L,j} of the 2x2 leaf block j (0 <= j < n/2) of the plan
 * for (p, f, n), n >= 2: block j of the result is the product of the
 * f_{L,j}-circulant 2x2 matrix with the matching entries. */
int fcirc_leaf_param(uint32_t p, uint32_t f, uint64_t n, uint64_t j,
                     uint32_t *phi);

/* The twiddle product the kernels form on the device, done on the host:
 * w = u * sigma mod p (canonical) and w_shoup = floor(w * 2^32 / p), where
 * the kernel derives w_shoup from the precomputed 64-bit quotient
 * floor(sigma * 2^64 / p) without a division.  u < p, sigma < p. */
int fcirc_twiddle_from_factor(uint32_t p, uint32_t u, uint32_t sigma,
                              uint32_t *w, uint32_t *w_shoup);

#ifdef __cplusplus
}
#endif

#endif /* FCIRC_PLAN_H */
