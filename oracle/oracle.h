/* Oracle for the sparse multivariate polynomial product.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library calls this code: only the
 * tests, the package's smoke check and the benchmark's CPU-baseline leg load
 * it.  It shares no code, header or table with the CUDA path.
 *
 * Everything here is plain C with 128-bit integers and works on exponent
 * VECTORS (never on packed keys), so the CUDA path's packing is checked
 * independently.
 *
 * Definition followed (Sec. 2): the product of A = sum_i a_i x^alpha_i and
 * B = sum_j b_j x^beta_j is the sum of all pairwise term products
 * a_i b_j x^(alpha_i + beta_j); equal monomials are combined and the result
 * is listed in ascending monomial order (its canonical form, Sec. 2 and
 * Alg. 1, line "concatenate ... using ascending order").
 *
 * Readings of points the paper leaves open (all shared with the library):
 *  - order: lexicographic with x_1 most significant;
 *  - coefficients: kind 0 = integers mod p = 2^61 - 1 (inputs any uint64,
 *    reduced mod p); kind 1 = int64 inputs, exact int128 result;
 *  - terms whose coefficient is zero are dropped, inputs may repeat a
 *    monomial (repeats are summed) and may come in any order;
 *  - exponent packing widths w_v include one guard bit: every input exponent
 *    must be < 2^(w_v - 1) and so must every exponent of the product,
 *    otherwise the call fails with OR_EEXP_OVERFLOW and returns no terms;
 *  - kind 1: a repeated input monomial whose summed coefficient leaves int64,
 *    or operands with max|a| * max|b| * min(n_a, n_b) >= 2^127, fail with
 *    OR_ECOEF_BOUND before any product is formed.
 */
#ifndef POLYMUL_ORACLE_H
#define POLYMUL_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_OK             0
#define OR_EINVAL        -1
#define OR_EEXP_OVERFLOW -2
#define OR_ECOEF_BOUND   -3
#define OR_ENOMEM        -5

#define OR_KIND_M61   0   /* coefficients uint64, result mod 2^61-1 */
#define OR_KIND_I64   1   /* coefficients int64, result int128 (lo, hi words) */
#define OR_KIND_I128  2   /* (evaluation only) int128 coefficients as (lo, hi) */

/* Full product by the definition: every (i, j) pair accumulated in a hash map
 * keyed on the exponent vector, then sorted.  Outputs are malloc'd and must
 * be released with oracle_free.  h_coefs: uint64 per term (kind 0) or two
 * uint64 words (lo, hi) per term (kind 1). */
int oracle_mul(uint32_t nvars, const uint8_t *field_bits, int kind,
               const uint32_t *f_exps, const void *f_coefs, uint64_t nf,
               const uint32_t *g_exps, const void *g_coefs, uint64_t ng,
               uint32_t **h_exps, void **h_coefs, uint64_t *nh);

/* Alg. 1 of the paper on CPU threads: packed 64-bit exponents (Sec. 7),
 * step 1 = the almost regular grid of Sec. 5 with parameter l, sorted and
 * deduplicated; step 2 = FindEdge staircase + a comparison sort per interval
 * with dynamic scheduling over `threads` threads; concatenation.  Same
 * outputs and error codes as oracle_mul. */
int oracle_mul_alg1(uint32_t nvars, const uint8_t *field_bits, int kind,
                    const uint32_t *f_exps, const void *f_coefs, uint64_t nf,
                    const uint32_t *g_exps, const void *g_coefs, uint64_t ng,
                    uint32_t l, uint32_t threads,
                    uint32_t **h_exps, void **h_coefs, uint64_t *nh,
                    uint64_t *n_intervals);

/* The grid S* of Sec. 5 for sorted packed keys (step 1 of Alg. 1 before the
 * sort): writes at most *n_out keys into out, returns the count needed. */
uint64_t oracle_grid(const uint64_t *alpha, uint64_t na, const uint64_t *beta,
                     uint64_t nb, uint32_t l, uint64_t *out, uint64_t cap);

/* Coefficient of each monomial gammas[k] (k < count) in f*g, computed one
 * monomial at a time as sum_i a_i * b(gamma - alpha_i).  For sampled checks
 * of products too large for oracle_mul.  out: uint64 (kind 0) or (lo, hi)
 * pairs (kind 1).  Returns OR_OK or an error code of oracle_mul's rules. */
int oracle_coef_at(uint32_t nvars, const uint8_t *field_bits, int kind,
                   const uint32_t *f_exps, const void *f_coefs, uint64_t nf,
                   const uint32_t *g_exps, const void *g_coefs, uint64_t ng,
                   const uint32_t *gammas, uint64_t count, void *out);

/* p(r) mod 2^61-1 for a polynomial with coefficients of the given kind
 * (0: uint64, 1: int64, 2: int128 as (lo, hi)) at the point r[0..nvars). */
uint64_t oracle_eval(uint32_t nvars, int kind, const uint32_t *exps,
                     const void *coefs, uint64_t n, const uint64_t *r);

void oracle_free(void *p);

#ifdef __cplusplus
}
#endif
#endif
