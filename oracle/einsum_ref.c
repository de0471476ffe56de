/*
 * Plain FP64 evaluation of one einsum -- TEST INFRASTRUCTURE ONLY.
 *
 * Computes Eq. (1) of the paper (Sec. "Preliminaries", Def. of an Einstein
 * summation):
 *
 *     R[I_out] = sum over (union_j I_in,j minus I_out) of prod_k A_k[I_in,k]
 *
 * with nested loops: output indices outermost in row-major order, the
 * contracted indices innermost in increasing index-id order (last one
 * fastest), the product taken left to right in operand order.  Alongside R
 * it returns the absolute contraction S[I_out] = sum prod_k |A_k[I_in,k]|,
 * the scale that the componentwise tolerances are stated against.
 *
 * An index repeated inside one operand is a diagonal (its strides add up).
 * A zero-length contracted index gives an empty sum (R = S = 0).
 * Operands are dense row-major FP64 arrays (the caller upcasts narrower
 * types exactly).  Optional ``sel`` evaluates only the listed output
 * positions (flat row-major indices).
 *
 * Also: elementwise sin / cos / exp from the host libm, used when the
 * oracle materialises lambda operands (Def. "Functional Batched Einstein
 * Summation").
 *
 * Parity: pinned in tests/test_oracle_eval.py by numpy.einsum on
 * integer-valued inputs (exact), by pure-Python brute force on tiny inputs,
 * by the paper's matmul and triple-product examples, and by trace / empty
 * axis special cases.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MAXI 26
#define MAXOPS 16

int oracle_einsum_f64(int n_idx, const int64_t *len,
                      int n_out, const int *out_ids,
                      int n_ops, const int *ndim, const int *ids,
                      const double *const *data,
                      int64_t n_sel, const int64_t *sel,
                      double *R, double *S)
{
    if (n_idx < 0 || n_idx > MAXI || n_ops < 1 || n_ops > MAXOPS || n_out < 0 || n_out > MAXI)
        return -1;
    /* coef[k][c]: how far operand k's flat offset moves per step of index c */
    int64_t coef[MAXOPS][MAXI];
    memset(coef, 0, sizeof coef);
    int pos = 0;
    for (int k = 0; k < n_ops; ++k) {
        int64_t st = 1;
        for (int d = ndim[k] - 1; d >= 0; --d) {
            int c = ids[pos + d];
            if (c < 0 || c >= n_idx) return -2;
            coef[k][c] += st;
            st *= len[c];
        }
        pos += ndim[k];
    }
    int is_out[MAXI] = {0};
    for (int d = 0; d < n_out; ++d) is_out[out_ids[d]] = 1;
    int con[MAXI], n_con = 0;
    for (int c = 0; c < n_idx; ++c)
        if (!is_out[c]) con[n_con++] = c;

    int64_t total_out = 1;
    for (int d = 0; d < n_out; ++d) total_out *= len[out_ids[d]];
    int64_t total_con = 1;
    for (int t = 0; t < n_con; ++t) total_con *= len[con[t]];
    int64_t n_eval = sel ? n_sel : total_out;

#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < n_eval; ++q) {
        int64_t o = sel ? sel[q] : q;
        int64_t base[MAXOPS];
        for (int k = 0; k < n_ops; ++k) base[k] = 0;
        int64_t rem = o;
        for (int d = n_out - 1; d >= 0; --d) {
            int c = out_ids[d];
            int64_t v = rem % len[c];
            rem /= len[c];
            for (int k = 0; k < n_ops; ++k) base[k] += v * coef[k][c];
        }
        double acc = 0.0, aacc = 0.0;
        if (total_con > 0) {
            int64_t ctr[MAXI];
            int64_t off[MAXOPS];
            for (int t = 0; t < n_con; ++t) ctr[t] = 0;
            for (int k = 0; k < n_ops; ++k) off[k] = base[k];
            for (int64_t it = 0; it < total_con; ++it) {
                double p = data[0][off[0]];
                for (int k = 1; k < n_ops; ++k) p *= data[k][off[k]];
                acc += p;
                aacc += fabs(p);
                /* odometer step, last contracted index fastest */
                for (int t = n_con - 1; t >= 0; --t) {
                    int c = con[t];
                    ctr[t] += 1;
                    for (int k = 0; k < n_ops; ++k) off[k] += coef[k][c];
                    if (ctr[t] < len[c]) break;
                    for (int k = 0; k < n_ops; ++k) off[k] -= coef[k][c] * len[c];
                    ctr[t] = 0;
                }
            }
        }
        R[q] = acc;
        if (S) S[q] = aacc;
    }
    return 0;
}

void oracle_sin(int64_t n, const double *x, double *y)
{
#pragma omp parallel for
    for (int64_t i = 0; i < n; ++i) y[i] = sin(x[i]);
}

void oracle_cos(int64_t n, const double *x, double *y)
{
#pragma omp parallel for
    for (int64_t i = 0; i < n; ++i) y[i] = cos(x[i]);
}

void oracle_exp(int64_t n, const double *x, double *y)
{
#pragma omp parallel for
    for (int64_t i = 0; i < n; ++i) y[i] = exp(x[i]);
}

#ifdef _OPENMP
#include <omp.h>
#endif

/* Thread count used by the parallel loops above (for the CPU baseline). */
int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
