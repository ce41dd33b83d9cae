/*
 * oracle.h -- plain FP64 CPU oracle for the all-pairs method.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or call this code: only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header, table or
 * helper with the CUDA library; both sides only see the same seeded inputs.
 *
 * Every routine is the textbook definition written out with double loops in
 * double precision (libm exp/sqrt/sin/cos), one pair at a time.  Pairs may be
 * spread over POSIX threads purely so that large samples finish; each pair is
 * still evaluated by one thread in the order written.
 *
 * Conventions (0-based, the paper is 1-based):
 *   - the problem is f(l(i), l(j)) for every i < j (Sec. III, Design);
 *   - the packed output index of the upper-triangle pair (i, j), 0 <= i < j < n,
 *     is p(i,j) = i*n - i*(i+1)/2 + (j - i - 1), the row-major enumeration of
 *     the strict upper triangle; there are n(n-1)/2 pairs (Sec. VI-A).
 */
#ifndef ALLPAIRS_ORACLE_H
#define ALLPAIRS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* number of unordered pairs, n(n-1)/2 (Sec. VI-A, Eq. 1 "n choose 2") */
int64_t or_pair_count(int64_t n);
/* packed row-major index of pair (i, j), 0 <= i < j < n; -1 if out of range */
int64_t or_pair_index(int64_t i, int64_t j, int64_t n);

/*
 * Divide-and-conquer order of Sec. IV-B: the n x n matrix is split into four
 * quadrants (top-left, top-right, bottom-left, bottom-right), each split again
 * recursively down to single entries; quadrants holding no entry with i < j
 * are skipped.  Writes the visited (i, j) leaves in order; returns their
 * number (always n(n-1)/2).  out_i/out_j must hold n(n-1)/2 entries.
 */
int64_t or_dc_order(int64_t n, int64_t *out_i, int64_t *out_j);

/*
 * Gaussian overlap cost between weighted point clouds (the cross term of the
 * GMM L2 distance named in Sec. V-C):
 *   f(i,j; theta,t) = sum_a sum_b w_a w_b exp(-|x_a - (R(theta) x_b + t)|^2
 *                                            / (2 (sigma_a^2 + sigma_b^2)))
 * with a over the points of item i and b over the points of item j.
 * dim is 2 or 3.  Points of item k are [off[k], off[k+1]) in the SoA arrays
 * x, y, z (z ignored when dim == 2), sigma, w (w == NULL means all weights 1).
 * params == NULL means the identity transform; otherwise params[3q..3q+2] =
 * (theta, tx, ty) for pair q (dim must be 2).  R(theta) = [[c,-s],[s,c]] acts
 * on the second item's points.
 * Optional outputs per pair (NULL to skip):
 *   kappa[q] = sum |arg| e / sum e  (arg = exponent, e = its exp), the FP32
 *              conditioning of the sum;
 *   bound[q] = sum (|arg| + 4) 2^-23 e, an absolute error scale for an FP32
 *              evaluation of the same sum.
 */
void or_overlap_pairs(int dim, const int64_t *off, const float *x,
                      const float *y, const float *z, const float *sigma,
                      const float *w, int64_t n_pairs, const int64_t *pi,
                      const int64_t *pj, const double *params, double *f,
                      double *kappa, double *bound, int n_threads);

/*
 * The two particle scores of the microscopy application (Sec. V-C names a
 * quadratic L2 distance between Gaussian mixtures and a Bhattacharyya
 * distance without writing either down; these are the standard forms).
 * Component a of item i: weight w_a, density N(x; x_a, sigma_a^2 I) in dim
 * dimensions; s2 = sigma_a^2 + sigma_b^2, u_b = R(theta) x_b + t as above.
 *
 * which == 1, the squared L2 distance between the mixtures:
 *   d(i,j) = S_i + S_j - 2 C_ij,
 *   C_ij = integral of p_i p_j = sum_a sum_b w_a w_b (2 pi s2)^(-dim/2)
 *                                          exp(-|x_a - u_b|^2 / (2 s2)),
 *   S_i = C_ii at the identity (every a, a' of item i, a = a' included).
 * which == 2, the Bhattacharyya cost: component pairs weighted by
 *   sqrt(w_a w_b) times the Bhattacharyya coefficient of the two Gaussians,
 *   f(i,j) = sum_a sum_b sqrt(w_a w_b) (2 sigma_a sigma_b / s2)^(dim/2)
 *                                     exp(-|x_a - u_b|^2 / (4 s2)).
 * Pairs may have i == j.  bound[q] (optional): an absolute error scale for an
 * FP32 evaluation, the sum over the terms involved (for which == 1 those of
 * S_i, S_j and twice those of C_ij) of (|arg| + 6) 2^-23 |term|, arg the
 * exponent's magnitude.
 */
void or_gmm_pairs(int which, int dim, const int64_t *off, const float *x,
                  const float *y, const float *z, const float *sigma,
                  const float *w, int64_t n_pairs, const int64_t *pi,
                  const int64_t *pj, const double *params, double *out,
                  double *bound, int n_threads);

/* S_i of every item (the which == 1 self term) and its error scale */
void or_gmm_self(int dim, const int64_t *off, const float *x, const float *y,
                 const float *z, const float *sigma, const float *w,
                 int64_t n_items, double *S, double *bound, int n_threads);

/*
 * Cosine of sparse composition vectors (the bioinformatics comparison of
 * Sec. V-B: "essentially the dot product between two sparse vectors"):
 *   c(i,j) = sum_k a_ik a_jk / sqrt(sum_k a_ik^2 sum_k a_jk^2),
 * rows in CSR form: entries [off[i], off[i+1]) with strictly increasing
 * indices idx[] and values val[].  The dot product is a merge of the two
 * sorted index lists; NaN when a row has no entries or only zeros.
 */
void or_sparse_cosine_pairs(const int64_t *off, const int32_t *idx, const float *val,
                            int64_t n_pairs, const int64_t *pi, const int64_t *pj,
                            double *c, int n_threads);

/*
 * The same cost (dim == 2) and its analytic gradient with respect to
 * (theta, tx, ty).  With y_b = R x_b + t, d = x_a - y_b, s2 = sa^2 + sb^2,
 * e = exp(-|d|^2 / (2 s2)):
 *   df/dt     = sum w_a w_b e d / s2
 *   df/dtheta = sum w_a w_b e (d . J R x_b) / s2,   J = [[0,-1],[1,0]].
 * g[3q..3q+2] = (df/dtheta, df/dtx, df/dty).
 */
void or_overlap_grad_pairs(const int64_t *off, const float *x, const float *y,
                           const float *sigma, const float *w, int64_t n_pairs,
                           const int64_t *pi, const int64_t *pj,
                           const double *params, double *f, double *g,
                           int n_threads);

/*
 * Per-item statistics of dense vectors (rows of a row-major [n_rows][D] FP32
 * array, row stride ld >= D elements), two passes in FP64:
 *   mu_i = (1/D) sum_k x_ik,   ss_i = sum_k (x_ik - mu_i)^2.
 */
void or_vector_stats(int64_t n_rows, int64_t D, int64_t ld, const float *X,
                     double *mu, double *ss, int n_threads);

/*
 * Pearson correlation (the normalised cross correlation of Sec. V-A):
 *   r_ij = sum_k (x_ik - mu_i)(x_jk - mu_j) / sqrt(ss_i ss_j)
 * for the listed row pairs, centred sums in FP64.  kahan != 0 accumulates the
 * centred products with Kahan compensation (used only to bound the plain sum's
 * own rounding).
 */
void or_pearson_pairs(int64_t D, int64_t ld, const float *X, const double *mu,
                      const double *ss, int64_t n_pairs, const int64_t *pi,
                      const int64_t *pj, int kahan, double *r, int n_threads);

/*
 * One batched gradient-ascent step on log f for each listed pair:
 *   p <- p + eta * grad f / f      (skipped, flag = 1, when f < fmin)
 * params is updated in place; f and g receive the values at the old params.
 */
void or_ascent_step(const int64_t *off, const float *x, const float *y,
                    const float *sigma, const float *w, int64_t n_pairs,
                    const int64_t *pi, const int64_t *pj, double *params,
                    double eta, double fmin, double *f, double *g,
                    int32_t *flag, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
