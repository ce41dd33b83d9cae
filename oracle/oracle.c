/*
 * oracle.c -- plain FP64 CPU oracle for the all-pairs method.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code
 * with the CUDA library.  See oracle.h for the definitions and citations.
 *
 * Pins that hold it to the mathematics rather than to itself live in the
 * CPU test suite (brute force in a second formulation, closed forms,
 * quadrature, invariances, finite differences, the paper's printed counts).
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* pair indexing (Sec. III problem statement, Sec. VI-A pair count)    */
/* ------------------------------------------------------------------ */

int64_t or_pair_count(int64_t n) { return n < 2 ? 0 : n * (n - 1) / 2; }

int64_t or_pair_index(int64_t i, int64_t j, int64_t n) {
  if (i < 0 || j <= i || j >= n) return -1;
  /* rows 0..i-1 hold (n-1) + (n-2) + ... + (n-i) pairs */
  int64_t before = 0;
  for (int64_t r = 0; r < i; ++r) before += n - 1 - r;
  return before + (j - i - 1);
}

/* ------------------------------------------------------------------ */
/* divide-and-conquer quadrant order (Sec. IV-B)                        */
/* ------------------------------------------------------------------ */

static void dc_rec(int64_t r0, int64_t r1, int64_t c0, int64_t c1,
                   int64_t *oi, int64_t *oj, int64_t *k) {
  if (r0 >= r1 || c0 >= c1) return;        /* empty quadrant */
  if (r0 >= c1 - 1) return;                 /* no entry with i < j */
  if (r1 - r0 == 1 && c1 - c0 == 1) {       /* a single entry: a leaf job */
    if (r0 < c0) { oi[*k] = r0; oj[*k] = c0; ++*k; }
    return;
  }
  int64_t rm = r0 + (r1 - r0 + 1) / 2;      /* split rows and columns */
  int64_t cm = c0 + (c1 - c0 + 1) / 2;
  dc_rec(r0, rm, c0, cm, oi, oj, k);        /* top-left */
  dc_rec(r0, rm, cm, c1, oi, oj, k);        /* top-right */
  dc_rec(rm, r1, c0, cm, oi, oj, k);        /* bottom-left */
  dc_rec(rm, r1, cm, c1, oi, oj, k);        /* bottom-right */
}

int64_t or_dc_order(int64_t n, int64_t *out_i, int64_t *out_j) {
  int64_t k = 0;
  dc_rec(0, n, 0, n, out_i, out_j, &k);
  return k;
}

/* ------------------------------------------------------------------ */
/* a tiny thread pool over pair ranges                                  */
/* ------------------------------------------------------------------ */

typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi);
typedef struct { range_fn fn; void *ctx; int64_t lo, hi; } range_job;

static void *range_thread(void *p) {
  range_job *j = (range_job *)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

static void parallel_ranges(range_fn fn, void *ctx, int64_t n, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  if (n_threads == 1 || n < 2) { fn(ctx, 0, n); return; }
  pthread_t th[256];
  range_job jobs[256];
  int64_t chunk = (n + n_threads - 1) / n_threads;
  int started = 0;
  for (int t = 0; t < n_threads; ++t) {
    int64_t lo = (int64_t)t * chunk, hi = lo + chunk;
    if (lo >= n) break;
    if (hi > n) hi = n;
    jobs[t].fn = fn; jobs[t].ctx = ctx; jobs[t].lo = lo; jobs[t].hi = hi;
    if (pthread_create(&th[t], NULL, range_thread, &jobs[t]) != 0) {
      fn(ctx, lo, hi);               /* could not start: run it here */
      jobs[t].fn = NULL;
    }
    started = t + 1;
  }
  for (int t = 0; t < started; ++t)
    if (jobs[t].fn) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------ */
/* Gaussian overlap cost (GMM L2 cross term, Sec. V-C)                  */
/* ------------------------------------------------------------------ */

typedef struct {
  int dim;
  const int64_t *off;
  const float *x, *y, *z, *sigma, *w;
  const int64_t *pi, *pj;
  const double *params;
  double *f, *kappa, *bound, *g;
} overlap_ctx;

static void overlap_range(void *vc, int64_t lo, int64_t hi) {
  overlap_ctx *c = (overlap_ctx *)vc;
  for (int64_t q = lo; q < hi; ++q) {
    int64_t i = c->pi[q], j = c->pj[q];
    double th = 0.0, tx = 0.0, ty = 0.0;
    if (c->params) { th = c->params[3 * q]; tx = c->params[3 * q + 1]; ty = c->params[3 * q + 2]; }
    double cs = cos(th), sn = sin(th);
    double sum = 0.0, sum_arg = 0.0, sum_bnd = 0.0;
    for (int64_t a = c->off[i]; a < c->off[i + 1]; ++a) {
      double wa = c->w ? (double)c->w[a] : 1.0;
      double sa = (double)c->sigma[a];
      for (int64_t b = c->off[j]; b < c->off[j + 1]; ++b) {
        double wb = c->w ? (double)c->w[b] : 1.0;
        double sb = (double)c->sigma[b];
        double xb = (double)c->x[b], yb = (double)c->y[b];
        /* transformed second point R x_b + t (identity when params == NULL) */
        double ux = cs * xb - sn * yb + tx;
        double uy = sn * xb + cs * yb + ty;
        double dx = (double)c->x[a] - ux;
        double dy = (double)c->y[a] - uy;
        double d2 = dx * dx + dy * dy;
        if (c->dim == 3) {
          double dz = (double)c->z[a] - (double)c->z[b];
          d2 += dz * dz;
        }
        double s2 = sa * sa + sb * sb;
        double arg = d2 / (2.0 * s2);
        double e = wa * wb * exp(-arg);
        sum += e;
        sum_arg += arg * e;
        sum_bnd += (arg + 4.0) * ldexp(1.0, -23) * e;
      }
    }
    c->f[q] = sum;
    if (c->kappa) c->kappa[q] = sum > 0.0 ? sum_arg / sum : 0.0;
    if (c->bound) c->bound[q] = sum_bnd;
  }
}

void or_overlap_pairs(int dim, const int64_t *off, const float *x,
                      const float *y, const float *z, const float *sigma,
                      const float *w, int64_t n_pairs, const int64_t *pi,
                      const int64_t *pj, const double *params, double *f,
                      double *kappa, double *bound, int n_threads) {
  overlap_ctx c;
  memset(&c, 0, sizeof c);
  c.dim = dim; c.off = off; c.x = x; c.y = y; c.z = z; c.sigma = sigma; c.w = w;
  c.pi = pi; c.pj = pj; c.params = params; c.f = f; c.kappa = kappa; c.bound = bound;
  parallel_ranges(overlap_range, &c, n_pairs, n_threads);
}

/* ------------------------------------------------------------------ */
/* Particle scores as Gaussian mixtures: GMM L2 distance, Bhattacharyya  */
/* ------------------------------------------------------------------ */

/* sum over a in item i, b in item j of one score's terms; the transform
 * (cs, sn, tx, ty) moves item j's points */
static void gmm_sum(int which, const overlap_ctx *c, int64_t i, int64_t j, double cs,
                    double sn, double tx, double ty, double *sum, double *bnd) {
  const double pi_ = 3.14159265358979323846;
  double acc = 0.0, eb = 0.0;
  for (int64_t a = c->off[i]; a < c->off[i + 1]; ++a) {
    double wa = c->w ? (double)c->w[a] : 1.0;
    double sa = (double)c->sigma[a];
    for (int64_t b = c->off[j]; b < c->off[j + 1]; ++b) {
      double wb = c->w ? (double)c->w[b] : 1.0;
      double sb = (double)c->sigma[b];
      double xb = (double)c->x[b], yb = (double)c->y[b];
      double dx = (double)c->x[a] - (cs * xb - sn * yb + tx);
      double dy = (double)c->y[a] - (sn * xb + cs * yb + ty);
      double d2 = dx * dx + dy * dy;
      if (c->dim == 3) {
        double dz = (double)c->z[a] - (double)c->z[b];
        d2 += dz * dz;
      }
      double s2 = sa * sa + sb * sb, arg, term;
      if (which == 1) {
        arg = d2 / (2.0 * s2);
        term = wa * wb * pow(2.0 * pi_ * s2, -0.5 * c->dim) * exp(-arg);
      } else {
        arg = d2 / (4.0 * s2);
        term = sqrt(wa * wb) * pow(2.0 * sa * sb / s2, 0.5 * c->dim) * exp(-arg);
      }
      acc += term;
      eb += (arg + 6.0) * ldexp(1.0, -23) * fabs(term);
    }
  }
  *sum = acc;
  *bnd = eb;
}

typedef struct {
  overlap_ctx c;
  int which;
} gmm_ctx;

static void gmm_range(void *vc, int64_t lo, int64_t hi) {
  gmm_ctx *g = (gmm_ctx *)vc;
  const overlap_ctx *c = &g->c;
  for (int64_t q = lo; q < hi; ++q) {
    int64_t i = c->pi[q], j = c->pj[q];
    double th = 0.0, tx = 0.0, ty = 0.0;
    if (c->params) { th = c->params[3 * q]; tx = c->params[3 * q + 1]; ty = c->params[3 * q + 2]; }
    double cs = cos(th), sn = sin(th), v, e;
    gmm_sum(g->which, c, i, j, cs, sn, tx, ty, &v, &e);
    if (g->which == 1) {
      double si, ei, sj, ej;
      gmm_sum(1, c, i, i, 1.0, 0.0, 0.0, 0.0, &si, &ei);
      gmm_sum(1, c, j, j, 1.0, 0.0, 0.0, 0.0, &sj, &ej);
      c->f[q] = si + sj - 2.0 * v;
      if (c->bound) c->bound[q] = ei + ej + 2.0 * e;
    } else {
      c->f[q] = v;
      if (c->bound) c->bound[q] = e;
    }
  }
}

void or_gmm_pairs(int which, int dim, const int64_t *off, const float *x,
                  const float *y, const float *z, const float *sigma,
                  const float *w, int64_t n_pairs, const int64_t *pi,
                  const int64_t *pj, const double *params, double *out,
                  double *bound, int n_threads) {
  gmm_ctx g;
  memset(&g, 0, sizeof g);
  g.which = which;
  g.c.dim = dim; g.c.off = off; g.c.x = x; g.c.y = y; g.c.z = z; g.c.sigma = sigma;
  g.c.w = w; g.c.pi = pi; g.c.pj = pj; g.c.params = params; g.c.f = out; g.c.bound = bound;
  parallel_ranges(gmm_range, &g, n_pairs, n_threads);
}

static void gmm_self_range(void *vc, int64_t lo, int64_t hi) {
  const overlap_ctx *c = (const overlap_ctx *)vc;
  for (int64_t i = lo; i < hi; ++i) {
    double v, e;
    gmm_sum(1, c, i, i, 1.0, 0.0, 0.0, 0.0, &v, &e);
    c->f[i] = v;
    if (c->bound) c->bound[i] = e;
  }
}

void or_gmm_self(int dim, const int64_t *off, const float *x, const float *y,
                 const float *z, const float *sigma, const float *w,
                 int64_t n_items, double *S, double *bound, int n_threads) {
  overlap_ctx c;
  memset(&c, 0, sizeof c);
  c.dim = dim; c.off = off; c.x = x; c.y = y; c.z = z; c.sigma = sigma; c.w = w;
  c.f = S; c.bound = bound;
  parallel_ranges(gmm_self_range, &c, n_items, n_threads);
}

/* ------------------------------------------------------------------ */
/* Cosine of sparse composition vectors (Sec. V-B)                      */
/* ------------------------------------------------------------------ */

typedef struct {
  const int64_t *off;
  const int32_t *idx;
  const float *val;
  const int64_t *pi, *pj;
  double *c;
} sparse_ctx;

static double sparse_norm2(const sparse_ctx *s, int64_t i) {
  double t = 0.0;
  for (int64_t e = s->off[i]; e < s->off[i + 1]; ++e) t += (double)s->val[e] * (double)s->val[e];
  return t;
}

static void sparse_range(void *vc, int64_t lo, int64_t hi) {
  sparse_ctx *s = (sparse_ctx *)vc;
  for (int64_t q = lo; q < hi; ++q) {
    int64_t i = s->pi[q], j = s->pj[q];
    int64_t a = s->off[i], ae = s->off[i + 1], b = s->off[j], be = s->off[j + 1];
    double dot = 0.0;
    while (a < ae && b < be) {          /* merge of the two sorted index lists */
      if (s->idx[a] < s->idx[b]) ++a;
      else if (s->idx[a] > s->idx[b]) ++b;
      else { dot += (double)s->val[a] * (double)s->val[b]; ++a; ++b; }
    }
    double ni = sparse_norm2(s, i), nj = sparse_norm2(s, j);
    s->c[q] = (ni > 0.0 && nj > 0.0) ? dot / sqrt(ni * nj) : NAN;
  }
}

void or_sparse_cosine_pairs(const int64_t *off, const int32_t *idx, const float *val,
                            int64_t n_pairs, const int64_t *pi, const int64_t *pj,
                            double *c, int n_threads) {
  sparse_ctx s;
  s.off = off; s.idx = idx; s.val = val; s.pi = pi; s.pj = pj; s.c = c;
  parallel_ranges(sparse_range, &s, n_pairs, n_threads);
}

static void overlap_grad_range(void *vc, int64_t lo, int64_t hi) {
  overlap_ctx *c = (overlap_ctx *)vc;
  for (int64_t q = lo; q < hi; ++q) {
    int64_t i = c->pi[q], j = c->pj[q];
    double th = c->params ? c->params[3 * q] : 0.0;
    double tx = c->params ? c->params[3 * q + 1] : 0.0;
    double ty = c->params ? c->params[3 * q + 2] : 0.0;
    double cs = cos(th), sn = sin(th);
    double f = 0.0, gth = 0.0, gtx = 0.0, gty = 0.0;
    for (int64_t a = c->off[i]; a < c->off[i + 1]; ++a) {
      double wa = c->w ? (double)c->w[a] : 1.0;
      double sa = (double)c->sigma[a];
      for (int64_t b = c->off[j]; b < c->off[j + 1]; ++b) {
        double wb = c->w ? (double)c->w[b] : 1.0;
        double sb = (double)c->sigma[b];
        double xb = (double)c->x[b], yb = (double)c->y[b];
        double rx = cs * xb - sn * yb;          /* R x_b */
        double ry = sn * xb + cs * yb;
        double dx = (double)c->x[a] - (rx + tx); /* d = x_a - (R x_b + t) */
        double dy = (double)c->y[a] - (ry + ty);
        double s2 = sa * sa + sb * sb;
        double e = wa * wb * exp(-(dx * dx + dy * dy) / (2.0 * s2));
        /* J R x_b = (-ry, rx) */
        double jrx = -ry, jry = rx;
        f += e;
        gtx += e * dx / s2;
        gty += e * dy / s2;
        gth += e * (dx * jrx + dy * jry) / s2;
      }
    }
    c->f[q] = f;
    c->g[3 * q] = gth;
    c->g[3 * q + 1] = gtx;
    c->g[3 * q + 2] = gty;
  }
}

void or_overlap_grad_pairs(const int64_t *off, const float *x, const float *y,
                           const float *sigma, const float *w, int64_t n_pairs,
                           const int64_t *pi, const int64_t *pj,
                           const double *params, double *f, double *g,
                           int n_threads) {
  overlap_ctx c;
  memset(&c, 0, sizeof c);
  c.dim = 2; c.off = off; c.x = x; c.y = y; c.sigma = sigma; c.w = w;
  c.pi = pi; c.pj = pj; c.params = params; c.f = f; c.g = g;
  parallel_ranges(overlap_grad_range, &c, n_pairs, n_threads);
}

/* ------------------------------------------------------------------ */
/* batched gradient ascent on log f                                     */
/* ------------------------------------------------------------------ */

void or_ascent_step(const int64_t *off, const float *x, const float *y,
                    const float *sigma, const float *w, int64_t n_pairs,
                    const int64_t *pi, const int64_t *pj, double *params,
                    double eta, double fmin, double *f, double *g,
                    int32_t *flag, int n_threads) {
  or_overlap_grad_pairs(off, x, y, sigma, w, n_pairs, pi, pj, params, f, g,
                        n_threads);
  for (int64_t q = 0; q < n_pairs; ++q) {
    if (!(f[q] >= fmin)) { if (flag) flag[q] = 1; continue; }
    if (flag) flag[q] = 0;
    for (int k = 0; k < 3; ++k) params[3 * q + k] += eta * g[3 * q + k] / f[q];
  }
}

/* ------------------------------------------------------------------ */
/* Pearson correlation (normalised cross correlation, Sec. V-A)         */
/* ------------------------------------------------------------------ */

typedef struct {
  int64_t D, ld;
  const float *X;
  const double *mu, *ss;
  const int64_t *pi, *pj;
  int kahan;
  double *r, *mu_out, *ss_out;
} vec_ctx;

static void stats_range(void *vc, int64_t lo, int64_t hi) {
  vec_ctx *c = (vec_ctx *)vc;
  for (int64_t i = lo; i < hi; ++i) {
    const float *row = c->X + i * c->ld;
    double s = 0.0;
    for (int64_t k = 0; k < c->D; ++k) s += (double)row[k];
    double mu = s / (double)c->D;
    double ss = 0.0;
    for (int64_t k = 0; k < c->D; ++k) {
      double d = (double)row[k] - mu;
      ss += d * d;
    }
    c->mu_out[i] = mu;
    c->ss_out[i] = ss;
  }
}

void or_vector_stats(int64_t n_rows, int64_t D, int64_t ld, const float *X,
                     double *mu, double *ss, int n_threads) {
  vec_ctx c;
  memset(&c, 0, sizeof c);
  c.D = D; c.ld = ld; c.X = X; c.mu_out = mu; c.ss_out = ss;
  parallel_ranges(stats_range, &c, n_rows, n_threads);
}

static void pearson_range(void *vc, int64_t lo, int64_t hi) {
  vec_ctx *c = (vec_ctx *)vc;
  for (int64_t q = lo; q < hi; ++q) {
    int64_t i = c->pi[q], j = c->pj[q];
    const float *xi = c->X + i * c->ld, *xj = c->X + j * c->ld;
    double mi = c->mu[i], mj = c->mu[j];
    double s = 0.0, comp = 0.0;
    for (int64_t k = 0; k < c->D; ++k) {
      double p = ((double)xi[k] - mi) * ((double)xj[k] - mj);
      if (c->kahan) {
        double yk = p - comp;
        double t = s + yk;
        comp = (t - s) - yk;
        s = t;
      } else {
        s += p;
      }
    }
    c->r[q] = s / sqrt(c->ss[i] * c->ss[j]);
  }
}

void or_pearson_pairs(int64_t D, int64_t ld, const float *X, const double *mu,
                      const double *ss, int64_t n_pairs, const int64_t *pi,
                      const int64_t *pj, int kahan, double *r, int n_threads) {
  vec_ctx c;
  memset(&c, 0, sizeof c);
  c.D = D; c.ld = ld; c.X = X; c.mu = mu; c.ss = ss; c.pi = pi; c.pj = pj;
  c.kahan = kahan; c.r = r;
  parallel_ranges(pearson_range, &c, n_pairs, n_threads);
}
