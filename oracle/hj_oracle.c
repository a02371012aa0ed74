/*
 * hj_oracle.c -- plain, slow FP64 CPU oracle for the grid-based
 * Hamilton-Jacobi level-set solve of Herbert, Choi et al., "Scalable Learning
 * of Safety Guarantees for Autonomous Systems using Hamilton-Jacobi
 * Reachability" (arXiv 2101.05916).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only tests/, the smoke check of __graft_entry__ and the
 * cpu_baseline / reference legs of bench.py use it.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * What it computes (paper Sec. II-A, Eq. 1 and Eq. 2, written for
 * W := -V and l := -c so that the safe set is {W >= 0}):
 *
 *   W(x, 0) = l(x)                          (cold start, Eq. 2 terminal value)
 *   W(x, 0) = min(w(x), l(x))               (warm start, Sec. III-B)
 *   dW/ds   = H(x, grad W),  H(x,p) = max_u min_d  p . f(x,u,d)
 *   W       <- min(W, l)   after every full step (the max{c - V, .} branch
 *                                             of the variational inequality)
 *
 * integrated in backward time s until the change over a check window falls
 * below a tolerance (Sec. II-A: iterate "until convergence"; the converged
 * value is the infinite-horizon fixed point).  Optionally the stop test only
 * watches a band |W| <= band around the zero level set that bounds the safe
 * set S (Sec. II-A), and only nodes at least band_margin cells inside the
 * grid box.  High-order schemes on a truncated grid can keep cycling far
 * inside S and next to the faces where trajectories leave the grid, without
 * moving S.
 *
 * The paper names no numerical scheme.  The discrete operator below is the
 * textbook one (Osher & Fedkiw 2003, Sec. 3.3-3.4 and 5.3; Jiang & Peng 2000;
 * Shu & Osher 1988) with these readings, where the paper is silent:
 *   - first-order upwind, ENO2 or WENO5 one-sided differences per axis;
 *   - ghost nodes by linear extrapolation from the two outermost nodes;
 *   - global Lax-Friedrichs: L(W) = H(x, (p-+p+)/2) + sum_i a_i (p+_i - p-_i)/2
 *     with a_i = max over grid nodes and input vertices of |f_i|
 *     (the sign of the dissipation term is that of dW/ds = +H);
 *   - dt = CFL / sum_i a_i / h_i, constant for the whole solve;
 *   - TVD-RK3 (Shu-Osher form), clamp after the third stage;
 *   - WENO epsilon = 1e-6 * max v_k^2 + 1e-18 (divided differences).
 *
 * H is evaluated from its definition: maximum over the vertices of the control
 * box of the minimum over the vertices of the disturbance box of p . f.  For
 * dynamics affine in u and in d separately this is exact.  Nothing here uses
 * a closed-form bang-bang expression.
 *
 * Everything is double precision; loops are plain and unblocked; OpenMP only
 * splits the outermost loop over grid points.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXD 6
#define OR_MAXIN 6

/* models (the dynamics f of Sec. II-A) */
#define OR_DRIFT 0   /* n-D: f = d,  one disturbance per axis                       */
#define OR_QUAD_Z 1  /* 2-D vertical quadcopter (z, vz): f = (vz, kT u - g + d)     */
#define OR_QUAD_X4 2 /* 4-D near-hover subsystem (p, v, th, w) of Eq. 3            */

/* constraint shapes: margin l = -c with c the signed distance of Sec. II-A */
#define OR_CON_BOX 0       /* safe inside an axis-aligned box (+-inf = free axis) */
#define OR_CON_BALL_OUT 1  /* safe outside a ball                                 */
#define OR_CON_FIELD 2     /* margin l given node by node (lfield)                */

#define OR_CLAMP_VI 0
#define OR_CLAMP_MONOTONE 1

typedef struct {
  int ndim;
  long n[OR_MAXD];
  double lo[OR_MAXD];
  double hi[OR_MAXD];
  int model;
  double params[8];
  int nd;                 /* number of disturbance inputs                       */
  double d_lo[OR_MAXIN];  /* disturbance box                                    */
  double d_hi[OR_MAXIN];
  int con_kind;
  double con_a[OR_MAXD];  /* box lo, or ball centre                              */
  double con_b[OR_MAXD];  /* box hi, or ball radius in con_b[0]                  */
  const double* dflo;     /* state-dependent disturbance box (Sec. II-C): input  */
  const double* dfhi;     /* j's bound at node k is [j * npts + k]; NULL = box   */
  const double* lfield;   /* OR_CON_FIELD: the margin l = -c at every node       */
} or_problem;

typedef struct {
  int scheme;        /* 1 = first-order upwind, 2 = ENO2, 5 = WENO5       */
  double cfl;
  double dt;         /* > 0: use this dt instead of the CFL rule          */
  double tol;
  double check_dt;   /* window length in simulated seconds                */
  long max_steps;
  long fixed_steps;  /* > 0: run exactly this many steps, no stop test    */
  int clamp;
  int warm;          /* 0 = start from l, 1 = start from min(W_in, l)     */
  double band;       /* > 0: the stop test only watches nodes with
                        min(|W|, |W_window_start|) <= band                 */
  int band_margin;   /* the stop test skips nodes closer than this many
                        cells to a face of an axis the box constraint
                        leaves free (every axis for a ball)                 */
} or_opts;

typedef struct {
  long steps;
  double t;
  double residual;
  double dt;
  int converged;
  long windows;
} or_stats;

/* ------------------------------------------------------------------ grid */

static double grid_h(const or_problem* P, int d) {
  return (P->hi[d] - P->lo[d]) / (double)(P->n[d] - 1);
}

static long grid_npts(const or_problem* P) {
  long m = 1;
  for (int d = 0; d < P->ndim; ++d) m *= P->n[d];
  return m;
}

/* row-major: the last axis is the fastest */
static long grid_stride(const or_problem* P, int d) {
  long s = 1;
  for (int e = P->ndim - 1; e > d; --e) s *= P->n[e];
  return s;
}

static void grid_unravel(const or_problem* P, long p, long* idx) {
  for (int d = P->ndim - 1; d >= 0; --d) {
    idx[d] = p % P->n[d];
    p /= P->n[d];
  }
}

static void grid_coords(const or_problem* P, const long* idx, double* x) {
  for (int d = 0; d < P->ndim; ++d) x[d] = P->lo[d] + (double)idx[d] * grid_h(P, d);
}

/* ------------------------------------------------------------ constraint */

/* l(x) = -c(x): the signed distance to the constraint set, positive inside
 * the safe region (Sec. II-A, "signed distance function").  For a box the
 * distance is taken in raw state units over the constrained axes only. */
double or_margin(const or_problem* P, const double* x) {
  if (P->con_kind == OR_CON_BALL_OUT) {
    double s = 0.0;
    for (int d = 0; d < P->ndim; ++d) {
      double e = x[d] - P->con_a[d];
      s += e * e;
    }
    return sqrt(s) - P->con_b[0];
  }
  int inside = 1;
  double m = INFINITY, out2 = 0.0;
  for (int d = 0; d < P->ndim; ++d) {
    double lo = P->con_a[d], hi = P->con_b[d];
    if (isinf(lo) && isinf(hi)) continue;
    double below = lo - x[d], above = x[d] - hi;
    if (below > 0.0) { inside = 0; out2 += below * below; }
    else if (above > 0.0) { inside = 0; out2 += above * above; }
    double in_d = fmin(x[d] - lo, hi - x[d]);
    if (in_d < m) m = in_d;
  }
  return inside ? m : -sqrt(out2);
}

/* -------------------------------------------------------------- dynamics */

static int model_nu(const or_problem* P) {
  return (P->model == OR_DRIFT) ? 0 : 1;
}

static void model_u_box(const or_problem* P, double* ulo, double* uhi) {
  if (P->model == OR_QUAD_Z) { ulo[0] = P->params[2]; uhi[0] = P->params[3]; }
  if (P->model == OR_QUAD_X4) { ulo[0] = P->params[4]; uhi[0] = P->params[5]; }
}

/* f(x, u, d) written out per model */
static void model_f(const or_problem* P, const double* x, const double* u,
                    const double* dd, double* f) {
  const double* q = P->params;
  switch (P->model) {
    case OR_DRIFT:
      for (int i = 0; i < P->ndim; ++i) f[i] = dd[i];
      break;
    case OR_QUAD_Z: /* q = (kT, g, u_lo, u_hi) */
      f[0] = x[1];
      f[1] = q[0] * u[0] - q[1] + dd[0];
      break;
    case OR_QUAD_X4: { /* q = (g, d1, d0, n0, u_lo, u_hi, dist_axis) */
      int ax = (int)q[6];
      f[0] = x[1];
      f[1] = q[0] * tan(x[2]);
      f[2] = -q[1] * x[2] + x[3];
      f[3] = -q[2] * x[2] + q[3] * u[0];
      f[ax] += dd[0];
      break;
    }
  }
}

/* vertex k of a box of dimension m (bit i of k picks hi on axis i) */
static void box_vertex(int m, const double* lo, const double* hi, int k, double* v) {
  for (int i = 0; i < m; ++i) v[i] = ((k >> i) & 1) ? hi[i] : lo[i];
}

/* Disturbance box at node pt: the state-dependent field when set, else the
 * uniform box. */
static void dist_box(const or_problem* P, long pt, double* lo, double* hi) {
  long npts = 1;
  for (int d = 0; d < P->ndim; ++d) npts *= P->n[d];
  for (int j = 0; j < P->nd; ++j) {
    lo[j] = P->dflo ? P->dflo[j * npts + pt] : P->d_lo[j];
    hi[j] = P->dfhi ? P->dfhi[j * npts + pt] : P->d_hi[j];
  }
}

/* H(x, p) = max_u min_d p . f(x, u, d) over the input boxes' vertices, with
 * the disturbance box (dlo, dhi) */
static double hamiltonian_box(const or_problem* P, const double* x, const double* p,
                              const double* dlo, const double* dhi) {
  double ulo[OR_MAXIN] = {0}, uhi[OR_MAXIN] = {0}, u[OR_MAXIN] = {0}, dd[OR_MAXIN] = {0};
  double f[OR_MAXD];
  int nu = model_nu(P);
  model_u_box(P, ulo, uhi);
  double best = -INFINITY;
  for (int ku = 0; ku < (1 << nu); ++ku) {
    box_vertex(nu, ulo, uhi, ku, u);
    double worst = INFINITY;
    for (int kd = 0; kd < (1 << P->nd); ++kd) {
      box_vertex(P->nd, dlo, dhi, kd, dd);
      model_f(P, x, u, dd, f);
      double s = 0.0;
      for (int i = 0; i < P->ndim; ++i) s += p[i] * f[i];
      if (s < worst) worst = s;
    }
    if (worst > best) best = worst;
  }
  return best;
}

/* H(x, p) = max_u min_d p . f(x, u, d), by enumeration of input-box vertices,
 * with the uniform disturbance box */
double or_hamiltonian(const or_problem* P, const double* x, const double* p) {
  return hamiltonian_box(P, x, p, P->d_lo, P->d_hi);
}

/* a_i = max over grid nodes and input vertices of |f_i(x, u, d)| */
void or_alpha(const or_problem* P, double* alpha) {
  double ulo[OR_MAXIN] = {0}, uhi[OR_MAXIN] = {0};
  int nu = model_nu(P);
  model_u_box(P, ulo, uhi);
  long npts = grid_npts(P);
  for (int i = 0; i < P->ndim; ++i) alpha[i] = 0.0;
  for (long pt = 0; pt < npts; ++pt) {
    long idx[OR_MAXD];
    double x[OR_MAXD], f[OR_MAXD], u[OR_MAXIN] = {0}, dd[OR_MAXIN] = {0};
    double dlo[OR_MAXIN], dhi[OR_MAXIN];
    grid_unravel(P, pt, idx);
    grid_coords(P, idx, x);
    dist_box(P, pt, dlo, dhi);
    for (int ku = 0; ku < (1 << nu); ++ku) {
      box_vertex(nu, ulo, uhi, ku, u);
      for (int kd = 0; kd < (1 << P->nd); ++kd) {
        box_vertex(P->nd, dlo, dhi, kd, dd);
        model_f(P, x, u, dd, f);
        for (int i = 0; i < P->ndim; ++i)
          if (fabs(f[i]) > alpha[i]) alpha[i] = fabs(f[i]);
      }
    }
  }
}

/* dt = CFL / sum_i a_i / h_i; 0 when nothing moves */
double or_cfl_dt(const or_problem* P, double cfl, const double* alpha) {
  double s = 0.0;
  for (int i = 0; i < P->ndim; ++i) s += alpha[i] / grid_h(P, i);
  return (s > 0.0) ? cfl / s : 0.0;
}

/* ------------------------------------------------------ one-sided slopes */

/* Value of the line at virtual index j (may lie outside [0, n)): ghost nodes
 * continue the line linearly through its two outermost nodes. */
static double line_at(const double* W, long base, long stride, long n, long j) {
  if (j < 0) {
    double w0 = W[base], w1 = W[base + stride];
    return w0 + (double)(-j) * (w0 - w1);
  }
  if (j > n - 1) {
    double wn = W[base + (n - 1) * stride], wm = W[base + (n - 2) * stride];
    return wn + (double)(j - (n - 1)) * (wn - wm);
  }
  return W[base + j * stride];
}

/* ENO2 (Osher & Fedkiw Sec. 3.3): the first divided difference plus the
 * second-order correction from the smoother of the two candidate stencils.
 * v[k] holds the line at offset k-2 (k = 0..4).  Ties take the left one. */
static void eno2(const double* v, double h, double* pm, double* pp) {
  double a = v[2] - 2.0 * v[1] + v[0]; /* second difference at i-1 */
  double b = v[3] - 2.0 * v[2] + v[1]; /* at i                      */
  double c = v[4] - 2.0 * v[3] + v[2]; /* at i+1                    */
  double m1 = (fabs(a) <= fabs(b)) ? a : b;
  double m2 = (fabs(b) <= fabs(c)) ? b : c;
  *pm = (v[2] - v[1]) / h + m1 / (2.0 * h);
  *pp = (v[3] - v[2]) / h - m2 / (2.0 * h);
}

/* WENO5 of Jiang & Peng (Osher & Fedkiw Sec. 3.4) applied to five divided
 * differences q1..q5 ordered in the upwind direction. */
static double weno5_combine(double q1, double q2, double q3, double q4, double q5) {
  double phi1 = q1 / 3.0 - 7.0 * q2 / 6.0 + 11.0 * q3 / 6.0;
  double phi2 = -q2 / 6.0 + 5.0 * q3 / 6.0 + q4 / 3.0;
  double phi3 = q3 / 3.0 + 5.0 * q4 / 6.0 - q5 / 6.0;
  double s1 = 13.0 / 12.0 * (q1 - 2.0 * q2 + q3) * (q1 - 2.0 * q2 + q3)
            + 0.25 * (q1 - 4.0 * q2 + 3.0 * q3) * (q1 - 4.0 * q2 + 3.0 * q3);
  double s2 = 13.0 / 12.0 * (q2 - 2.0 * q3 + q4) * (q2 - 2.0 * q3 + q4)
            + 0.25 * (q2 - q4) * (q2 - q4);
  double s3 = 13.0 / 12.0 * (q3 - 2.0 * q4 + q5) * (q3 - 2.0 * q4 + q5)
            + 0.25 * (3.0 * q3 - 4.0 * q4 + q5) * (3.0 * q3 - 4.0 * q4 + q5);
  double mx = q1 * q1;
  if (q2 * q2 > mx) mx = q2 * q2;
  if (q3 * q3 > mx) mx = q3 * q3;
  if (q4 * q4 > mx) mx = q4 * q4;
  if (q5 * q5 > mx) mx = q5 * q5;
  double eps = 1e-6 * mx + 1e-18;
  double a1 = 0.1 / ((s1 + eps) * (s1 + eps));
  double a2 = 0.6 / ((s2 + eps) * (s2 + eps));
  double a3 = 0.3 / ((s3 + eps) * (s3 + eps));
  double sum = a1 + a2 + a3;
  return (a1 * phi1 + a2 * phi2 + a3 * phi3) / sum;
}

/* v[k] holds the line at offset k-3 (k = 0..6) */
static void weno5(const double* v, double h, double* pm, double* pp) {
  double D[6]; /* D[k] = (v[k+1] - v[k]) / h, the difference ending at offset k-2 */
  for (int k = 0; k < 6; ++k) D[k] = (v[k + 1] - v[k]) / h;
  /* left-biased: differences ending at i-2, i-1, i, i+1, i+2 */
  *pm = weno5_combine(D[0], D[1], D[2], D[3], D[4]);
  /* right-biased: forward differences at i+2, i+1, i, i-1, i-2 */
  *pp = weno5_combine(D[5], D[4], D[3], D[2], D[1]);
}

static void first_order(const double* v, double h, double* pm, double* pp) {
  *pm = (v[1] - v[0]) / h;
  *pp = (v[2] - v[1]) / h;
}

/* Exported for unit tests: one-sided slopes at every node of a 1-D line. */
void or_line_slopes(const double* W, long n, double h, int scheme, double* pm, double* pp) {
  int r = (scheme == 5) ? 3 : (scheme == 2) ? 2 : 1;
  for (long i = 0; i < n; ++i) {
    double v[7];
    for (int k = -r; k <= r; ++k) v[k + r] = line_at(W, 0, 1, n, i + k);
    if (scheme == 5) weno5(v, h, &pm[i], &pp[i]);
    else if (scheme == 2) eno2(v, h, &pm[i], &pp[i]);
    else first_order(v, h, &pm[i], &pp[i]);
  }
}

/* ------------------------------------------------------------ operators */

/* L(W) at every node: Lax-Friedrichs numerical Hamiltonian for dW/ds = H. */
static void lf_rhs(const or_problem* P, int scheme, const double* alpha,
                   const double* W, double* out) {
  long npts = grid_npts(P);
  int r = (scheme == 5) ? 3 : (scheme == 2) ? 2 : 1;
#pragma omp parallel for schedule(static)
  for (long pt = 0; pt < npts; ++pt) {
    long idx[OR_MAXD] = {0};
    double x[OR_MAXD] = {0}, pm[OR_MAXD] = {0}, pp[OR_MAXD] = {0}, pbar[OR_MAXD] = {0};
    grid_unravel(P, pt, idx);
    grid_coords(P, idx, x);
    for (int d = 0; d < P->ndim; ++d) {
      long s = grid_stride(P, d);
      long base = pt - idx[d] * s;
      double v[7];
      for (int k = -r; k <= r; ++k) v[k + r] = line_at(W, base, s, P->n[d], idx[d] + k);
      double h = grid_h(P, d);
      if (scheme == 5) weno5(v, h, &pm[d], &pp[d]);
      else if (scheme == 2) eno2(v, h, &pm[d], &pp[d]);
      else first_order(v, h, &pm[d], &pp[d]);
      pbar[d] = 0.5 * (pm[d] + pp[d]);
    }
    double dlo[OR_MAXIN], dhi[OR_MAXIN];
    dist_box(P, pt, dlo, dhi);
    double L = hamiltonian_box(P, x, pbar, dlo, dhi);
    for (int d = 0; d < P->ndim; ++d) L += alpha[d] * 0.5 * (pp[d] - pm[d]);
    out[pt] = L;
  }
}

static void fill_margin(const or_problem* P, double* l) {
  long npts = grid_npts(P);
#pragma omp parallel for schedule(static)
  for (long pt = 0; pt < npts; ++pt) {
    long idx[OR_MAXD];
    double x[OR_MAXD];
    grid_unravel(P, pt, idx);
    grid_coords(P, idx, x);
    l[pt] = P->con_kind == OR_CON_FIELD ? P->lfield[pt] : or_margin(P, x);
  }
}

/* One TVD-RK3 step (Shu & Osher) followed by the variational-inequality clamp. */
static void rk3_step(const or_problem* P, int scheme, int clamp, const double* alpha,
                     double dt, const double* l, double* W, double* W1, double* W2,
                     double* L) {
  long npts = grid_npts(P);
  lf_rhs(P, scheme, alpha, W, L);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < npts; ++i) W1[i] = W[i] + dt * L[i];
  lf_rhs(P, scheme, alpha, W1, L);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < npts; ++i) W2[i] = 0.75 * W[i] + 0.25 * (W1[i] + dt * L[i]);
  lf_rhs(P, scheme, alpha, W2, L);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < npts; ++i) {
    double w3 = W[i] / 3.0 + 2.0 / 3.0 * (W2[i] + dt * L[i]);
    double wn = fmin(w3, l[i]);
    if (clamp == OR_CLAMP_MONOTONE) wn = fmin(wn, W[i]);
    W[i] = wn;
  }
}

/* Full solve.  W holds the warm-start value on entry when o->warm is set and
 * the result on return.  Returns 0 on success, 1 when the step cap was hit,
 * negative on bad arguments. */
int or_solve(const or_problem* P, const or_opts* o, double* W, or_stats* st) {
  if (P->ndim < 1 || P->ndim > OR_MAXD) return -1;
  for (int d = 0; d < P->ndim; ++d)
    if (P->n[d] < 3 || !(P->hi[d] > P->lo[d])) return -1;
  if (o->scheme != 1 && o->scheme != 2 && o->scheme != 5) return -1;
  long npts = grid_npts(P);
  double* l = malloc(sizeof(double) * npts);
  double* W1 = malloc(sizeof(double) * npts);
  double* W2 = malloc(sizeof(double) * npts);
  double* L = malloc(sizeof(double) * npts);
  double* snap = malloc(sizeof(double) * npts);
  fill_margin(P, l);
  for (long i = 0; i < npts; ++i) W[i] = o->warm ? fmin(W[i], l[i]) : l[i];

  double alpha[OR_MAXD];
  or_alpha(P, alpha);
  double dt = (o->dt > 0.0) ? o->dt : or_cfl_dt(P, o->cfl, alpha);
  memset(st, 0, sizeof(*st));
  st->dt = dt;
  int rc = 0;
  if (dt <= 0.0) {
    /* no motion at all: W = min(W0, l) is already the fixed point */
    st->converged = 1;
  } else if (o->fixed_steps > 0) {
    for (long k = 0; k < o->fixed_steps; ++k)
      rk3_step(P, o->scheme, o->clamp, alpha, dt, l, W, W1, W2, L);
    st->steps = o->fixed_steps;
  } else {
    long per = (long)ceil(o->check_dt / dt - 1e-9);
    if (per < 1) per = 1;
    for (;;) {
      memcpy(snap, W, sizeof(double) * npts);
      long todo = per;
      if (o->max_steps > 0 && st->steps + todo > o->max_steps) todo = o->max_steps - st->steps;
      for (long k = 0; k < todo; ++k)
        rk3_step(P, o->scheme, o->clamp, alpha, dt, l, W, W1, W2, L);
      st->steps += todo;
      st->windows += 1;
      double r = 0.0;
      for (long i = 0; i < npts; ++i) {
        if (o->band > 0.0 && fmin(fabs(W[i]), fabs(snap[i])) > o->band) continue;
        if (o->band_margin > 0) {
          /* faces of axes the box constraint leaves free */
          long idx[OR_MAXD];
          grid_unravel(P, i, idx);
          int inside = 1;
          for (int d = 0; d < P->ndim; ++d) {
            int constrained = P->con_kind == OR_CON_BOX &&
                              !(isinf(P->con_a[d]) && isinf(P->con_b[d]));
            if (constrained) continue;
            if (idx[d] < o->band_margin || idx[d] > P->n[d] - 1 - o->band_margin) inside = 0;
          }
          if (!inside) continue;
        }
        double e = fabs(W[i] - snap[i]);
        if (e > r) r = e;
      }
      st->residual = r;
      if (r < o->tol) { st->converged = 1; break; }
      if (o->max_steps > 0 && st->steps >= o->max_steps) { rc = 1; break; }
    }
  }
  st->t = dt * (double)st->steps;
  free(l); free(W1); free(W2); free(L); free(snap);
  return rc;
}

/* Fill l at every node (exported for tests). */
void or_fill_margin(const or_problem* P, double* l) { fill_margin(P, l); }

/* ------------------------------------------------- prolongation, queries */

/* Multilinear interpolation of a grid function at an arbitrary point inside
 * the grid box.  Returns 0, or -1 when the point is outside. */
static int interp(const or_problem* G, const double* F, const double* x, double* out) {
  long i0[OR_MAXD];
  double fr[OR_MAXD];
  for (int d = 0; d < G->ndim; ++d) {
    double h = grid_h(G, d);
    double tol = 1e-9 * h;
    if (x[d] < G->lo[d] - tol || x[d] > G->hi[d] + tol) return -1;
    double t = (x[d] - G->lo[d]) / h;
    long i = (long)floor(t);
    if (i < 0) i = 0;
    if (i > G->n[d] - 2) i = G->n[d] - 2;
    double f = t - (double)i;
    if (f < 0.0) f = 0.0;
    if (f > 1.0) f = 1.0;
    i0[d] = i;
    fr[d] = f;
  }
  double acc = 0.0;
  for (int c = 0; c < (1 << G->ndim); ++c) {
    double wgt = 1.0;
    long off = 0;
    for (int d = 0; d < G->ndim; ++d) {
      int bit = (c >> d) & 1;
      wgt *= bit ? fr[d] : 1.0 - fr[d];
      off += (i0[d] + bit) * grid_stride(G, d);
    }
    acc += wgt * F[off];
  }
  *out = acc;
  return 0;
}

/* Coarse-to-fine migration (Sec. III-C): multilinear interpolation of the
 * coarse value at every fine node, then min with the fine margin. */
int or_prolong(const or_problem* C, const double* Wc, const or_problem* Fp, double* Wf) {
  if (C->ndim != Fp->ndim) return -1;
  long npts = grid_npts(Fp);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (long pt = 0; pt < npts; ++pt) {
    long idx[OR_MAXD];
    double x[OR_MAXD], v;
    grid_unravel(Fp, pt, idx);
    grid_coords(Fp, idx, x);
    if (interp(C, Wc, x, &v) != 0) { bad |= 1; continue; }
    Wf[pt] = fmin(v, Fp->con_kind == OR_CON_FIELD ? Fp->lfield[pt] : or_margin(Fp, x));
  }
  return bad ? -1 : 0;
}

int or_query_value(const or_problem* G, const double* W, long npts, const double* xs, double* out) {
  for (long k = 0; k < npts; ++k)
    if (interp(G, W, xs + k * G->ndim, &out[k]) != 0) return -1;
  return 0;
}

/* Node gradient: central differences inside, one-sided at the two ends of
 * each axis; then multilinear interpolation of each component. */
int or_query_gradient(const or_problem* G, const double* W, long npts, const double* xs,
                      double* out) {
  long m = grid_npts(G);
  double* g = malloc(sizeof(double) * m);
  int rc = 0;
  for (int d = 0; d < G->ndim && rc == 0; ++d) {
    long s = grid_stride(G, d);
    double h = grid_h(G, d);
    for (long pt = 0; pt < m; ++pt) {
      long idx[OR_MAXD];
      grid_unravel(G, pt, idx);
      long i = idx[d];
      if (i == 0) g[pt] = (W[pt + s] - W[pt]) / h;
      else if (i == G->n[d] - 1) g[pt] = (W[pt] - W[pt - s]) / h;
      else g[pt] = (W[pt + s] - W[pt - s]) / (2.0 * h);
    }
    for (long k = 0; k < npts; ++k) {
      double v;
      if (interp(G, g, xs + k * G->ndim, &v) != 0) { rc = -1; break; }
      out[k * G->ndim + d] = v;
    }
  }
  free(g);
  return rc;
}

/* One call of the right-hand side L(W) (exported for tests). */
void or_rhs(const or_problem* P, int scheme, const double* W, double* out) {
  double alpha[OR_MAXD];
  or_alpha(P, alpha);
  lf_rhs(P, scheme, alpha, W, out);
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int k) {
#ifdef _OPENMP
  if (k > 0) omp_set_num_threads(k);
#else
  (void)k;
#endif
}
