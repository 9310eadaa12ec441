/*
 * CPU FP64 oracle for the time-global implicit-Euler system.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links or calls
 * this file; only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header, table or constant
 * with the CUDA path.
 *
 * What it computes is the plain definition the whole method must reproduce:
 * sequential implicit Euler time stepping (§2, eq. 2.1)
 *
 *     M (u_n - u_{n-1}) + tau_n A_n u_n = tau_n M f_n,   u_0 = u_I,
 *
 * with M = I (finite differences, mass = 0) or, for mass = 1 (dim <= 2), the P1
 * finite-element mass matrix of the uniform mesh divided by h^d (1-D: the
 * tridiagonal [1/6, 2/3, 1/6]; 2-D, each grid square cut by its diagonal from
 * the lower-left to the upper-right corner: 1/2 at the point and 1/12 at the
 * four axis neighbours and at the upper-right and lower-left diagonal ones),
 * and the source entering as the consistent load M f_n of its nodal values.
 * The finite-element stiffness matrix of the coefficient taken at the edge
 * midpoints is h^d times the finite-difference operator below, so dividing the
 * finite-element system by h^d gives exactly this one.  Time steps tau_n
 * (uniform T/N unless the
 * caller passes the N step lengths; then t_n = tau_1 + ... + tau_n), on the
 * unit box with n_d interior points per axis, h_d = 1/(n_d+1), homogeneous
 * Dirichlet data, and the conservative finite-difference operator
 *
 *   (A_n v)_i = sum_d h_d^-2 [ a(x_i - h_d e_d/2, t_n) (v_i - v_{i-e_d})
 *                             + a(x_i + h_d e_d/2, t_n) (v_i - v_{i+e_d}) ]
 *
 * (coefficient sampled at face midpoints, v = 0 outside the grid).  Each
 * step factors M + tau A_n by a hand-written banded Cholesky (band = one
 * grid line / plane, one more for the 2-D P1 mass) and solves; for grids where
 * the band is too wide the per-step solve is conjugate gradients to a relative
 * residual of cg_tol.
 *
 * Also provided: the action of the time-global matrix B = K (x) M +
 * diag(tau_n A_n) of §2, eq. 2.3-2.4, used to check residuals at any size.
 *
 * Coefficient model:  a(x,t) = a0 + c * prod_d g_d(pi m_d x_d) * g_t(pi m_t t)
 * with g in {1, sin, cos}.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double a0, c;
  int fx[3];
  double mx[3];
  int ft;
  double mt;
} oc_coeff;

static double oc_trig(int kind, double arg) {
  if (kind == 1) return sin(arg);
  if (kind == 2) return cos(arg);
  return 1.0;
}

/* a(x, t) at a point given by its coordinates (dim entries of x). */
static double oc_coef(const oc_coeff* k, int dim, const double* x, double t) {
  double g = k->c * oc_trig(k->ft, M_PI * k->mt * t);
  for (int d = 0; d < dim; ++d) g *= oc_trig(k->fx[d], M_PI * k->mx[d] * x[d]);
  return k->a0 + g;
}

typedef struct {
  int dim;
  int n[3];
  long stride[3];
  long ns;
  double h[3];
} oc_grid;

static void oc_grid_init(oc_grid* g, int dim, const int* n) {
  g->dim = dim;
  g->ns = 1;
  for (int d = 0; d < 3; ++d) {
    g->n[d] = d < dim ? n[d] : 1;
    g->h[d] = d < dim ? 1.0 / (n[d] + 1) : 0.0;
  }
  g->stride[0] = 1;
  g->stride[1] = g->n[0];
  g->stride[2] = (long)g->n[0] * g->n[1];
  for (int d = 0; d < dim; ++d) g->ns *= g->n[d];
}

static void oc_coords(const oc_grid* g, long i, int* idx) {
  for (int d = 0; d < 3; ++d) {
    idx[d] = (int)(i % g->n[d]);
    i /= g->n[d];
  }
}

/* Face coefficients of point i along axis d: lower face (minus) and upper face (plus).
 * Grid node j (0..n+1, 0 and n+1 on the boundary) sits at j*h; the face between
 * nodes j and j+1 sits at (j + 1/2) h, so a face shared by two points is
 * evaluated from the same coordinate on both sides. */
static void oc_faces(const oc_grid* g, const oc_coeff* k, double t, const int* idx, int d,
                     double* am, double* ap) {
  double x[3];
  for (int e = 0; e < g->dim; ++e) x[e] = (idx[e] + 1) * g->h[e];
  x[d] = (idx[d] + 0.5) * g->h[d];
  *am = oc_coef(k, g->dim, x, t);
  x[d] = (idx[d] + 1.5) * g->h[d];
  *ap = oc_coef(k, g->dim, x, t);
}

/* out = M v for one spatial slice (mass 0: M = I; 1: the P1 mass over h^d, dim <= 2). */
static void oc_apply_M_slice(const oc_grid* g, int mass, const double* v, double* out) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < g->ns; ++i) {
    if (mass == 0) {
      out[i] = v[i];
      continue;
    }
    int idx[3];
    oc_coords(g, i, idx);
    if (g->dim == 1) {
      double vm = idx[0] > 0 ? v[i - 1] : 0.0;
      double vp = idx[0] < g->n[0] - 1 ? v[i + 1] : 0.0;
      out[i] = (2.0 / 3.0) * v[i] + (vm + vp) / 6.0;
    } else {
      int x = idx[0], y = idx[1], nx = g->n[0], ny = g->n[1];
      long sy = g->stride[1];
      double s = 0.0;
      if (x > 0) s += v[i - 1];
      if (x < nx - 1) s += v[i + 1];
      if (y > 0) s += v[i - sy];
      if (y < ny - 1) s += v[i + sy];
      if (x > 0 && y > 0) s += v[i - sy - 1];
      if (x < nx - 1 && y < ny - 1) s += v[i + sy + 1];
      out[i] = 0.5 * v[i] + s / 12.0;
    }
  }
}

/* out = A(t) v for one spatial slice. */
static void oc_apply_A_slice(const oc_grid* g, const oc_coeff* k, double t, const double* v,
                             double* out) {
#pragma omp parallel for schedule(static)
  for (long i = 0; i < g->ns; ++i) {
    int idx[3];
    oc_coords(g, i, idx);
    double s = 0.0;
    for (int d = 0; d < g->dim; ++d) {
      double am, ap;
      oc_faces(g, k, t, idx, d, &am, &ap);
      double vm = idx[d] > 0 ? v[i - g->stride[d]] : 0.0;
      double vp = idx[d] < g->n[d] - 1 ? v[i + g->stride[d]] : 0.0;
      s += (am * (v[i] - vm) + ap * (v[i] - vp)) / (g->h[d] * g->h[d]);
    }
    out[i] = s;
  }
}

/* ---- banded Cholesky of M + tau A(t) ----------------------------------
 * Lower band storage, column major: ab[j*(b+1) + (i-j)] = M[i][j], j <= i <= j+b.
 * b is the stride of the slowest axis (one grid line in 2-D, one plane in 3-D), plus one
 * for the upper-right diagonal coupling of the 2-D P1 mass. */
static void oc_assemble_band(const oc_grid* g, const oc_coeff* k, double t, double tau, long b,
                             int mass, double* ab) {
  memset(ab, 0, sizeof(double) * (size_t)(b + 1) * (size_t)g->ns);
  const double mc = mass == 0 ? 1.0 : (g->dim == 1 ? 2.0 / 3.0 : 0.5);
  const double mo = mass == 0 ? 0.0 : (g->dim == 1 ? 1.0 / 6.0 : 1.0 / 12.0);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < g->ns; ++i) {
    int idx[3];
    oc_coords(g, i, idx);
    double diag = mc;
    for (int d = 0; d < g->dim; ++d) {
      double am, ap, w = tau / (g->h[d] * g->h[d]);
      oc_faces(g, k, t, idx, d, &am, &ap);
      diag += w * (am + ap);
      /* coupling to the upper neighbour (row i + stride, column i) */
      if (idx[d] < g->n[d] - 1) ab[i * (b + 1) + g->stride[d]] = -w * ap + mo;
    }
    /* 2-D P1 mass: the upper-right diagonal neighbour (row i + stride + 1, column i) */
    if (mass && g->dim == 2 && idx[0] < g->n[0] - 1 && idx[1] < g->n[1] - 1)
      ab[i * (b + 1) + g->stride[1] + 1] = mo;
    ab[i * (b + 1)] = diag;
  }
}

static int oc_band_cholesky(long n, long b, double* ab) {
  for (long j = 0; j < n; ++j) {
    double* cj = ab + j * (b + 1);
    if (!(cj[0] > 0.0)) return -1;
    double d = sqrt(cj[0]);
    cj[0] = d;
    long m = b < n - 1 - j ? b : n - 1 - j;
    for (long i = 1; i <= m; ++i) cj[i] /= d;
    /* trailing update of the (m x m) lower triangle */
#pragma omp parallel for schedule(static, 8) if (m >= 64)
    for (long kk = 1; kk <= m; ++kk) {
      double lk = cj[kk];
      if (lk == 0.0) continue;
      double* ck = ab + (j + kk) * (b + 1);
      for (long i = kk; i <= m; ++i) ck[i - kk] -= cj[i] * lk;
    }
  }
  return 0;
}

static void oc_band_solve(long n, long b, const double* ab, double* x) {
  /* L y = x */
  for (long j = 0; j < n; ++j) {
    const double* cj = ab + j * (b + 1);
    x[j] /= cj[0];
    long m = b < n - 1 - j ? b : n - 1 - j;
    double xj = x[j];
    for (long i = 1; i <= m; ++i) x[j + i] -= cj[i] * xj;
  }
  /* L^T x = y */
  for (long j = n - 1; j >= 0; --j) {
    const double* cj = ab + j * (b + 1);
    long m = b < n - 1 - j ? b : n - 1 - j;
    double s = x[j];
    for (long i = 1; i <= m; ++i) s -= cj[i] * x[j + i];
    x[j] = s / cj[0];
  }
}

/* ---- conjugate gradients on M + tau A(t) ------------------------------ */
static double oc_dot(long n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (long i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static int oc_cg(const oc_grid* g, const oc_coeff* k, double t, double tau, int mass, const double* rhs,
                 double* x, double tol, int max_it, double* work) {
  long n = g->ns;
  double *r = work, *p = work + n, *q = work + 2 * n, *m = work + 3 * n;
  /* x holds the initial guess */
  oc_apply_A_slice(g, k, t, x, q);
  oc_apply_M_slice(g, mass, x, m);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) {
    r[i] = rhs[i] - (m[i] + tau * q[i]);
    p[i] = r[i];
  }
  double bb = oc_dot(n, rhs, rhs);
  double rr = oc_dot(n, r, r);
  if (bb == 0.0) bb = 1.0;
  int it = 0;
  while (rr > tol * tol * bb && it < max_it) {
    oc_apply_A_slice(g, k, t, p, q);
    oc_apply_M_slice(g, mass, p, m);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) q[i] = m[i] + tau * q[i];
    double alpha = rr / oc_dot(n, p, q);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    double rr_new = oc_dot(n, r, r);
    double beta = rr_new / rr;
    rr = rr_new;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    ++it;
  }
  return rr <= tol * tol * bb ? it : -1;
}

/*
 * Sequential implicit Euler, steps n = 1..n_steps (n_steps <= N).
 *   f  : [N][ns]  source values f(x_i, t_n), x fastest
 *   u0 : [ns] initial datum u_I, or NULL for zero
 *   u  : [n_steps][ns] output
 *   method : 0 = banded Cholesky, 1 = CG to relative residual cg_tol
 *   mass   : 0 = M = I, 1 = P1 mass over h^d (dim <= 2)
 * Returns 0 on success, -1 on a failed factorization, -2 on CG failure,
 * -3 on allocation failure, -4 on an unsupported mass.
 */
int oc_implicit_euler(int dim, const int* n, int N, double T, const oc_coeff* k,
                      const double* f, const double* u0, double* u, int n_steps, int method,
                      double cg_tol, int nthreads, const double* steps, int mass) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  oc_grid g;
  oc_grid_init(&g, dim, n);
  if (mass != 0 && (mass != 1 || dim > 2)) return -4;
  long ns = g.ns;
  long b = dim == 1 ? 1 : g.stride[dim - 1] + (mass && dim == 2 ? 1 : 0);
  double tau = T / N;
  double* ab = NULL;
  double* work = NULL;
  double* tmp = (double*)malloc(sizeof(double) * (size_t)ns);
  if (!tmp) return -3;
  if (method == 0) {
    ab = (double*)malloc(sizeof(double) * (size_t)(b + 1) * (size_t)ns);
    if (!ab) {
      free(tmp);
      return -3;
    }
  } else {
    work = (double*)malloc(sizeof(double) * 4 * (size_t)ns);
    if (!work) {
      free(tmp);
      return -3;
    }
  }
  int rc = 0;
  double t_acc = 0.0;
  for (int s = 1; s <= n_steps; ++s) {
    double t = s * tau;
    if (steps) {
      tau = steps[s - 1];
      t_acc += tau;
      t = t_acc;
    }
    const double* prev = s == 1 ? u0 : u + (size_t)(s - 2) * ns;
    double* cur = u + (size_t)(s - 1) * ns;
    const double* fs = f + (size_t)(s - 1) * ns;
    /* right-hand side M (u_{n-1} + tau_n f_n) */
    for (long i = 0; i < ns; ++i) tmp[i] = (prev ? prev[i] : 0.0) + tau * fs[i];
    oc_apply_M_slice(&g, mass, tmp, cur);
    if (method == 0) {
      oc_assemble_band(&g, k, t, tau, b, mass, ab);
      if (oc_band_cholesky(ns, b, ab) != 0) {
        rc = -1;
        break;
      }
      oc_band_solve(ns, b, ab, cur);
    } else {
      double* rhs = (double*)malloc(sizeof(double) * (size_t)ns);
      if (!rhs) {
        rc = -3;
        break;
      }
      memcpy(rhs, cur, sizeof(double) * (size_t)ns);
      /* initial guess: the previous step (or the rhs) */
      if (prev)
        memcpy(cur, prev, sizeof(double) * (size_t)ns);
      int it = oc_cg(&g, k, t, tau, mass, rhs, cur, cg_tol, 100000, work);
      free(rhs);
      if (it < 0) {
        rc = -2;
        break;
      }
    }
  }
  free(ab);
  free(work);
  free(tmp);
  return rc;
}

/* out = B u = (K (x) M) u + diag(tau_n A_n) u with u_0 := 0 (§2, eq. 2.3-2.4); steps and mass
 * as in oc_implicit_euler. */
void oc_apply_B(int dim, const int* n, int N, double T, const oc_coeff* k, const double* u,
                double* out, int nthreads, const double* steps, int mass) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  oc_grid g;
  oc_grid_init(&g, dim, n);
  long ns = g.ns;
  double tau = T / N;
  double t_acc = 0.0;
  double* diff = (double*)malloc(sizeof(double) * (size_t)ns);
  double* mdiff = (double*)malloc(sizeof(double) * (size_t)ns);
  if (!diff || !mdiff) {
    free(diff);
    free(mdiff);
    return;
  }
  for (int s = 1; s <= N; ++s) {
    const double* us = u + (size_t)(s - 1) * ns;
    double* os = out + (size_t)(s - 1) * ns;
    double t = s * tau;
    if (steps) {
      tau = steps[s - 1];
      t_acc += tau;
      t = t_acc;
    }
    oc_apply_A_slice(&g, k, t, us, os);
    for (long i = 0; i < ns; ++i) diff[i] = us[i] - (s > 1 ? us[i - ns] : 0.0);
    oc_apply_M_slice(&g, mass, diff, mdiff);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < ns; ++i) os[i] = mdiff[i] + tau * os[i];
  }
  free(diff);
  free(mdiff);
}

/* out = A(t) v on one slice. */
void oc_apply_A(int dim, const int* n, double t, const oc_coeff* k, const double* v, double* out,
                int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  oc_grid g;
  oc_grid_init(&g, dim, n);
  oc_apply_A_slice(&g, k, t, v, out);
}

int oc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
