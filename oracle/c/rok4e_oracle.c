/* C oracle of the ROK4E reaction step and the Simpler balanced split step.
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow-but-compiled restatement of the
 * method for long checks (1000 split steps) and for the timed CPU baseline.
 * It shares no code with the CUDA library and neither includes the other; it
 * is pinned against the numpy oracle (the Python modules of oracle/), whose
 * own pins tie it to the paper (tests/test_oracle_c.py).  Compiled by
 * oracle/c_oracle.py (gcc -O3 -fopenmp -ffp-contract=off) into
 * oracle/c/_lib/liboracle_rok4e.so.
 *
 * What it computes (arXiv:1712.00953):
 *  - the constant-pressure reactor right-hand side (rhs_body.h);
 *  - Jacobian-vector products: analytic to rounding by the complex step
 *    J v = Im f(u + i eps v) / eps, or the forward difference of Sec. 4.3
 *    with delta = sqrt(eps_mach) (1 + ||u||) / ||v||;
 *  - Arnoldi on K_M(J_n, f_n) (Sec. 4.1): modified Gram-Schmidt with one
 *    reorthogonalisation pass, breakdown when the orthogonalised vector keeps
 *    <= 1e-12 of ||J q_j||;
 *  - the four stages of the Rosenbrock form (Eq. s_stage_row, with the factor
 *    h on its A_n term) for A_n = Q H Q^T (Eq. jac_proj), solved on the
 *    Krylov coordinates, (I - h gamma H) kappa_i = Q^T f_i + h H sum_j
 *    gamma_ij kappa_j, plus the part of f_i orthogonal to the Krylov space;
 *    the coefficient table of Sec. 4.2 with the reading b = (b1, b2, 0, b4),
 *    bhat = (bhat1, bhat2, bhat3, 0);
 *  - the RMS error norm and the PI controller of Sec. 4.3 (err_n = 1 before
 *    the first step, errors floored at 1e-10, non-finite error: reject with
 *    factor 0.2), h clipped to t_end - t, done when t_end - t <= 1e-12 t_end;
 *  - Eq. simpler_balanced on the 1-D system: T(U_n) by second-order central
 *    differences with zero-gradient ends, the reaction sub-step over dt with
 *    the constant source T(U_n), one SSP-RK3 step of dU/dt = T(U) - T(U_n)
 *    over dt/2.
 * A recorded step sequence (+h accepted, -h rejected, 0 ends it; the GPU's
 * trace format) can replace the controller's decisions. */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>

#define ORC_R 8.314462618
#define ORC_PREF 101325.0
#define ORC_LN10 2.302585092994046
#define ORC_MAX_SP 256
#define ORC_MAX_RX 2048
#define ORC_MAX_M 8
#define ORC_MAX_RS 4 /* species entries per reaction */

typedef struct {
  int n, sp[ORC_MAX_RS], nu[ORC_MAX_RS]; /* entries: reactants < 0, products > 0 */
  int kind, rev, dnu;
  double lnA, b, EaR, lnA0, b0, Ea0R, ta, T3, T1, T2;
} orc_rxn;

typedef struct orc_mech {
  int ns, nr;
  double* W;    /* [ns] */
  double* nasa; /* [ns x 17]: Tlo, Tmid, Thi, 7 low, 7 high */
  double* eff;  /* [nr x ns] */
  orc_rxn* rx;
} orc_mech;

#define SCALAR double
#define FN(name) name##_r
#include "rhs_body.h"
#undef SCALAR
#undef FN
#define SCALAR double complex
#define FN(name) name##_c
#include "rhs_body.h"
#undef SCALAR
#undef FN

/* ROK4E coefficients (Sec. 4.2, table of ROK4E), zero-based stages */
static const double GAM = 0.572816062482135;
static const double GIJ[4][4] = {{0, 0, 0, 0},
                                 {-0.602765307997356, 0, 0, 0},
                                 {-1.389195789724843, 1.072950969011413, 0, 0},
                                 {0.992356412977094, -1.390032613873701, -0.440875890223325, 0}};
static const double AIJ[4][4] = {{0, 0, 0, 0},
                                 {0.432364435748567, 0, 0, 0},
                                 {-0.514211316876170, 1.382271144617360, 0, 0},
                                 {-0.514211316876170, 1.382271144617360, 0, 0}};
static const double BW[4] = {0.194335256262729, 0.483167813989227, 0.0, 0.322496929748044};
static const double BH[4] = {-0.217819895945721, 1.03130847478467, 0.186511421161047, 0.0};

/* ------------------------------------------------------------- mechanism */
orc_mech* orc_mech_new(int ns, int nr, const double* W, const double* nasa, const int* rxn_sp, const int* rxn_nu,
                       const double* arrh, const unsigned char* reversible, const int* kind, const double* eff,
                       const double* falloff) {
  if (ns < 1 || ns > ORC_MAX_SP - 1 || nr < 0 || nr > ORC_MAX_RX) return NULL;
  orc_mech* m = (orc_mech*)calloc(1, sizeof(orc_mech));
  m->ns = ns;
  m->nr = nr;
  m->W = (double*)malloc(sizeof(double) * ns);
  m->nasa = (double*)malloc(sizeof(double) * 17 * ns);
  m->eff = (double*)malloc(sizeof(double) * (size_t)(nr > 0 ? nr : 1) * ns);
  m->rx = (orc_rxn*)calloc(nr > 0 ? nr : 1, sizeof(orc_rxn));
  memcpy(m->W, W, sizeof(double) * ns);
  memcpy(m->nasa, nasa, sizeof(double) * 17 * ns);
  memcpy(m->eff, eff, sizeof(double) * (size_t)nr * ns);
  for (int j = 0; j < nr; ++j) {
    orc_rxn* r = m->rx + j;
    /* the reaction's entries as given (a species may appear on both sides) */
    int order_f = 0;
    r->n = 0;
    r->dnu = 0;
    for (int e = 0; e < 4; ++e) {
      const int s = rxn_sp[4 * j + e], nu = rxn_nu[4 * j + e];
      if (s < 0 || s >= ns || nu == 0) continue;
      if (nu < 0) order_f += -nu;
      r->sp[r->n] = s;
      r->nu[r->n] = nu;
      r->n++;
      r->dnu += nu;
    }
    r->kind = kind[j];
    r->rev = reversible[j] != 0;
    const double ln1e6 = log(1e-6);
    /* A in cm-mol-s to SI: concentration order (reactant order, +1 for a plain third body) minus 1 */
    r->lnA = log(arrh[3 * j]) + (order_f + (r->kind == 1 ? 1 : 0) - 1) * ln1e6;
    r->b = arrh[3 * j + 1];
    r->EaR = arrh[3 * j + 2] / ORC_R;
    if (r->kind == 2) {
      const double* fo = falloff + 7 * j;
      r->lnA0 = log(fo[0]) + order_f * ln1e6;
      r->b0 = fo[1];
      r->Ea0R = fo[2] / ORC_R;
      r->ta = fo[3];
      r->T3 = fo[4];
      r->T1 = fo[5];
      r->T2 = fo[6];
    }
  }
  return m;
}

void orc_mech_free(orc_mech* m) {
  if (!m) return;
  free(m->W);
  free(m->nasa);
  free(m->eff);
  free(m->rx);
  free(m);
}

/* ----------------------------------------------------------- J v products */
typedef struct {
  const orc_mech* m;
  const double* u;
  const double* src;
  double p;
  int jv_mode;
  double unorm;
  const double* fu; /* f(u) (with src) for the forward difference */
} orc_jv;

static double norm2(const double* v, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += v[i] * v[i];
  return sqrt(s);
}

static void apply_jv(const orc_jv* J, const double* v, double* out) {
  const int N = J->m->ns + 1;
  if (J->jv_mode == 0) {
    const double eps = 1e-30;
    double complex uc[ORC_MAX_SP], fc[ORC_MAX_SP];
    for (int e = 0; e < N; ++e) uc[e] = J->u[e] + I * (eps * v[e]);
    rhs_c(J->m, uc, NULL, J->p, fc);
    for (int e = 0; e < N; ++e) out[e] = cimag(fc[e]) / eps;
    return;
  }
  const double nv = norm2(v, N);
  if (nv == 0.0) {
    for (int e = 0; e < N; ++e) out[e] = 0.0;
    return;
  }
  const double d = sqrt(2.220446049250313e-16) * (1.0 + J->unorm) / nv;
  double ud[ORC_MAX_SP], fd[ORC_MAX_SP];
  for (int e = 0; e < N; ++e) ud[e] = J->u[e] + d * v[e];
  rhs_r(J->m, ud, J->src, J->p, fd);
  for (int e = 0; e < N; ++e) out[e] = (fd[e] - J->fu[e]) / d;
}

/* ---------------------------------------------------------------- Arnoldi */
/* Q: [ORC_MAX_M][N] rows, H: [ORC_MAX_M][ORC_MAX_M]; returns m */
static int arnoldi(const orc_jv* J, const double* fn, int M, double Q[][ORC_MAX_SP], double H[][ORC_MAX_M]) {
  const int N = J->m->ns + 1;
  if (M > N) M = N;
  for (int i = 0; i < ORC_MAX_M; ++i)
    for (int j = 0; j < ORC_MAX_M; ++j) H[i][j] = 0.0;
  const double beta = norm2(fn, N);
  if (M <= 0 || beta == 0.0 || !isfinite(beta)) return 0;
  for (int e = 0; e < N; ++e) Q[0][e] = fn[e] / beta;
  int m = M;
  double w[ORC_MAX_SP];
  for (int j = 0; j < M; ++j) {
    apply_jv(J, Q[j], w);
    const double w0 = norm2(w, N);
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i <= j; ++i) {
        double h = 0.0;
        for (int e = 0; e < N; ++e) h += Q[i][e] * w[e];
        H[i][j] += h;
        for (int e = 0; e < N; ++e) w[e] -= h * Q[i][e];
      }
    const double hn = norm2(w, N);
    if (j + 1 == M) break;
    if (hn <= 1e-12 * w0 || hn == 0.0) {
      m = j + 1;
      break;
    }
    H[j + 1][j] = hn;
    for (int e = 0; e < N; ++e) Q[j + 1][e] = w[e] / hn;
  }
  return m;
}

/* Gaussian elimination with partial pivoting of A (m x m, row stride ORC_MAX_M)
 * in place; solve with the factors. */
static void lu_factor(double A[][ORC_MAX_M], int m, int* piv) {
  for (int c = 0; c < m; ++c) {
    int pr = c;
    for (int r = c + 1; r < m; ++r)
      if (fabs(A[r][c]) > fabs(A[pr][c])) pr = r;
    piv[c] = pr;
    if (pr != c)
      for (int j = 0; j < m; ++j) {
        const double t = A[c][j];
        A[c][j] = A[pr][j];
        A[pr][j] = t;
      }
    for (int r = c + 1; r < m; ++r) {
      const double l = A[r][c] / A[c][c];
      A[r][c] = l;
      for (int j = c + 1; j < m; ++j) A[r][j] -= l * A[c][j];
    }
  }
}

static void lu_solve(double A[][ORC_MAX_M], int m, const int* piv, double* x) {
  for (int c = 0; c < m; ++c)
    if (piv[c] != c) {
      const double t = x[c];
      x[c] = x[piv[c]];
      x[piv[c]] = t;
    }
  for (int r = 1; r < m; ++r)
    for (int c = 0; c < r; ++c) x[r] -= A[r][c] * x[c];
  for (int r = m - 1; r >= 0; --r) {
    for (int c = r + 1; c < m; ++c) x[r] -= A[r][c] * x[c];
    x[r] /= A[r][r];
  }
}

/* -------------------------------------------------------- one attempt */
static int attempt(const orc_mech* mech, const double* src, double p, const double* u, const double* fn,
                   double Q[][ORC_MAX_SP], double H[][ORC_MAX_M], int m, double h, double* us, double* uh) {
  const int N = mech->ns + 1;
  double A[ORC_MAX_M][ORC_MAX_M];
  int piv[ORC_MAX_M];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) A[i][j] = (i == j ? 1.0 : 0.0) - h * GAM * H[i][j];
  lu_factor(A, m, piv);
  static const int same_arg[4] = {0, 0, 0, 1}; /* stage 4: alpha_4j = alpha_3j */
  double K[4][ORC_MAX_SP], kap[4][ORC_MAX_M], fi[ORC_MAX_SP], arg[ORC_MAX_SP];
  int nf = 0;
  for (int i = 0; i < 4; ++i) {
    if (i == 0) {
      memcpy(fi, fn, sizeof(double) * N);
    } else if (!same_arg[i]) {
      for (int e = 0; e < N; ++e) {
        double a = 0.0;
        for (int j = 0; j < i; ++j) a += AIJ[i][j] * K[j][e];
        arg[e] = u[e] + h * a;
      }
      rhs_r(mech, arg, src, p, fi);
      nf++;
    }
    double proj[ORC_MAX_M], z[ORC_MAX_M];
    for (int l = 0; l < m; ++l) {
      double s = 0.0;
      for (int e = 0; e < N; ++e) s += Q[l][e] * fi[e];
      proj[l] = s;
    }
    for (int l = 0; l < m; ++l) {
      double c = 0.0;  /* h (H sum_j gamma_ij kappa_j)_l */
      for (int r = 0; r < m; ++r) {
        double g = 0.0;
        for (int j = 0; j < i; ++j) g += GIJ[i][j] * kap[j][r];
        c += H[l][r] * g;
      }
      z[l] = proj[l] + h * c;
    }
    lu_solve(A, m, piv, z);
    for (int l = 0; l < m; ++l) kap[i][l] = z[l];
    for (int e = 0; e < N; ++e) {
      double qk = 0.0, qp = 0.0;
      for (int l = 0; l < m; ++l) {
        qk += Q[l][e] * kap[i][l];
        qp += Q[l][e] * proj[l];
      }
      K[i][e] = qk + (fi[e] - qp);
    }
  }
  for (int e = 0; e < N; ++e) {
    double sb = 0.0, sh = 0.0;
    for (int j = 0; j < 4; ++j) {
      sb += BW[j] * K[j][e];
      sh += BH[j] * K[j][e];
    }
    us[e] = u[e] + h * sb;
    uh[e] = u[e] + h * sh;
  }
  return nf;
}

/* ------------------------------------------------------ one cell over dt */
/* status: 0 ok, 1 attempt cap, 2 non-finite accepted state, 3 step underflow */
static void integrate_cell(const orc_mech* mech, double* u, const double* src, double p, double dt, double rtol,
                           double atol, int M, int jv_mode, double* h_io, const double* replay, int cap,
                           int32_t* stats, double* rec) {
  const int N = mech->ns + 1;
  double Q[ORC_MAX_M][ORC_MAX_SP], H[ORC_MAX_M][ORC_MAX_M];
  double fn[ORC_MAX_SP], us[ORC_MAX_SP], uh[ORC_MAX_SP];
  double h = (h_io && *h_io > 0.0) ? *h_io : dt;
  double t = 0.0, h_last = h, err_prev = 1.0;
  int n_acc = 0, n_rej = 0, n_f = 0, status = 0, n_att = 0;
  orc_jv J = {mech, u, src, p, jv_mode, 0.0, fn};
  rhs_r(mech, u, src, p, fn);
  n_f++;
  J.unorm = norm2(u, N);
  int m = arnoldi(&J, fn, M, Q, H);
  if (jv_mode) n_f += m;
  while (1) {
    if (dt - t <= 1e-12 * dt) break;
    if (n_att >= 100000) {
      status = 1;
      break;
    }
    int forced = -1;
    if (replay) {
      if (n_att >= cap || replay[n_att] == 0.0) break;
      h = fabs(replay[n_att]);
      forced = replay[n_att] > 0.0;
    } else {
      h = fmin(h, dt - t);
    }
    n_f += attempt(mech, src, p, u, fn, Q, H, m, h, us, uh);
    n_att++;
    double s = 0.0;
    int bad = 0;
    for (int e = 0; e < N; ++e) {
      const double d = (uh[e] - us[e]) / (atol + rtol * fabs(us[e]));
      s += d * d;
      bad |= !isfinite(us[e]);
    }
    const double err = sqrt(s / N);
    double fac = 0.2;
    if (isfinite(err)) {
      const double ef = err > 1e-10 ? err : 1e-10;
      fac = 0.8 * pow(err_prev, 0.1) / pow(ef, 0.175);
      fac = fac > 5.0 ? 5.0 : (fac < 0.2 ? 0.2 : fac);
    }
    const double h_new = h * fac;
    const int accept = forced >= 0 ? forced : (isfinite(err) && err <= 1.0);
    if (rec && n_att - 1 < cap) rec[n_att - 1] = accept ? h : -h;
    if (accept) {
      if (bad) {
        status = 2;
        break;
      }
      memcpy(u, us, sizeof(double) * N);
      t += h;
      err_prev = err > 1e-10 ? err : 1e-10;
      n_acc++;
      h_last = h_new;
      h = h_new;
      if (!(dt - t <= 1e-12 * dt)) {
        rhs_r(mech, u, src, p, fn);
        n_f++;
        J.unorm = norm2(u, N);
        m = arnoldi(&J, fn, M, Q, H);
        if (jv_mode) n_f += m;
      }
    } else {
      n_rej++;
      h = h_new;
      if (!replay && h < 1e-12 * dt) {
        status = 3;
        break;
      }
    }
  }
  if (h_io) *h_io = h_last;
  if (stats) {
    stats[0] = n_acc;
    stats[1] = n_rej;
    stats[2] = n_f;
    stats[3] = status;
  }
}

/* --------------------------------------------------------------- C ABI */
int orc_rhs(const orc_mech* m, const double* u, const double* src, double p, double* f) {
  if (!m || !u || !f) return -1;
  rhs_r(m, u, src, p, f);
  return 0;
}

int orc_jvp(const orc_mech* m, const double* u, const double* v, double p, int jv_mode, double* out) {
  if (!m || !u || !v || !out) return -1;
  double fu[ORC_MAX_SP];
  rhs_r(m, u, NULL, p, fu);
  orc_jv J = {m, u, NULL, p, jv_mode, norm2(u, m->ns + 1), fu};
  apply_jv(&J, v, out);
  return 0;
}

/* Every row of U [ncell x (ns+1)] over dt in place (OpenMP over cells).
 * src [ncell x N] or NULL; h [ncell]: in h0 (<= 0: dt), out the next step;
 * replay [ncell x cap] or NULL; record [ncell x cap] or NULL (the attempts
 * taken, +h accepted / -h rejected, first cap of them; zero the buffer first);
 * stats [ncell x 4] or NULL. */
int orc_integrate(const orc_mech* m, double* U, const double* src, double* h, int64_t ncell, double p, double dt,
                  double rtol, double atol, int M, int jv_mode, const double* replay, double* record, int cap,
                  int32_t* stats, int nthreads) {
  if (!m || !U || ncell < 0 || M < 0 || M > ORC_MAX_M || !(dt > 0.0)) return -1;
  const int N = m->ns + 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
  for (int64_t c = 0; c < ncell; ++c)
    integrate_cell(m, U + c * N, src ? src + c * N : NULL, p, dt, rtol, atol, M, jv_mode, h ? h + c : NULL,
                   replay ? replay + c * cap : NULL, cap, stats ? stats + 4 * c : NULL,
                   record ? record + c * cap : NULL);
  return 0;
}

/* T(U): D times the second difference with zero-gradient ends */
static void diffusion(const double* U, double* TU, int64_t npts, int nv, double D, double dx) {
  const double idx2 = 1.0 / (dx * dx);
  for (int64_t i = 0; i < npts; ++i) {
    const int64_t im = i > 0 ? i - 1 : 0, ip = i + 1 < npts ? i + 1 : npts - 1;
    for (int v = 0; v < nv; ++v) TU[i * nv + v] = D * ((U[im * nv + v] - 2.0 * U[i * nv + v] + U[ip * nv + v]) * idx2);
  }
}

/* nsteps Simpler balanced split steps (Eq. simpler_balanced) of the 1-D
 * system U [npts x N] in place, h [npts] carried; replay and record
 * [nsteps x npts x cap] or NULL; stats [nsteps x npts x 4] or NULL. */
int orc_simpler_steps(const orc_mech* m, double* U, double* h, int64_t npts, double p, double dt, double D,
                      double dx, double rtol, double atol, int M, int nsteps, const double* replay, double* record,
                      int cap, int32_t* stats, int nthreads) {
  if (!m || !U || !h || npts < 1 || nsteps < 0) return -1;
  const int nv = m->ns + 1;
  const size_t n = (size_t)npts * nv;
  double* Tn = (double*)malloc(sizeof(double) * n);
  double* U1 = (double*)malloc(sizeof(double) * n);
  double* V = (double*)malloc(sizeof(double) * n);
  double* G = (double*)malloc(sizeof(double) * n);
  for (int s = 0; s < nsteps; ++s) {
    diffusion(U, Tn, npts, nv, D, dx);
    orc_integrate(m, U, Tn, h, npts, p, dt, rtol, atol, M, 0, replay ? replay + (size_t)s * npts * cap : NULL,
                  record ? record + (size_t)s * npts * cap : NULL, cap,
                  stats ? stats + (size_t)s * npts * 4 : NULL, nthreads);
    /* one SSP-RK3 step of dU/dt = T(U) - T(U_n) over dt/2 (Shu-Osher form) */
    const double k = 0.5 * dt;
    memcpy(U1, U, sizeof(double) * n);
    diffusion(U1, G, npts, nv, D, dx);
    for (size_t i = 0; i < n; ++i) V[i] = U1[i] + k * (G[i] - Tn[i]);
    diffusion(V, G, npts, nv, D, dx);
    for (size_t i = 0; i < n; ++i) V[i] = 0.75 * U1[i] + 0.25 * (V[i] + k * (G[i] - Tn[i]));
    diffusion(V, G, npts, nv, D, dx);
    for (size_t i = 0; i < n; ++i) U[i] = U1[i] / 3.0 + 2.0 / 3.0 * (V[i] + k * (G[i] - Tn[i]));
  }
  free(Tn);
  free(U1);
  free(V);
  free(G);
  return 0;
}
