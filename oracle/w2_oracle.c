/*
 * w2_oracle.c -- plain, slow FP64 CPU oracle for one time step of the Wigner
 * equation of the two-body reduced density matrix (2-RDM) in the spatially
 * periodic 1-D case, following arXiv:2511.11354:
 *
 *   - periodic pseudo-difference operators (Sec. 3.1, Eq. Hartree_FSM for the
 *     one-body Hartree-exchange-correlation part, Eq. two_body_FSM for the
 *     two-body collision part), with the Fourier modes of the potential taken
 *     from a 2 N_p-point DFT at spacing L / (2 N_p) (Sec. 3.1.2);
 *   - the periodic cubic B-spline (Sec. 4.1: the B_nu pieces, the three-term
 *     relation and the (N_x+3) x (N_x+3) matrix A_per);
 *   - the Lawson predictor-corrector (Sec. 4.1, first display);
 *   - densities, mass and the 1-RDM purity (Sec. 2 definitions).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or table with the CUDA
 * path.
 *
 * Readings of the paper fixed here (each also listed in the design notes):
 *   R1 sign: Theta_U f = (i/hbar) sum_m U^_m e^{2 pi i m x/L}
 *            [f(p + m dp) - f(p - m dp)], U = sum_m U^_m e^{2 pi i m x / L};
 *            this reproduces both closed forms of Sec. 5.1 exactly.
 *   R2 momentum lattice p_n = (n - N_k/2) dp, dp = pi hbar / L.
 *   R4 potentials are sampled pointwise at x + l h', h' = L/(2 N_k), so N_x
 *      need not equal 2 N_p; the local 2 N_k-point DFT replaces the global
 *      Fourier modes (identical when N_x divides 2 N_k).
 *   R5 non-periodic potentials are folded: fold(x) in [-L/2, L/2).
 *   R6 Hartree on the torus: V_H(y) = gamma dx sum_q W(fold(y - x_q)) n(x_q),
 *      weighted by c_H.
 *   R7 XC: c_xc * phi(n), phi(n) = n (xc_kind 1) or the Hedin-Lundqvist form
 *      in atomic units (xc_kind 2), evaluated at max(n, 0); n between grid
 *      points by trigonometric interpolation.
 *   R8 Lawson: the HXC potential of each Theta is built from that Theta's
 *      input (f^n for the predictor, f~ for the corrector).
 *   R12 entropy: linear entropy 1 - Tr rho1^2, Tr rho1^2 = 2 pi hbar sum f1^2 dx dp.
 *   R15 neutralised Poisson Hartree (plasma workloads): the N_x-point Fourier
 *      solution of -V'' = n - mean(n), Nyquist mode as its cosine half.
 *
 * Layout of every phase-space array: f[i1][i2][n1][n2], n2 fastest, double.
 * "parity pinned": every function here is checked by tests/test_oracle_*.py
 * against closed forms, invariants, library routines or brute force.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

typedef double (*orc_fn)(double x, void *user);

typedef struct orc_problem {
  int nx, nk, M;          /* M = 2 nk: padded momentum length, Sec. 3.1 */
  double L, dt, hbar, mass, gamma, c_h, c_xc;
  int xc_kind;
  double dx, dp, hp;      /* dx = L/nx, dp = pi hbar / L, h' = L / M */
  double *vext_fine;      /* [nx][M]: V_ext(fold(x_i + l h'))            */
  double *vext_grid;      /* [nx]   : V_ext(x_i)                          */
  double *w_shift;        /* [nx][M]: W(fold(d dx + l h')), d = 0..nx-1   */
  int hartree_kind;       /* 0: gamma dx sum_q W n (R6); 1: neutralised periodic Poisson (R15) */
  double *h_shift;        /* [nx][M]: G(d dx + l h'), the Poisson kernel (hartree_kind 1) */
  double *ainv;           /* [(nx+3)^2]: inverse of A_per                 */
} orc_problem;

static double orc_fold(double x, double L) { return x - L * floor((x + 0.5 * L) / L); }

static size_t idx4(const orc_problem *P, int i1, int i2, int n1, int n2) {
  return (((size_t)i1 * P->nx + i2) * P->nk + n1) * P->nk + n2;
}

/* ------------------------------------------------------------------------ */
/* Periodic cubic spline, Sec. 4.1                                           */
/* ------------------------------------------------------------------------ */

/* A_per of Sec. 4.1, size (N+3) x (N+3), acting on (eta_{-1}, ..., eta_{N+1}).
 * Row 0: (eta_{-1} - eta_{N-1}) / 6 = 0;  rows 1..N+1: (eta_{v-1} + 4 eta_v +
 * eta_{v+1}) / 6 = f(r_v), v = 0..N;  last row: (eta_{N+1} - eta_1) / 6 = 0. */
static void build_aper(int N, double *A) {
  int n = N + 3;
  memset(A, 0, sizeof(double) * n * n);
  A[0 * n + 0] = 1.0 / 6.0;                 /* eta_{-1}            */
  A[0 * n + (N - 1 + 1)] = -1.0 / 6.0;      /* eta_{N-1}: column N */
  for (int v = 0; v <= N; ++v) {
    int row = v + 1;
    A[row * n + (v - 1 + 1)] += 1.0 / 6.0;
    A[row * n + (v + 1)] += 4.0 / 6.0;
    A[row * n + (v + 1 + 1)] += 1.0 / 6.0;
  }
  A[(n - 1) * n + (1 + 1)] = -1.0 / 6.0;    /* eta_1               */
  A[(n - 1) * n + (n - 1)] = 1.0 / 6.0;     /* eta_{N+1}           */
}

/* Gauss-Jordan inversion with partial pivoting; returns 0 on success. */
static int invert(int n, double *A, double *Ainv) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return -1;
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        double t = A[c * n + j]; A[c * n + j] = A[piv * n + j]; A[piv * n + j] = t;
        t = Ainv[c * n + j]; Ainv[c * n + j] = Ainv[piv * n + j]; Ainv[piv * n + j] = t;
      }
    double d = A[c * n + c];
    for (int j = 0; j < n; ++j) { A[c * n + j] /= d; Ainv[c * n + j] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double m = A[r * n + c];
      if (m == 0.0) continue;
      for (int j = 0; j < n; ++j) { A[r * n + j] -= m * A[c * n + j]; Ainv[r * n + j] -= m * Ainv[c * n + j]; }
    }
  }
  return 0;
}

/* Cubic B-spline B_nu(r) exactly as the four pieces of Sec. 4.1, with
 * r_nu = r0 + nu h. */
static double bspline(int nu, double r, double r0, double h) {
  double rm2 = r0 + (nu - 2) * h, rm1 = r0 + (nu - 1) * h, rn = r0 + nu * h;
  double rp1 = r0 + (nu + 1) * h, rp2 = r0 + (nu + 2) * h;
  double h2 = h * h, h3 = h2 * h;
  if (r >= rm2 && r <= rm1) { double t = r - rm2; return t * t * t / (6 * h3); }
  if (r > rm1 && r <= rn) { double t = r - rm1; return -t * t * t / (2 * h3) + t * t / (2 * h2) + t / (2 * h) + 1.0 / 6.0; }
  if (r > rn && r <= rp1) { double t = rp1 - r; return -t * t * t / (2 * h3) + t * t / (2 * h2) + t / (2 * h) + 1.0 / 6.0; }
  if (r > rp1 && r <= rp2) { double t = rp2 - r; return t * t * t / (6 * h3); }
  return 0.0;
}

/* Spline value at the foot of the characteristic: given the samples f(r_v),
 * v = 0..N-1 of one periodic line (r_v = -L/2 + v h), return the periodic
 * cubic spline interpolant evaluated at r_i - shift for every i. */
static void spline_shift_line(const orc_problem *P, int N, double h, const double *fin,
                              double shift, double *fout, double *rhs, double *eta) {
  int n = N + 3;
  double r0 = -0.5 * P->L;
  rhs[0] = 0.0;
  for (int v = 0; v < N; ++v) rhs[v + 1] = fin[v];
  rhs[N + 1] = fin[0];  /* f(r_N) = f(r_0) */
  rhs[N + 2] = 0.0;
  for (int a = 0; a < n; ++a) {
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += P->ainv[a * n + b] * rhs[b];
    eta[a] = s;  /* eta[a] = eta_{a-1} */
  }
  for (int i = 0; i < N; ++i) {
    double r = r0 + i * h - shift;
    r = r0 + (r - r0) - P->L * floor((r - r0) / P->L); /* into [r0, r0+L) */
    int k = (int)floor((r - r0) / h);
    if (k < 0) k = 0;
    if (k > N - 1) k = N - 1;
    double v = 0.0;
    for (int nu = k - 1; nu <= k + 2; ++nu) v += eta[nu + 1] * bspline(nu, r, r0, h);
    fout[i] = v;
  }
}

/* ------------------------------------------------------------------------ */
/* Set-up                                                                   */
/* ------------------------------------------------------------------------ */

void orc_destroy(orc_problem *P) {
  if (!P) return;
  free(P->vext_fine); free(P->vext_grid); free(P->w_shift); free(P->ainv); free(P->h_shift);
  free(P);
}

/* Potentials are sampled once here (single-threaded callbacks). */
orc_problem *orc_create(int nx, int nk, double L, double dt, double hbar, double mass,
                        double gamma, double c_h, double c_xc, int xc_kind,
                        orc_fn vext, void *ue, orc_fn vee, void *ui) {
  if (nx < 4 || nk < 2 || (nk & 1) || !(L > 0) || !(hbar > 0) || !(mass > 0)) return NULL;
  orc_problem *P = (orc_problem *)calloc(1, sizeof(orc_problem));
  P->nx = nx; P->nk = nk; P->M = 2 * nk;
  P->L = L; P->dt = dt; P->hbar = hbar; P->mass = mass;
  P->gamma = gamma; P->c_h = c_h; P->c_xc = c_xc; P->xc_kind = xc_kind;
  P->dx = L / nx; P->dp = ORC_PI * hbar / L; P->hp = L / P->M;
  int M = P->M;
  P->vext_fine = (double *)malloc(sizeof(double) * nx * M);
  P->vext_grid = (double *)malloc(sizeof(double) * nx);
  P->w_shift = (double *)malloc(sizeof(double) * nx * M);
  for (int i = 0; i < nx; ++i) {
    double xi = -0.5 * L + i * P->dx;
    P->vext_grid[i] = vext ? vext(orc_fold(xi, L), ue) : 0.0;
    for (int l = 0; l < M; ++l) {
      P->vext_fine[i * M + l] = vext ? vext(orc_fold(xi + l * P->hp, L), ue) : 0.0;
      P->w_shift[i * M + l] = vee ? vee(orc_fold(i * P->dx + l * P->hp, L), ui) : 0.0;
    }
  }
  int n = nx + 3;
  double *A = (double *)malloc(sizeof(double) * n * n);
  P->ainv = (double *)malloc(sizeof(double) * n * n);
  build_aper(nx, A);
  int rc = invert(n, A, P->ainv);
  free(A);
  if (rc) { orc_destroy(P); return NULL; }
  return P;
}

int orc_nx(const orc_problem *P) { return P->nx; }

/* ------------------------------------------------------------------------ */
/* Densities and potentials                                                 */
/* ------------------------------------------------------------------------ */

/* n_1(x1) = sum_{x2,p1,p2} f dx dp^2 and n_2(x2) likewise (Sec. 2, the
 * one-body densities entering the HXC potentials). */
void orc_marginals(const orc_problem *P, const double *f, double *n1, double *n2) {
  int nx = P->nx, nk = P->nk;
  double w = P->dx * P->dp * P->dp;
  for (int i = 0; i < nx; ++i) { n1[i] = 0.0; n2[i] = 0.0; }
  for (int i1 = 0; i1 < nx; ++i1)
    for (int i2 = 0; i2 < nx; ++i2) {
      double s = 0.0;
      for (int a = 0; a < nk; ++a)
        for (int b = 0; b < nk; ++b) s += f[idx4(P, i1, i2, a, b)];
      n1[i1] += s * w;
      n2[i2] += s * w;
    }
}

/* Trigonometric interpolant of the grid density n at y (Nyquist mode halved). */
/* Fourier coefficients c_m = (1/N) sum_q n_q e^{-2 pi i m q / N}, m = -N/2..N/2
 * (index m + N/2), of the grid samples n_q = n(x_q) */
static void trig_coeffs(const orc_problem *P, const double *n, double complex *c) {
  int N = P->nx;
  for (int m = -N / 2; m <= N / 2; ++m) {
    double complex s = 0.0;
    for (int q = 0; q < N; ++q) s += n[q] * cexp(-2.0 * I * ORC_PI * m * q / N);
    c[m + N / 2] = s / N;
  }
}

/* The trigonometric interpolant of the samples at y (Nyquist terms halved). */
static double trig_eval(const orc_problem *P, const double complex *c, double y) {
  int N = P->nx;
  double x0 = -0.5 * P->L, val = 0.0;
  for (int m = -N / 2; m <= N / 2; ++m) {
    double wgt = (N % 2 == 0 && (m == N / 2 || m == -N / 2)) ? 0.5 : 1.0;
    val += wgt * creal(c[m + N / 2] * cexp(2.0 * I * ORC_PI * m * (y - x0) / P->L));
  }
  return val;
}

static double phi_xc(int kind, double n) {
  if (kind == 1) return n;
  /* Hedin-Lundqvist (Sec. 2.2) in atomic units, defined for n >= 0 */
  if (kind == 2) { double c = cbrt(n > 0.0 ? n : 0.0); return 0.985 * c + 0.985 * 0.034 * log(1.0 + 18.37 * c); }
  return 0.0;
}

/* U(x_i + l h') for i in [0,nx), l in [0, M): the one-body potential of a
 * particle whose density is n:  V_ext + c_H V_H[n] + c_xc phi(n)  (Sec. 2.3
 * V_HXC; readings R6, R7).  out is [nx][M]. */
void orc_potential_fine(const orc_problem *P, const double *n, double *out) {
  int nx = P->nx, M = P->M;
  double complex *tc = NULL;
  if (P->c_xc != 0.0 && P->xc_kind && n) {
    tc = (double complex *)malloc(sizeof(double complex) * (nx + 1));
    trig_coeffs(P, n, tc);
  }
  for (int i = 0; i < nx; ++i)
    for (int l = 0; l < M; ++l) {
      double u = P->vext_fine[i * M + l];
      if (P->c_h != 0.0 && n && P->hartree_kind == 1) {
        /* neutralised Poisson (R15): V_H(y) = sum_q G(y - x_q) n(x_q) */
        double vh = 0.0;
        for (int q = 0; q < nx; ++q) {
          int d = ((i - q) % nx + nx) % nx;
          vh += P->h_shift[d * M + l] * n[q];
        }
        u += P->c_h * vh;
      } else if (P->c_h != 0.0 && n) {
        /* V_H(y) = gamma dx sum_q W(fold(y - x_q)) n(x_q), y = x_i + l h';
         * y - x_q = (i - q) dx + l h' */
        double vh = 0.0;
        for (int q = 0; q < nx; ++q) {
          int d = ((i - q) % nx + nx) % nx;
          vh += P->w_shift[d * M + l] * n[q];
        }
        u += P->c_h * P->gamma * P->dx * vh;
      }
      if (P->c_xc != 0.0 && P->xc_kind && n) {
        double y = -0.5 * P->L + i * P->dx + l * P->hp;
        u += P->c_xc * phi_xc(P->xc_kind, trig_eval(P, tc, y));
      }
      out[i * M + l] = u;
    }
  free(tc);
}

/* Fourier modes of a periodic function from its M samples u(y + l h'),
 * l = 0..M-1 (the 2 N_p-point DFT of Sec. 3.1.2, spacing L/(2 N_p)):
 *   c_m(y) = (1/M) sum_l u(y + l h') e^{-2 pi i m l / M}  ~  U^_m e^{2 pi i m y/L}.
 * Returns c_m for m = -(nk-1)..(nk-1) at index m + nk - 1. */
static void local_modes(const orc_problem *P, const double *u, double complex *c) {
  int M = P->M, nk = P->nk;
  for (int m = -(nk - 1); m <= nk - 1; ++m) {
    double complex s = 0.0;
    for (int l = 0; l < M; ++l) s += u[l] * cexp(-2.0 * I * ORC_PI * (double)m * l / M);
    c[m + nk - 1] = s / M;
  }
}

/* ------------------------------------------------------------------------ */
/* Pseudo-difference operator Theta, Sec. 3.1                               */
/* ------------------------------------------------------------------------ */

/* Theta f with explicitly given one-body potentials U1 (for particle 1, as a
 * function of x1) and U2 (particle 2, of x2), both [nx][M] on the fine points,
 * and the pair potential gamma W(fold(r)) from the set-up tables.
 * terms: bit 0 = one-body particle 1, bit 1 = one-body particle 2,
 *        bit 2 = two-body.  f outside the momentum window is zero. */
void orc_theta_with(const orc_problem *P, const double *f, const double *U1, const double *U2,
                    int terms, double *out) {
  int nx = P->nx, nk = P->nk, M = P->M;
  double hb = P->hbar;
  double complex *c1 = (double complex *)malloc(sizeof(double complex) * nx * (2 * nk - 1));
  double complex *c2 = (double complex *)malloc(sizeof(double complex) * nx * (2 * nk - 1));
  double complex *c12 = (double complex *)malloc(sizeof(double complex) * nx * (2 * nk - 1));
  double *u12 = (double *)malloc(sizeof(double) * M);
  for (int i = 0; i < nx; ++i) {
    local_modes(P, U1 + (size_t)i * M, c1 + (size_t)i * (2 * nk - 1));
    local_modes(P, U2 + (size_t)i * M, c2 + (size_t)i * (2 * nk - 1));
    for (int l = 0; l < M; ++l) u12[l] = P->gamma * P->w_shift[i * M + l];  /* r = i dx */
    local_modes(P, u12, c12 + (size_t)i * (2 * nk - 1));
  }
  free(u12);
#pragma omp parallel for collapse(2) schedule(static)
  for (int i1 = 0; i1 < nx; ++i1)
    for (int i2 = 0; i2 < nx; ++i2) {
      const double complex *a1 = c1 + (size_t)i1 * (2 * nk - 1) + (nk - 1);
      const double complex *a2 = c2 + (size_t)i2 * (2 * nk - 1) + (nk - 1);
      int d = ((i1 - i2) % nx + nx) % nx;   /* r = x1 - x2 = d dx (mod L) */
      const double complex *a12 = c12 + (size_t)d * (2 * nk - 1) + (nk - 1);
      const double *F = f + idx4(P, i1, i2, 0, 0);
#define FV(a, b) (((a) >= 0 && (a) < nk && (b) >= 0 && (b) < nk) ? F[(size_t)(a) * nk + (b)] : 0.0)
      for (int n1 = 0; n1 < nk; ++n1)
        for (int n2 = 0; n2 < nk; ++n2) {
          double complex s = 0.0;
          for (int m = -(nk - 1); m <= nk - 1; ++m) {
            if (terms & 1) s += a1[m] * (FV(n1 + m, n2) - FV(n1 - m, n2));
            if (terms & 2) s += a2[m] * (FV(n1, n2 + m) - FV(n1, n2 - m));
            if (terms & 4) s += a12[m] * (FV(n1 + m, n2 - m) - FV(n1 - m, n2 + m));
          }
          out[idx4(P, i1, i2, n1, n2)] = creal((I / hb) * s);
        }
#undef FV
    }
  free(c1); free(c2); free(c12);
}

/* orc_theta_with restricted to the spatial points xs[0..nxs) (X = i1 nx + i2):
 * out[q][n1][n2] = (Theta f)(xs[q], n1, n2).  Same arithmetic; for checks of
 * grids too large to sweep whole. */
void orc_theta_with_sample(const orc_problem *P, const double *f, const double *U1, const double *U2, int terms,
                           const int *xs, int nxs, double *out) {
  int nx = P->nx, nk = P->nk, M = P->M;
  double hb = P->hbar;
  size_t W = 2 * nk - 1;
  double complex *c1 = (double complex *)malloc(sizeof(double complex) * nx * W);
  double complex *c2 = (double complex *)malloc(sizeof(double complex) * nx * W);
  double complex *c12 = (double complex *)malloc(sizeof(double complex) * nx * W);
  double *u12 = (double *)malloc(sizeof(double) * M);
  for (int i = 0; i < nx; ++i) {
    local_modes(P, U1 + (size_t)i * M, c1 + (size_t)i * W);
    local_modes(P, U2 + (size_t)i * M, c2 + (size_t)i * W);
    for (int l = 0; l < M; ++l) u12[l] = P->gamma * P->w_shift[i * M + l];
    local_modes(P, u12, c12 + (size_t)i * W);
  }
  free(u12);
#pragma omp parallel for schedule(static)
  for (int q = 0; q < nxs; ++q) {
    int i1 = xs[q] / nx, i2 = xs[q] % nx;
    const double complex *a1 = c1 + (size_t)i1 * W + (nk - 1);
    const double complex *a2 = c2 + (size_t)i2 * W + (nk - 1);
    int d = ((i1 - i2) % nx + nx) % nx;
    const double complex *a12 = c12 + (size_t)d * W + (nk - 1);
    const double *F = f + idx4(P, i1, i2, 0, 0);
#define FV(a, b) (((a) >= 0 && (a) < nk && (b) >= 0 && (b) < nk) ? F[(size_t)(a) * nk + (b)] : 0.0)
    for (int n1 = 0; n1 < nk; ++n1)
      for (int n2 = 0; n2 < nk; ++n2) {
        double complex s = 0.0;
        for (int m = -(nk - 1); m <= nk - 1; ++m) {
          if (terms & 1) s += a1[m] * (FV(n1 + m, n2) - FV(n1 - m, n2));
          if (terms & 2) s += a2[m] * (FV(n1, n2 + m) - FV(n1, n2 - m));
          if (terms & 4) s += a12[m] * (FV(n1 + m, n2 - m) - FV(n1 - m, n2 + m));
        }
        out[((size_t)q * nk + n1) * nk + n2] = creal((I / hb) * s);
      }
#undef FV
  }
  free(c1); free(c2); free(c12);
}

/* Full Theta_V f of Eq. two_body_truncated_Wigner: HXC for both particles
 * (built from the densities of f itself) plus the two-body term. */
void orc_theta(const orc_problem *P, const double *f, double *out) {
  int nx = P->nx, M = P->M;
  double *n1 = (double *)malloc(sizeof(double) * nx), *n2 = (double *)malloc(sizeof(double) * nx);
  double *U1 = (double *)malloc(sizeof(double) * nx * M), *U2 = (double *)malloc(sizeof(double) * nx * M);
  orc_marginals(P, f, n1, n2);
  orc_potential_fine(P, n1, U1);
  orc_potential_fine(P, n2, U2);
  /* a two-body term with gamma = 0 is identically zero: leave it out */
  orc_theta_with(P, f, U1, U2, P->gamma != 0.0 ? 7 : 3, out);
  free(n1); free(n2); free(U1); free(U2);
}

/* ------------------------------------------------------------------------ */
/* Characteristic shift f(X - tau P / m, P), Sec. 4.1                        */
/* ------------------------------------------------------------------------ */

/* One periodic line: samples fin[0..N) at x_i, output at x_i - shift. */
void orc_shift_line(const orc_problem *P, const double *fin, double shift, double *fout) {
  int N = P->nx;
  double *rhs = (double *)malloc(sizeof(double) * (N + 3)), *eta = (double *)malloc(sizeof(double) * (N + 3));
  spline_shift_line(P, N, P->dx, fin, shift, fout, rhs, eta);
  free(rhs); free(eta);
}

/* Tensor-product spline: along x1 by tau p_{n1}/m, then along x2 by
 * tau p_{n2}/m (the two 1-D operators act on different axes). */
void orc_advect(const orc_problem *P, const double *f, double tau, double *out) {
  int nx = P->nx, nk = P->nk;
#pragma omp parallel
  {
    double *line = (double *)malloc(sizeof(double) * nx), *res = (double *)malloc(sizeof(double) * nx);
    double *rhs = (double *)malloc(sizeof(double) * (nx + 3)), *eta = (double *)malloc(sizeof(double) * (nx + 3));
    double *plane = (double *)malloc(sizeof(double) * nx * nx);
#pragma omp for collapse(2) schedule(static)
    for (int n1 = 0; n1 < nk; ++n1)
      for (int n2 = 0; n2 < nk; ++n2) {
        double s1 = tau * ((n1 - nk / 2) * P->dp) / P->mass;
        double s2 = tau * ((n2 - nk / 2) * P->dp) / P->mass;
        for (int i1 = 0; i1 < nx; ++i1)
          for (int i2 = 0; i2 < nx; ++i2) plane[i1 * nx + i2] = f[idx4(P, i1, i2, n1, n2)];
        for (int i2 = 0; i2 < nx; ++i2) {           /* x1 lines */
          for (int i1 = 0; i1 < nx; ++i1) line[i1] = plane[i1 * nx + i2];
          spline_shift_line(P, nx, P->dx, line, s1, res, rhs, eta);
          for (int i1 = 0; i1 < nx; ++i1) plane[i1 * nx + i2] = res[i1];
        }
        for (int i1 = 0; i1 < nx; ++i1) {           /* x2 lines */
          spline_shift_line(P, nx, P->dx, plane + i1 * nx, s2, res, rhs, eta);
          for (int i2 = 0; i2 < nx; ++i2) out[idx4(P, i1, i2, n1, n2)] = res[i2];
        }
      }
    free(line); free(res); free(rhs); free(eta); free(plane);
  }
}

/* orc_advect restricted to the momentum planes planes[0..np) (= n1 nk + n2):
 * out[q][i1][i2] = (A_tau f)(i1, i2, planes[q]). */
void orc_advect_sample(const orc_problem *P, const double *f, double tau, const int *planes, int np, double *out) {
  int nx = P->nx, nk = P->nk;
#pragma omp parallel
  {
    double *line = (double *)malloc(sizeof(double) * nx), *res = (double *)malloc(sizeof(double) * nx);
    double *rhs = (double *)malloc(sizeof(double) * (nx + 3)), *eta = (double *)malloc(sizeof(double) * (nx + 3));
    double *plane = (double *)malloc(sizeof(double) * nx * nx);
#pragma omp for schedule(static)
    for (int q = 0; q < np; ++q) {
      int n1 = planes[q] / nk, n2 = planes[q] % nk;
      double s1 = tau * ((n1 - nk / 2) * P->dp) / P->mass;
      double s2 = tau * ((n2 - nk / 2) * P->dp) / P->mass;
      for (int i1 = 0; i1 < nx; ++i1)
        for (int i2 = 0; i2 < nx; ++i2) plane[i1 * nx + i2] = f[idx4(P, i1, i2, n1, n2)];
      for (int i2 = 0; i2 < nx; ++i2) {
        for (int i1 = 0; i1 < nx; ++i1) line[i1] = plane[i1 * nx + i2];
        spline_shift_line(P, nx, P->dx, line, s1, res, rhs, eta);
        for (int i1 = 0; i1 < nx; ++i1) plane[i1 * nx + i2] = res[i1];
      }
      for (int i1 = 0; i1 < nx; ++i1) {
        spline_shift_line(P, nx, P->dx, plane + i1 * nx, s2, res, rhs, eta);
        for (int i2 = 0; i2 < nx; ++i2) out[((size_t)q * nx + i1) * nx + i2] = res[i2];
      }
    }
    free(line); free(res); free(rhs); free(eta); free(plane);
  }
}

/* ------------------------------------------------------------------------ */
/* Lawson predictor-corrector, Sec. 4.1                                      */
/* ------------------------------------------------------------------------ */

/* f <- f after nsteps steps of
 *   f~      = A_tau f^n + tau A_tau Theta[f^n]
 *   f^{n+1} = A_tau f^n + tau/2 Theta[f~] + tau/2 A_tau Theta[f^n]
 * where A_tau g = g(X - tau P/m, P). */
int orc_step(const orc_problem *P, double *f, int nsteps) {
  size_t n = (size_t)P->nx * P->nx * P->nk * P->nk;
  double tau = P->dt;
  double *g = (double *)malloc(sizeof(double) * n), *a = (double *)malloc(sizeof(double) * n);
  double *b = (double *)malloc(sizeof(double) * n), *c = (double *)malloc(sizeof(double) * n);
  if (!g || !a || !b || !c) { free(g); free(a); free(b); free(c); return -1; }
  for (int s = 0; s < nsteps; ++s) {
    orc_theta(P, f, g);                 /* Theta[f^n]           */
    orc_advect(P, f, tau, a);           /* A_tau f^n            */
    orc_advect(P, g, tau, b);           /* A_tau Theta[f^n]     */
    for (size_t k = 0; k < n; ++k) f[k] = a[k] + tau * b[k];   /* f~ (in f) */
    orc_theta(P, f, c);                 /* Theta[f~]            */
    for (size_t k = 0; k < n; ++k) f[k] = a[k] + 0.5 * tau * (b[k] + c[k]);
  }
  free(g); free(a); free(b); free(c);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Observables                                                              */
/* ------------------------------------------------------------------------ */

/* obs[0] mass      = sum f dx^2 dp^2
 * obs[1] energy    = sum f (p1^2/2m + p2^2/2m + V(x1) + V(x2) + gamma W(r)) dV
 *                    + (c_H/2) sum_i (n_1 V_H[n_1] + n_2 V_H[n_2])(x_i) dx
 * obs[2] purity    = Tr rho1^2 = 2 pi hbar sum f1^2 dx dp, f1 = sum_{x2,p2} f dx dp
 * obs[3] linear entropy = 1 - purity
 * obs[4] l2 norm   = sqrt(sum f^2 dV)
 * n1 (optional)    = n_1(x_i);  n12 (optional) = sum_{p1,p2} f dp^2 on [i1][i2]. */
void orc_observables(const orc_problem *P, const double *f, double *obs, double *n1out, double *n12) {
  int nx = P->nx, nk = P->nk, M = P->M;
  double dV = P->dx * P->dx * P->dp * P->dp;
  double mass = 0.0, ekin = 0.0, epot = 0.0, l2 = 0.0;
  double *f1 = (double *)calloc((size_t)nx * nk, sizeof(double));
  for (int i1 = 0; i1 < nx; ++i1)
    for (int i2 = 0; i2 < nx; ++i2) {
      double pair = 0.0;
      int d = ((i1 - i2) % nx + nx) % nx;
      double vx = P->vext_grid[i1] + P->vext_grid[i2] + P->gamma * P->w_shift[d * M + 0];
      for (int a = 0; a < nk; ++a)
        for (int b = 0; b < nk; ++b) {
          double v = f[idx4(P, i1, i2, a, b)];
          double p1 = (a - nk / 2) * P->dp, p2 = (b - nk / 2) * P->dp;
          mass += v * dV;
          ekin += v * (p1 * p1 + p2 * p2) / (2 * P->mass) * dV;
          epot += v * vx * dV;
          l2 += v * v * dV;
          pair += v * P->dp * P->dp;
          f1[(size_t)i1 * nk + a] += v * P->dx * P->dp;
        }
      if (n12) n12[i1 * nx + i2] = pair;
    }
  double *na = (double *)malloc(sizeof(double) * nx), *nb = (double *)malloc(sizeof(double) * nx);
  orc_marginals(P, f, na, nb);
  double eh = 0.0;
  if (P->c_h != 0.0) {
    const double *ker = P->hartree_kind == 1 ? P->h_shift : P->w_shift;
    const double fac = P->hartree_kind == 1 ? 1.0 : P->gamma * P->dx;
    for (int i = 0; i < nx; ++i) {
      double va = 0.0, vb = 0.0;
      for (int q = 0; q < nx; ++q) {
        int d = ((i - q) % nx + nx) % nx;
        va += ker[d * M + 0] * na[q];
        vb += ker[d * M + 0] * nb[q];
      }
      eh += 0.5 * P->c_h * fac * (va * na[i] + vb * nb[i]) * P->dx;
    }
  }
  double pur = 0.0;
  for (size_t k = 0; k < (size_t)nx * nk; ++k) pur += f1[k] * f1[k];
  pur *= 2.0 * ORC_PI * P->hbar * P->dx * P->dp;
  obs[0] = mass; obs[1] = ekin + epot + eh; obs[2] = pur; obs[3] = 1.0 - pur; obs[4] = sqrt(l2);
  if (n1out) for (int i = 0; i < nx; ++i) n1out[i] = na[i];
  free(f1); free(na); free(nb);
}

/* Neutralised periodic Poisson Hartree term (the 1-D Coulomb example of
 * Sec. 2.3 with an ion background that cancels the zero mode):
 *   -V_H'' = n - mean(n),  V_H(y) = sum_{m != 0} a_m e^{i k_m y} / k_m^2,
 *   k_m = 2 pi m / L,  a_m = (1/N_x) sum_q n(x_q) e^{-i k_m x_q},
 * the N_x-point series with, for even N_x, the Nyquist mode m = N_x/2 taken
 * as its cosine half (reading R15).  As a convolution:
 *   V_H(y) = sum_q G(y - x_q) n(x_q),
 *   G(r) = (1/N_x) [ 2 sum_{0 < m < N_x/2} cos(k_m r) / k_m^2 + cos(k_{N_x/2} r) / k_{N_x/2}^2 ].
 * Sets G on the fine points d dx + l h' and switches the Hartree term to it. */
void orc_set_hartree_poisson(orc_problem *P) {
  int nx = P->nx, M = P->M;
  if (!P->h_shift) P->h_shift = (double *)malloc(sizeof(double) * nx * M);
  for (int d = 0; d < nx; ++d)
    for (int l = 0; l < M; ++l) {
      double r = d * P->dx + l * P->hp, g = 0.0;
      for (int m = 1; 2 * m < nx; ++m) {
        double k = 2.0 * ORC_PI * m / P->L;
        g += 2.0 * cos(k * r) / (k * k);
      }
      if (nx % 2 == 0) {
        double k = ORC_PI * nx / P->L;
        g += cos(k * r) / (k * k);
      }
      P->h_shift[d * M + l] = g / nx;
    }
  P->hartree_kind = 1;
}

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
