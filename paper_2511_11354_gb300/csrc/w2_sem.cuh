// Internal declarations of the non-periodic (spectral-element) path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/w2_sem.h"

namespace w2sem {

// Batched FP64 matrix product on the FP64 pipe:
//   C_b = alpha * A_b * B_b + beta * C_b,   b in [0, nbatch)
// A(m, k) = A[m * lda + k] (a_col = 0) or A[m + k * lda] (a_col = 1);
// B(k, n) = B[k * ldb + n] (b_col = 0) or B[k + n * ldb] (b_col = 1);
// C(m, n) = C[m * ldc + n].  Batch b splits as (b / bdiv, b % bdiv) and moves
// each operand by b1 * s?1 + b2 * s?2 elements.  C must not overlap A or B.
struct Gemm64 {
  int M, N, K;
  const double *A;
  long long lda;
  int a_col;
  const double *B;
  long long ldb;
  int b_col;
  double *C;
  long long ldc;
  double alpha, beta;
  int nbatch, bdiv;
  long long sA1, sA2, sB1, sB2, sC1, sC2;
};
cudaError_t launch_gemm64(const Gemm64 &g, cudaStream_t s);

// Static tables (Sec. 3.2).
struct SemTabArgs {
  int nx, M, Q, np, h;
  double dx, width, hbar, Lp;
  const double *p;      // [np] collocation momenta
  const double *centre; // [M] cell centres
  const double *cheb;   // [Q][Q] discrete Chebyshev transform C[l][q]
  double *osc;          // [nx][Q][2]: O_l(width d dx / hbar), d = 0..nx-1 (re, im)
  double *psi;          // [2nx-1][np][np] one-body table (d = -(nx-1)..nx-1)
  double *phir, *phii;  // [Ny][np] transform rows Phi_j(y_n), n = -h..h
  double *ph;           // [2Nyh][2np]  [[Phr_h, -Phi_h], [Phi_h, Phr_h]]
  double *eh;           // [2][np][2Nyh] [Er_h | -Ei_h] and [Ei_h | Er_h]
  double *eier;         // [np][2Ny]   [Ei | Er]
};
cudaError_t launch_sem_osc(const SemTabArgs &a, cudaStream_t s);
cudaError_t launch_sem_tables(const SemTabArgs &a, cudaStream_t s);

// Per-X weighted sums xs[X] = sum_{j1,j2} w_j1 w_j2 f[X][j1][j2] and the
// densities n[0..nx) = dx sum_i2 xs, n[nx..2nx) = dx sum_i1 xs.
cudaError_t launch_sem_marginal(int nx, int np, double dx, const double *f, const double *w, double *xs,
                                double *n, cudaStream_t s);

// Potentials U_i = vext + c_h dx sum_q W((i-q) dx) n_q + c_xc phi(n_i) for
// both particles (n, U: [2][nx]), and the Toeplitz rows
// ut[k][d + nx - 1] = U_k-particle(m + d) of the one-body table product.
struct SemPotArgs {
  int nx, xc_kind;
  double dx, c_h, c_xc;
  const double *n;      // [2][nx]
  const double *vext;   // [nx]
  const double *wgrid;  // [4nx-3]: W(k dx), k = -2(nx-1)..2(nx-1)
  double *U;            // [2][nx]
  double *ut;           // [2nx][2nx-1]
};
cudaError_t launch_sem_potential(const SemPotArgs &a, cudaStream_t s);

// A[b][r][c] *= wgt(r) * (W(rho + r' - c') - W(rho - r' + c')) on a chunk of
// X = x0 .. x0 + nb - 1 (both real and imaginary row blocks).
cudaError_t launch_sem_dmul(int nx, int h, int x0, int nb, const double *wgrid, double *A, cudaStream_t s);

// Natural-boundary cubic spline shift along x1 (axis 0) or x2 (axis 1).
struct SemAdvArgs {
  int nx, np, C;
  const double *in;
  double *out;
  const double *cp;     // [nx] Thomas factors c'_i of the (1,4,1) interior system
  const int *k0;        // [np] integer part of the foot offset
  const double *wts;    // [np][4] B-spline weights
};
cudaError_t launch_sem_adv(int axis, const SemAdvArgs &a, cudaStream_t s);
int sem_adv_cols(int nx, int np);

// out = x + a * y (y2 == null) or out = x + a * (y + y2), n elements.
cudaError_t launch_sem_axpy(long long n, const double *x, double a, const double *y, const double *y2, double *out,
                            cudaStream_t s);

// Observables: per-X partials then one fixed-order reduction.
struct SemObsArgs {
  int nx, np;
  double dx, hbar, mass, gamma, c_h;
  const double *f, *p, *w, *vext, *wgrid, *n;
  double *xpart;        // [nx*nx][4 + np]
  double *out;          // [8 + nx]
};
cudaError_t launch_sem_obs(const SemObsArgs &a, cudaStream_t s);

}  // namespace w2sem
