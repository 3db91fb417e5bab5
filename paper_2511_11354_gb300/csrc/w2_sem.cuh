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
cudaError_t launch_sem_phi(const SemTabArgs &a, cudaStream_t s);  // Phi rows only (rows -h .. h at spacing dx)

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
  const float2 *cpdf = nullptr;   // the same factors as double-float (hi, lo) pairs
  const float2 *wtsdf = nullptr;  // 6 times the weights, as pairs (the pair solve runs on eta / 6)
  const float2 *fwdc = nullptr;   // [28] (-1)^k c*^(k+1) and (-c*)^k, c* = 2 - sqrt(3), as pairs
  const float2 *bwdc = nullptr;
};
// df = 1: the recursion and the four-term evaluation in double-float pairs on
// the FP32 pipe (FP64 in and out, converted with integer operations).
cudaError_t launch_sem_adv(int axis, const SemAdvArgs &a, cudaStream_t s, int df = 0);
int sem_adv_cols(int nx, int np);

// out = x + a * y (y2 == null) or out = x + a * (y + y2), n elements.
cudaError_t launch_sem_axpy(long long n, const double *x, double a, const double *y, const double *y2, double *out,
                            cudaStream_t s);

// Observables: per-X partials, per-x1 partials (with the densities), then one
// fixed-order reduction.
struct SemObsArgs {
  int nx, np;
  double dx, hbar, mass, gamma, c_h;
  const double *f, *p, *w, *vext, *wgrid;
  double *xpart;        // [nx*nx][4 + np] per-X partials, then [nx][5] per-x1 partials
  double *out;          // [8 + nx]
};
cudaError_t launch_sem_obs(const SemObsArgs &a, cudaStream_t s);

// Occupation numbers on the bounded box: f1[i][j] = dx sum_{i2} sum_{j2} w_{j2} f
// (f1: [nx][np]); g[k] = f1 at x_0 + k dx / 2 (k < 2 nx - 1; the odd rows from the
// natural cubic spline of each column, eta scratch [nx + 2][np]); and
// rho[b][c] = dx sum_j g[b + c][j] conj(Phi_j((c - b) dx / 2)) with the
// transform rows phr/phi [2 nx - 1][np] (k_sem_phi at half steps), made
// Hermitian.
cudaError_t launch_sem_rdm(int nx, int np, double dx, const double *f, const double *w, const double *cp, double *f1,
                           double *eta, double *g, const double *phr, const double *phi, double2 *rho, cudaStream_t s);

// erm[i] = [Er | -Ei](i) from eier[i] = [Ei | Er](i) (np rows of 2 Ny).
cudaError_t launch_sem_erm(int np, int Ny, const double *eier, double *erm, cudaStream_t s);

// out[r][c] = in[r][c] for c < c0, -in[r][c] for c >= c0 (rows x cols, row-major).
cudaError_t launch_sem_negcols(int rows, int cols, int c0, const double *in, double *out, cudaStream_t s);

// Scaling: out = a * in (n elements).
cudaError_t launch_sem_scale(long long n, double a, const double *in, double *out, cudaStream_t s);

// Exact slices of FP64 lines for the tensor-core products (w2_gemms.cu).
// Row mode (cols = 0): line l holds in[l * ls + k], k < K (K <= 512); the
// planes are [6][L][Kp] (plane stride pP = L * Kp), zero past K.  Column
// mode (cols = 1): line l is column l of a row-major K x L matrix with row
// stride ks; the planes are [6][Kp][ldp] (pP = Kp * ldp), zero past K and L.
// ex[l] receives the line exponent E (every |v| < 2^E).  Batch b splits as
// (b / bdiv, b % bdiv) for the input (strides sIn1, sIn2); planes and
// exponents move by b * sP and b * sE.  Mode 1 (rows only) first multiplies
// element (c = l, k) by w(r) (W(rho + u dx) - W(rho - u dx)), r = k % (h+1),
// u = r - (c - h), rho = i1 - i2 of X = x0 + b (the two-body D_V weighting),
// read from dtab[w == 2][rho + nx - 1][u + 2h] ((2 nx - 1) x (4h + 1) each).
struct SliceArgs {
  int L, K, Kp, ldp;
  const double *in;
  long long ls, ks, sIn1, sIn2;
  uint16_t *planes;
  long long pP, sP;
  int *ex;
  long long sE;
  int nbatch, bdiv;
  const double *dtab;
  int nx, h, x0;
};
cudaError_t launch_slice(int cols, int mode, const SliceArgs &a, cudaStream_t s);
// Column slices of w D (.) A for S'^T = E B (see k_slice_dstack): L = Nyh lines,
// K = 2 Ny, in = A^T per X (row stride ls, batch stride sIn1), dtab, nx, h, x0.
cudaError_t launch_slice_dstack(const SliceArgs &a, cudaStream_t s);
int slice_kp(int K);

// C_b (=|+=) A_b B_b from slices: A planes [6][M][lda] (pA plane stride,
// line = row), B planes [6][N][ldb] (b_kn = 0, line = column) or [6][K][ldb]
// (b_kn = 1, row-major), contraction over k0 .. k0 + K - 1 (K <= 256, k0 a
// multiple of 32; the planes hold zeros past the data up to the next
// multiple of 32).  Exponents Ae[M], Be[N].  beta = 1 adds to C.
struct GemmSArgs {
  int M, N, K, k0;
  const uint16_t *A;
  long long lda, pA, sA1, sA2;
  const int *Ae;
  long long sAe1, sAe2;
  const uint16_t *B;
  long long ldb, pB, sB1, sB2;
  const int *Be;
  long long sBe1, sBe2;
  double *C;
  long long ldc, sC1, sC2;
  int beta, nbatch, bdiv;
};
cudaError_t launch_gemms(int b_kn, const GemmSArgs &g, cudaStream_t s);

}  // namespace w2sem
