// Internal declarations shared by the w2 library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/w2.h"

namespace w2 {

// Sum of term(k) over k in [0, len), split over the four lanes of a quad
// (lane r of the quad takes k = r, r + 4, ...) and combined by two xor
// shuffles, so the bits do not depend on the block size.  Every lane of the
// warp calls it; valid = false contributes zero.
template <typename F>
__device__ __forceinline__ double quad_sum(bool valid, int len, F term) {
  const int r = threadIdx.x & 3;
  double s = 0.0;
  if (valid) {
#pragma unroll 4
    for (int k = r; k < len; k += 4) s += term(k);
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  return s;
}


// Static one-body / pair potential samples and the per-call densities that
// build the kernels K(x, j) of the pseudo-difference operator (Sec. 3.1):
//   K(x, j) = 1/(hbar nk) sum_{l=1}^{nk-1} [U(x + l h') - U(x - l h')] sin(pi l j / nk)
// with h' = L / (2 nk); K(x, -j) = -K(x, j), K(x, 0) = 0.
struct TabArgs {
  int nx, nk, M;
  double dx, dp, hbar;
  double gamma, c_h, c_xc;
  int xc_kind;
  int pair_mode;            // 1: U = gamma W(d dx + l h') for row d (the pair kernel K12)
  const double *xsum;       // [nx][nx] per-X momentum sums of the state (or null)
  const double *vext_fine;  // [nx][M]
  const double *w_fine;     // [nx][M]
  const double *d_fine;     // [nx][M] trigonometric interpolation weights (xc only)
  const double *sintab;     // [M] sin(pi m / nk)
  double *K;                // pair_mode 0: [2][nx][2nk-1]; pair_mode 1: [nx][2nk-1]
  const double *h_fine = nullptr;  // [nx][M] Hartree kernel G(d dx + l h') (neutralised Poisson);
                                   // null: gamma dx W (w_fine)
};

struct ThetaArgs {
  int nx;
  const double *in;         // state the operator acts on
  const double *h;          // corrector base (mode 1) or null
  double *out;              // mode 0: Theta[in]; mode 1: h + half_tau Theta[in]
  double *xsum;             // mode 1: per-X sums of out
  const double *K1, *K2, *K12;
  double half_tau;
  const float *pair = nullptr;  // if set: the two-body term, [nx*nx][nk*nk], used instead of K12
};

struct AdvArgs {
  int nx;
  const double *in0, *in1;  // arrays to shift (in1 may be null)
  double *out0, *out1;      // outputs
  const int *k0tab;         // [nk] integer part of the foot offset
  const double *wtab;       // [nk][4] B-spline weights times -6 z
  double z, zscale;         // pole z = sqrt(3) - 2 and 1/(1 - z^n) (or 1)
  int nterm;                // terms of the periodic initial sums
  double tau;               // combination weight (x1 pass with two arrays)
};

// The shift of the sliced FP64 path in double-float pairs (w2_adv_df.cu).
struct AdvDFArgs {
  int nx;
  const void *in0, *in1;    // FP64 arrays, or pair arrays in the second pass (in1 may be null)
  void *out0, *out1;        // pair arrays in the first pass, FP64 in the second
  const int *k0tab;         // [nk] integer part of the foot offset
  const float2 *wdf;        // [nk][4] B-spline weights times -6 z, (hi, lo)
  const float2 *zpow;       // [32] z^k, (hi, lo)
  float2 z, zscale, tau, half_tau;  // (hi, lo)
  int nterm;                // terms of the periodic start sums (<= 32)
};

struct ObsArgs {
  int nx, nk, M;
  double dx, dp, hbar, mass, gamma, c_h;
  const double *f;          // FP64 state, or
  const float *f32;         // FP32 state (exactly one is non-null)
  const double *vext_grid;  // [nx]
  const double *w_fine;     // [nx][M]; column 0 is W(fold(d dx))
  double *xpart;            // [nx*nx][3 + nk] per-X partials, then [nx][8] per-x1 partials
  double *out;              // [8 + nx + nx*nx]
  const double *h_fine = nullptr;  // as in TabArgs (column 0: the kernel at grid distances)
};

struct Theta32Args {
  int nx;
  const float *in;          // state the operator acts on
  const float *base;        // mode 1: the state f
  const float *h;           // mode 1: the corrector increment
  float *out;               // mode 0: Theta[in]; mode 1: base + (h + half_tau Theta[in])
  const double *K1, *K2, *K12;
  float half_tau;
};

struct Adv32Args {
  int nx;
  const float *f, *g;       // DIR 0 inputs (g may be null); DIR 1 reads f
  float *d2, *g2;           // DIR 0 outputs
  const float *d2in, *g2in; // DIR 1 inputs (g2in may be null)
  float *ft, *dh;           // DIR 1 outputs
  const int *k0tab;         // [nk]
  const float *wtab;        // [nk][4] evaluation weights (times -6 z)
  const float *ctab;        // [nk][8] merged increment taps, offsets -3..3, [7] = usable
  float z, zscale;
  int nterm;
  float tau;
};

// A persistent batched launch over the work items of several instances:
// inst[k] is the k-th instance of the class, items [off[k], off[k+1]) are its.
struct BatchLaunch {
  int grid;
  const int *inst;
  const int *off;
  int n;
};

struct BXsum {
  const float *f;
  double *xsum;
  int nk;
};

// Harmonics of the pair distance r = x1 - x2 in an MLP input row.
constexpr int kMlpHarmonics = 8;

enum GemmEpi { GEMM_STORE = 0, GEMM_BIAS_SILU = 1, GEMM_BIAS_SCALE = 2, GEMM_DSILU = 3 };

// C[M][N] = sum_k A(m, k) B(k, n) with bf16 A(m, k) = A[m*sam + k*sak] and
// B(k, n) = B[k*sbk + n*sbn], followed by the epilogue `epi`.
struct GemmArgs {
  const void *A, *B;
  long long sam, sak, sbk, sbn;
  int M, N, K;
  int epi;
  const float *bias;   // [N] (BIAS_*)
  const float *aux;    // [M][N] pre-activation Z (DSILU)
  float scale;         // BIAS_SCALE
  float *out_f32;      // [M][N]
  uint16_t *out_bf16;  // [M][N] (BIAS_SILU, DSILU)
};

// Input rows of the learned two-body term (see w2_mlp.cu).
struct FeatArgs {
  int nx, nk, din;
  double dx, dp;
  float s_f, s_f1;
  float *f1;           // [nx][nk] reduced one-body Wigner function (refreshed when f1_src_rows > 0)
  int f1_src_rows;
  const int *xs;       // spatial points of the rows (null: row r is X = r)
  uint16_t *x;         // [rows][din] bf16
};

// Occupation numbers (w2_rdm.cu): f1 of the state, rho1 dx on the grid, and
// the batched Jacobi eigensolver of complex Hermitian matrices.
cudaError_t launch_rdm_f1(const void *f, int f64, double *f1, int nx, int nk, double dx, double dp, cudaStream_t s);
cudaError_t launch_rdm_rho(const double *f1, const double *kh, double *fh, const double2 *ph, double2 *rho, int nx,
                           int nk, double dx, cudaStream_t s);
cudaError_t launch_jacobi_herm(double2 *mats, int n, int batch, double *eig, cudaStream_t s);
cudaError_t launch_corr_entropy(const double *eig, int n, double *entropy, cudaStream_t s);
// Eigenvalues of Hermitian matrices (w2_heig.cu): Householder tridiagonal
// reduction in a cluster of 8 CTAs (matrix in shared memory) and bisection,
// for n up to herm_eig_tridiag_max_n(); the Jacobi solver above beyond.  The
// matrices are overwritten; eig [batch][n], largest first.
cudaError_t launch_herm_eigvals(double2 *mats, int n, int batch, double *eig, cudaStream_t s);
int herm_eig_tridiag_max_n();

// Record the CUDA error behind a W2_ERR_CUDA return (read by w2_last_cuda_error).
void note_cuda_error(cudaError_t e);

// Launchers (return the launch error).
cudaError_t launch_tables(const TabArgs &a, cudaStream_t s);
cudaError_t launch_theta_f64(int nk, int mode, const ThetaArgs &a, cudaStream_t s);
// FP64-accurate sweep by exact 8-bit slices on the BF16 tensor cores (w2_f64s.cu);
// nk in {16, 32, 48, 64}; a.xsum must be null.
cudaError_t launch_theta_f64s(int nk, int mode, const ThetaArgs &a, cudaStream_t s);
cudaError_t prepare_kernels_f64s(int nk);
bool nk_supported_f64s(int nk);
cudaError_t launch_adv_f64(int nk, int dir, int two, const AdvArgs &a, cudaStream_t s);
cudaError_t launch_adv_df(int nk, int dir, int two, const AdvDFArgs &a, cudaStream_t s);
cudaError_t prepare_kernels_adv_df(int nk);
cudaError_t launch_xsum_f64(int nx, int nk, const double *f, double *xsum, cudaStream_t s);
cudaError_t launch_xsum_f32(int nx, int nk, const float *f, double *xsum, cudaStream_t s);
cudaError_t launch_obs(const ObsArgs &a, cudaStream_t s);
cudaError_t prepare_kernels_f64(int nk);
bool nk_supported_f64(int nk);
cudaError_t prepare_kernels_f32(int nk);
bool nk_supported_f32(int nk);
int adv_items_per_line_f32(int nk);  // column blocks of the FP32 shift per (n1, x) line
cudaError_t launch_theta_f32(int nk, int mode, const Theta32Args &a, cudaStream_t s);
cudaError_t launch_adv_f32(int nk, int dir, const Adv32Args &a, cudaStream_t s);
cudaError_t launch_btheta_f32(int nk, int mode, const BatchLaunch &b, const Theta32Args *args, cudaStream_t s);
cudaError_t launch_badv_f32(int nk, int dir, const BatchLaunch &b, const Adv32Args *args, int nxmax, int pieces,
                            cudaStream_t s);
// Threads per column of the FP32 shift for lines of nx points (pieces of 32
// rows or more, at most 8).
__host__ __device__ inline int adv32_pieces(int nx) { return nx >= 256 ? 8 : nx >= 128 ? 4 : nx >= 64 ? 2 : 1; }
cudaError_t launch_btables(const TabArgs *args, const int *off, int n, int grid, int nxmax, int mmax,
                           cudaStream_t s);
cudaError_t launch_bxsum(const BXsum *args, const int *off, int n, int grid, cudaStream_t s);
cudaError_t launch_gemm(const GemmArgs &a, cudaStream_t s);
// Pipelined inference GEMM (unit-stride A rows and B rows; BIAS_SILU / BIAS_SCALE epilogues).
cudaError_t launch_gemm_fwd(const GemmArgs &a, cudaStream_t s);
cudaError_t launch_features(const FeatArgs &a, const void *f, int f64, int rows, cudaStream_t s);
cudaError_t launch_colsum(const float *in, float *out, int M, int N, cudaStream_t s);
cudaError_t launch_adam(float *p, const float *g, float *m, float *v, uint16_t *pb, size_t n, float lr, float b1,
                        float b2, int t, float eps, cudaStream_t s);
cudaError_t launch_f2bf(const float *in, uint16_t *out, size_t n, cudaStream_t s);
cudaError_t launch_mse(const float *Y, const float *T, float *dY, double *part, size_t n, float gscale,
                       cudaStream_t s);
cudaError_t launch_sqdiff(const float *a, const void *b, int b_f64, double *part, size_t n, double bscale,
                          cudaStream_t s);

}  // namespace w2

// A single problem on one device (the object behind the w2_ctx handle).
struct w2_ctx {
  w2_config cfg;
  cudaStream_t stream;       // borrowed
  cudaStream_t cap;          // private stream used only for graph capture
  int dev;
  int prec;                  // w2_precision
  size_t esz;                // bytes per phase-space element
  int nx, nk, M;
  size_t npts;
  double dx, dp, hp, tau;
  double gamma, c_h, c_xc;
  bool have_pot, have_state;
  int64_t steps;
  w2_status sticky;
  // phase-space arrays
  double *f, *g, *t1, *t2;
  // small device buffers
  double *xsum, *xsum2;       // [nx*nx]
  double *K, *K12;            // [2][nx][2nk-1], [nx][2nk-1]
  double *vext_fine, *w_fine, *d_fine, *sintab, *vext_grid;
  int *k0tab;
  double *wtab;
  float2 *wdf, *zpow;        // double-float shift weights [nk][4] and z^k [32] (sliced path)
  int hartree_kind;          // W2_HARTREE_PAIR or W2_HARTREE_POISSON
  double *h_fine;            // [nx][M] Poisson Hartree kernel (W2_HARTREE_POISSON), else null
  // occupation numbers (allocated by the first w2_occupations)
  double *rdm_f1, *rdm_fh, *rdm_kh, *rdm_eig;  // [nx][nk], [nx][nk], [nx], [nx + 1]
  double2 *rdm_ph, *rdm_rho;                   // [nx][nk] phases, [nx][nx] rho1 dx
  float *wtab32, *ctab32;    // FP32 shift weights and merged increment taps
  double *xpart, *obs_out, *h_obs;
  double z, zscale;
  int nterm;
  cudaGraphExec_t graph;
  bool graph_ready;
  // learned form (FP64 contexts): the MLP's pair term replaces K12
  w2_mlp *mlp;
  bool learned_active;     // the step currently uses the network
  int judge_every;         // steps between judgements (0: never)
  double judge_tol;        // fall back to the exact term above this error
  int since_judge, judged;
  double last_err;
  float *f1;               // [nx][nk] reduced Wigner function for the features
  uint16_t *xrows;         // [nx*nx][din] feature rows
  double *Kzero;           // [2][nx][2nk-1] zero one-body tables (pair-only sweeps)
  // staged host input (allocated by the first w2_stage_state): one state,
  // filled on a private copy stream while the context's stream computes
  void *stage;
  cudaStream_t copy;
  cudaEvent_t ev_staged;   // recorded on copy after the host copy
  cudaEvent_t ev_taken;    // recorded on stream after w2_use_staged_state read the stage
  bool stage_pending, taken_recorded;
};

namespace w2 {
int mlp_din(const w2_mlp *m);
int mlp_nk(const w2_mlp *m);
int mlp_maxrows(const w2_mlp *m);
float mlp_scale(const w2_mlp *m, int which);  // 0: s_f, 1: s_f1, 2: s_y
float *mlp_out(w2_mlp *m);
double *mlp_part(w2_mlp *m);
double *mlp_hpart(w2_mlp *m);
// Inference forward (pipelined GEMM with fused epilogues).
cudaError_t mlp_forward(w2_mlp *m, const uint16_t *x, int rows, float *y, float s, cudaStream_t st);
TabArgs tab_args(w2_ctx *ctx, const double *xsum, int pair_mode);
Adv32Args adv32_args(w2_ctx *ctx);
}  // namespace w2
