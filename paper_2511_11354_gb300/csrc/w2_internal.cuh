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
  // sliced sweep only: the input is exchange symmetric, in(x2, x1, p2, p1) =
  // in(x1, x2, p1, p2), so the blocks with i1 <= i2 are computed and the
  // mirror block X' = (i2, i1) of each is written from its transpose
  int sym = 0;
  // tcgen05 sweep only: set to nonzero if a bounded wait on the tensor core gave up
  int *err = nullptr;
  int stall = 0;               // tcgen05 sweep, fault injection: leave one batch of products out
  long long wait_limit = 0;    // tcgen05 sweep: SM clocks per bounded wait (0: about a second)
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

// The shift of one axis split into np patches joined by perfectly matched
// boundary conditions (w2_pmbc.cu).
struct PatchArgs {
  int nx, np, M, G, nnb;    // grid, patches, points per patch, ghost points per side, slope stencil half-width
  const double *in0, *in1;  // arrays to shift (in1 may be null)
  double *out0, *out1;
  double *xs;               // [arrays][np][2][lines] slope parts sent to the neighbours
  double *gh;               // [arrays][np][2][G][lines] ghost samples sent to the neighbours
  const double *D;          // [2 nnb + 1] slope stencil D_{-nnb..nnb}
  const double *inv_m, *cp; // [M + 2G] Thomas factors of the local system
  const int *k0tab;         // [nk]
  const double *wb;         // [nk][4] B-spline weights b_a(theta)
  double h, tau;
};
cudaError_t launch_adv_pmbc(int nk, int dir, int two, const PatchArgs &a, cudaStream_t s);
// The per-X sums of a context's state (which the next step's tables read).
cudaError_t state_sums(w2_ctx *ctx, cudaStream_t s);

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
  const int *err = nullptr;         // device error word of the sweeps (out[5] = its value), or null
};

struct Theta32Args {
  int nx;
  const float *in;          // state the operator acts on
  const float *base;        // mode 1: the state f
  const float *h;           // mode 1: the corrector increment
  float *out;               // mode 0: Theta[in]; mode 1: base + (h + half_tau Theta[in])
  const double *K1, *K2, *K12;
  float half_tau;
  double *xsum = nullptr;   // mode 1: exact per-X sums of out (or null)
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
  // the coefficient solve in double-float pairs (hi, lo)
  float2 zdf, zscale_df;    // z and 1/(1 - z^n) (or 1) of the start sums
  const float2 *zpow;       // [32] z^k
  int nterm_df;             // terms of the start sums (<= 28: |z|^28 < 2^-53)
};

struct BXsum {
  const float *f;
  double *xsum;
  int nk;
};

// One step of a batch of FP32 instances as a single persistent launch.  The
// work items of the seven phases of a Lawson step (tables of f^n, Theta
// predictor, shift x2, shift x1 + combination, per-X sums of f~, tables,
// Theta corrector with the per-X sums of f^{n+1}) form one list, phase after
// phase (the sums of f^n come from the previous step); CTAs take items
// from a global counter, and an item of phase p of instance i starts once
// every item of phase p - 1 of instance i has finished (per-instance counters).
// Items are taken in list order by running CTAs only, so every wait is for
// items already taken by running CTAs and ends; each wait is still bounded by
// wait_cycles (clock64), after which the CTA records W2_ERR_TIMEOUT in *err
// and every CTA stops taking items.  The last CTA to leave resets the
// counters, so the launch can be replayed (one graph node per step).
constexpr int kBatchPhases = 7;
constexpr int kBatchThreads = 256;
struct BStepPlan {
  int n;                      // instances
  const int *phase_off;       // [kBatchPhases + 1] first global item of each phase
  const int *inst_off;        // [kBatchPhases][n + 1] items of each instance within its phase
  const int *units;           // [kBatchPhases][n] work units (X, table row or shift slab) of each instance
  const int *gsz;             // [kBatchPhases] units per item of each phase
  const int *nk;              // [n]
  const int *nx;              // [n]
  int smem;                   // dynamic shared memory of the launch (bytes)
  const BXsum *xs_ft;         // [n] per-X sums of f~
  const TabArgs *tab;         // [n]
  const Theta32Args *th;      // [2 n] predictor, corrector
  const Adv32Args *adv;       // [2 n] x2 pass, x1 pass
  int *next;                  // the work counter
  int *done;                  // [kBatchPhases][n] finished items
  int *left;                  // CTAs that have left
  int *err;                   // 0, or a w2_status of the step
  const int *skip;            // test hook: 1 + p * n + i stops counting phase p of instance i (or 0)
  long long wait_cycles;      // bound of every wait
};
// Tile shapes of the persistent step: columns per CTA of the shift items (32
// or 64, at most nk), warps per 16-row block of the Theta items (1 or 2), and
// the work units a CTA takes per item (each phase's units divided into about
// items_per_cta items per CTA of the grid).
struct BStepShape {
  int shift_cols, theta_split, items_per_cta;
};
size_t bstep_smem(const BStepShape &sh, int nxmax, int nkmax);
cudaError_t prepare_bstep(const BStepShape &sh);
int bstep_max_ctas_per_sm(const BStepShape &sh, size_t smem);
cudaError_t launch_bstep(const BStepShape &sh, const BStepPlan &p, int grid, size_t smem, cudaStream_t s);
// Columns per shift item for a tile width CS: CS, or nk when nk <= CS, or 16
// when CS does not divide nk.
__host__ __device__ constexpr int bstep_cols(int nk, int cs) { return nk <= cs ? nk : (nk % cs == 0 ? cs : 16); }
int bstep_shift_items(int nk, int shift_cols);  // shift items per (n1, x) line

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
// The same sweep with every digit product on tcgen05 (w2_f64t.cu): N_k = 64,
// no learned pair term.
bool theta_t_supported(int nk, const ThetaArgs &a);
cudaError_t prepare_kernels_f64t();
cudaError_t launch_theta_f64t(int mode, const ThetaArgs &a, cudaStream_t s);
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
cudaError_t launch_theta_f32(int nk, int mode, const Theta32Args &a, cudaStream_t s);
// The same sweep with the state in three BF16 parts and the kernel in four
// (mma.sync m16n8k16); nk as launch_theta_f32.
cudaError_t prepare_kernels_b3(int nk);
cudaError_t launch_theta_b3(int nk, int mode, const Theta32Args &a, cudaStream_t s);
cudaError_t launch_adv_f32(int nk, int dir, const Adv32Args &a, cudaStream_t s);
// Threads per column of the FP32 shift for lines of nx points (at most 16;
// from 128 points on, pieces of 16 rows or more: the double-float recursions
// are serial chains, and more of them per SM hide their latency better than
// the extra start sums cost).
__host__ __device__ inline int adv32_pieces(int nx) { return nx >= 256 ? 16 : nx >= 128 ? 8 : nx >= 64 ? 2 : 1; }
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
cudaError_t launch_sqdiff64(const double *a, const double *b, double *part, size_t n, cudaStream_t s);

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
  // w2_observables_enqueue / _collect: two pinned result slots, their copy
  // events and the step counts at enqueue time
  double *h_obs_slot[2];
  cudaEvent_t ev_obs[2];
  bool obs_pending[2];
  long long obs_steps[2];
  double z, zscale;
  int nterm;
  // patch decomposition of the shift (w2_set_patches): patches along x1 and x2
  // (1: the global spline), ghost points, stencil and Thomas tables per axis
  int np_ax[2], pm_G;
  double *pm_D, *pm_wb, *pm_tab[2], *pm_xs, *pm_gh;
  // captured steps, one per state buffer the step has run on (w2_use_staged_state
  // swaps the state and staging buffers, so two graphs alternate)
  cudaGraphExec_t graph[2];
  const void *graph_f[2];
  bool graph_ok[2];
  // learned form (FP64 contexts): the MLP's pair term replaces K12
  w2_mlp *mlp;
  bool learned_active;     // the step currently uses the network
  bool exchange_sym;       // w2_set_exchange_symmetry: sliced sweeps on the blocks i1 <= i2
  bool tc_path;            // w2_set_tensor_path: sliced sweeps on tcgen05 where supported
  int *d_err;              // device error word: bounded tensor-core waits that gave up
  int dbg_stall;           // w2_debug_sweep_stall: fault injection into the tcgen05 sweep
  long long dbg_wait;      // and its wait limit (SM clocks; 0: the default)
  int judge_every;         // steps between judgements (0: never)
  double judge_tol;        // fall back to the exact term above this error
  int since_judge, judged;
  double last_err;
  float *f1;               // [nx][nk] reduced Wigner function for the features
  uint16_t *xrows;         // [nx*nx][din] feature rows
  double *Kzero;           // [2][nx][2nk-1] zero one-body tables (pair-only sweeps)
  double *Klearn;          // [nx][2nk-1] the kernel network's pair table (kernel networks)
  // staged host input (allocated by the first w2_stage_state): one state,
  // filled on a private copy stream while the context's stream computes
  void *stage;
  cudaStream_t copy;
  cudaEvent_t ev_staged;   // recorded on copy after the host copy
  cudaEvent_t ev_taken;    // recorded on stream after w2_use_staged_state read the stage
  bool stage_pending, taken_recorded;
};

namespace w2 {
// Every allocation of the library: cudaMalloc / cudaMallocHost behind the
// host-side failure hook (w2_debug_fail_alloc).  On an injected failure *p
// is null and the result is cudaErrorMemoryAllocation.
cudaError_t dev_alloc(void **p, size_t bytes);
cudaError_t host_alloc(void **p, size_t bytes);
int mlp_din(const w2_mlp *m);
int mlp_nk(const w2_mlp *m);
int mlp_maxrows(const w2_mlp *m);
float mlp_scale(const w2_mlp *m, int which);  // 0: s_f, 1: s_f1, 2: s_y
float *mlp_out(w2_mlp *m);
double *mlp_part(w2_mlp *m);
double *mlp_hpart(w2_mlp *m);
// Inference forward (pipelined GEMM with fused epilogues).
cudaError_t mlp_forward(w2_mlp *m, const uint16_t *x, int rows, float *y, float s, cudaStream_t st);
int mlp_kind(const w2_mlp *m);  // 0: the pair term per point; 1: the pair kernel per distance
// Kernel network (w2_pairk.cu): the distance features, the predicted pair
// table, and the training residual, row gradients and targets.
cudaError_t launch_rfeat(uint16_t *x, int nx, int din, cudaStream_t s);
cudaError_t launch_pairk_table(const float *y, int nx, int nk, float inv_sy, double *K, cudaStream_t s);
cudaError_t launch_pairk_grad(const double *f, const double *p, const int *dr, int rows, const float *y, int nx, int nk,
                              float inv_sy, double *res, double *g, double *part, cudaStream_t s);
cudaError_t launch_pairk_target(const float *y, const double *g, const int *dr, int rows, int nx, int nk, float inv_sy,
                                double inv_p2, float *t, double *dldy, cudaStream_t s);
TabArgs tab_args(w2_ctx *ctx, const double *xsum, int pair_mode);
Adv32Args adv32_args(w2_ctx *ctx);
}  // namespace w2
