// C ABI of the w2 library: context, host-side tables, stability precheck,
// step orchestration (one Lawson step captured into a CUDA graph).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include "w2_internal.cuh"

using namespace w2;



#define W2_TRY(call)                                    \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) {                            \
      w2::note_cuda_error(e_);                          \
      ctx->sticky = W2_ERR_CUDA;                        \
      return W2_ERR_CUDA;                               \
    }                                                   \
  } while (0)

static double fold(double x, double L) { return x - L * floor((x + 0.5 * L) / L); }

static thread_local cudaError_t g_last_cuda_error = cudaSuccess;
void w2::note_cuda_error(cudaError_t e) { g_last_cuda_error = e; }

extern "C" const char *w2_last_cuda_error(void) {
  return g_last_cuda_error == cudaSuccess ? "no CUDA error recorded" : cudaGetErrorString(g_last_cuda_error);
}

// Precisions whose state and results are FP64.
static inline bool f64_state(int prec) { return prec == W2_F64 || prec == W2_F64_SLICED; }

// The FP64 sweep of a context: on the FP64 pipe, or by exact slices on the
// BF16 tensor cores.
static cudaError_t theta64(const w2_ctx *ctx, int mode, const ThetaArgs &th, cudaStream_t s) {
  if (ctx->prec != W2_F64_SLICED) return launch_theta_f64(ctx->nk, mode, th, s);
  if (ctx->tc_path && theta_t_supported(ctx->nk, th)) {
    ThetaArgs t = th;
    t.err = ctx->d_err;
    t.stall = ctx->dbg_stall;
    t.wait_limit = ctx->dbg_wait;
    return launch_theta_f64t(mode, t, s);
  }
  return launch_theta_f64s(ctx->nk, mode, th, s);
}

// Forget the captured steps (the potentials, the Hartree kind, the patches or
// the learned form changed).
static void drop_graphs(w2_ctx *ctx) {
  for (int k = 0; k < 2; ++k) {
    if (ctx->graph_ok[k]) cudaGraphExecDestroy(ctx->graph[k]);
    ctx->graph_ok[k] = false;
    ctx->graph_f[k] = nullptr;
  }
}

// The FP32 sweep of a precision-form context: TF32 or BF16 operand splits.
static cudaError_t theta32(const w2_ctx *ctx, int mode, const Theta32Args &th, cudaStream_t s) {
  return ctx->prec == W2_F32_BF16X3 ? launch_theta_b3(ctx->nk, mode, th, s) : launch_theta_f32(ctx->nk, mode, th, s);
}

static void free_all(w2_ctx *c) {
  void *ptrs[] = {c->f, c->g, c->t1, c->t2, c->xsum, c->xsum2, c->K, c->K12, c->vext_fine, c->w_fine,
                  c->d_fine, c->sintab, c->vext_grid, c->k0tab, c->wtab, c->xpart, c->obs_out,
                  c->wtab32, c->ctab32, c->wdf, c->zpow, c->h_fine, c->rdm_f1, c->rdm_fh, c->rdm_kh,
                  c->rdm_eig, c->rdm_ph, c->rdm_rho, c->d_err};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (c->h_obs) cudaFreeHost(c->h_obs);
  for (int k = 0; k < 2; ++k) {
    if (c->h_obs_slot[k]) cudaFreeHost(c->h_obs_slot[k]);
    if (c->ev_obs[k]) cudaEventDestroy(c->ev_obs[k]);
  }
  if (c->f1) cudaFree(c->f1);
  if (c->xrows) cudaFree(c->xrows);
  if (c->Kzero) cudaFree(c->Kzero);
  if (c->Klearn) cudaFree(c->Klearn);
  for (int k = 0; k < 2; ++k)
    if (c->graph_ok[k]) cudaGraphExecDestroy(c->graph[k]);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->copy) {
    cudaStreamSynchronize(c->copy);
    cudaStreamDestroy(c->copy);
  }
  if (c->ev_staged) cudaEventDestroy(c->ev_staged);
  if (c->ev_taken) cudaEventDestroy(c->ev_taken);
  if (c->stage) cudaFree(c->stage);
  void *pm[] = {c->pm_D, c->pm_wb, c->pm_tab[0], c->pm_tab[1], c->pm_xs, c->pm_gh};
  for (void *p : pm)
    if (p) cudaFree(p);
}

namespace w2 {
namespace {
std::atomic<long long> g_alloc_fail_in{-1};  // allocations before the injected failure; -1: off
std::atomic<long long> g_alloc_count{0};

bool injected_alloc_failure() {
  g_alloc_count.fetch_add(1);
  long long v = g_alloc_fail_in.load();
  while (v >= 0)
    if (g_alloc_fail_in.compare_exchange_weak(v, v - 1)) return v == 0;
  return false;
}
}  // namespace

cudaError_t dev_alloc(void **p, size_t bytes) {
  if (injected_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t host_alloc(void **p, size_t bytes) {
  if (injected_alloc_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(p, bytes);
}
}  // namespace w2

extern "C" w2_status w2_debug_fail_alloc(int32_t n) {
  w2::g_alloc_fail_in.store(n < 0 ? -1 : (long long)n);
  return W2_OK;
}

extern "C" int64_t w2_debug_alloc_count(void) { return (int64_t)w2::g_alloc_count.load(); }

extern "C" const char *w2_status_string(w2_status s) {
  switch (s) {
    case W2_OK: return "ok";
    case W2_ERR_ARG: return "invalid argument";
    case W2_ERR_CUDA: return "CUDA error";
    case W2_ERR_OOM: return "out of memory";
    case W2_ERR_STATE: return "call order violated";
    case W2_ERR_UNSTABLE: return "time step unstable for these potentials";
    case W2_ERR_NONFINITE: return "non-finite value in state";
    case W2_ERR_TIMEOUT: return "device wait timed out";
    case W2_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

extern "C" void w2_destroy(w2_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
}

// Spline shift tables: the foot of the characteristic of momentum p_n lies
// s = tau p_n / (m dx) cells behind each grid point; with k0 = floor(-s) and
// theta = -s - k0 the value is sum_{a=-1..2} eta_{i+k0+a} b_a(theta) (the
// four B-spline pieces of Sec. 4.1 on [0, 1)), eta = -6 z d.
// v as a double-float pair (hi = v rounded to FP32, lo = the rest rounded).
static float2 split_df(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

static void spline_tables(const w2_ctx *c, std::vector<int> &k0, std::vector<double> &w) {
  k0.resize(c->nk);
  w.resize(4 * c->nk);
  for (int n = 0; n < c->nk; ++n) {
    const double p = (n - c->nk / 2) * c->dp;
    const double s = c->tau * p / (c->cfg.mass * c->dx);
    const double fl = floor(-s);
    const double th = -s - fl;
    k0[n] = (int)fl;
    const double b[4] = {(1 - th) * (1 - th) * (1 - th) / 6.0, (3 * th * th * th - 6 * th * th + 4) / 6.0,
                         (-3 * th * th * th + 3 * th * th + 3 * th + 1) / 6.0, th * th * th / 6.0};
    for (int a = 0; a < 4; ++a) w[4 * n + a] = -6.0 * c->z * b[a];
  }
}

extern "C" w2_status w2_create(const w2_config *cfg, void *cuda_stream, w2_ctx **out) {
  if (!out) return W2_ERR_ARG;
  *out = nullptr;
  if (!cfg) return W2_ERR_ARG;
  if (cfg->nx < 4 || cfg->nx > 1024 || cfg->nk < 2 || (cfg->nk & 1) || !(cfg->L > 0) || !(cfg->dt > 0) ||
      !(cfg->hbar > 0) || !(cfg->mass > 0) || !isfinite(cfg->L) || !isfinite(cfg->dt) ||
      cfg->xc_kind < 0 || cfg->xc_kind > 2)
    return W2_ERR_ARG;
  if (cfg->precision != W2_F64 && cfg->precision != W2_F32_TF32X3 && cfg->precision != W2_F32_BF16X3 &&
      cfg->precision != W2_F64_SLICED)
    return W2_ERR_UNSUPPORTED;
  if (cfg->precision == W2_F64 && (!nk_supported_f64(cfg->nk) || cfg->nx > 128)) return W2_ERR_UNSUPPORTED;
  if (cfg->precision == W2_F64_SLICED && (!nk_supported_f64s(cfg->nk) || cfg->nx > 128)) return W2_ERR_UNSUPPORTED;
  if ((cfg->precision == W2_F32_TF32X3 || cfg->precision == W2_F32_BF16X3) &&
      (!nk_supported_f32(cfg->nk) || cfg->nx > 256))
    return W2_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return W2_ERR_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return W2_ERR_CUDA;
  if (prop.major < 10) return W2_ERR_CUDA;

  w2_ctx *ctx = new (std::nothrow) w2_ctx();
  if (!ctx) return W2_ERR_OOM;
  memset(ctx, 0, sizeof(*ctx));
  ctx->cfg = *cfg;
  ctx->stream = (cudaStream_t)cuda_stream;
  ctx->dev = dev;
  ctx->prec = cfg->precision;
  ctx->esz = f64_state(cfg->precision) ? sizeof(double) : sizeof(float);
  ctx->nx = cfg->nx;
  ctx->nk = cfg->nk;
  ctx->M = 2 * cfg->nk;
  ctx->npts = (size_t)cfg->nx * cfg->nx * cfg->nk * cfg->nk;
  ctx->dx = cfg->L / cfg->nx;
  ctx->dp = M_PI * cfg->hbar / cfg->L;
  ctx->hp = cfg->L / ctx->M;
  ctx->tau = cfg->dt;
  ctx->z = sqrt(3.0) - 2.0;
  // periodic start sums: |z|^k below the storage precision (z^32 ~ 5e-19, z^16 ~ 7e-10)
  const int kmax = f64_state(cfg->precision) ? 32 : 16;
  ctx->nterm = ctx->nx <= kmax ? ctx->nx : kmax;
  ctx->np_ax[0] = ctx->np_ax[1] = 1;
  ctx->zscale = (ctx->nterm == ctx->nx) ? 1.0 / (1.0 - pow(ctx->z, ctx->nx)) : 1.0;

  const int nx = ctx->nx, nk = ctx->nk, M = ctx->M, W = 2 * nk - 1;
  cudaError_t e = cudaSuccess;
#define W2_ALLOC(ptr, bytes)                                  \
  if (e == cudaSuccess) e = dev_alloc((void **)&(ptr), (bytes));
  const size_t fb = ctx->esz * ctx->npts;
  W2_ALLOC(ctx->f, fb) W2_ALLOC(ctx->g, fb) W2_ALLOC(ctx->t1, fb) W2_ALLOC(ctx->t2, fb)
  W2_ALLOC(ctx->xsum, sizeof(double) * nx * nx) W2_ALLOC(ctx->xsum2, sizeof(double) * nx * nx)
  W2_ALLOC(ctx->K, sizeof(double) * 2 * nx * W) W2_ALLOC(ctx->K12, sizeof(double) * nx * W)
  W2_ALLOC(ctx->vext_fine, sizeof(double) * nx * M) W2_ALLOC(ctx->w_fine, sizeof(double) * nx * M)
  W2_ALLOC(ctx->d_fine, sizeof(double) * nx * M) W2_ALLOC(ctx->sintab, sizeof(double) * M)
  W2_ALLOC(ctx->vext_grid, sizeof(double) * nx) W2_ALLOC(ctx->k0tab, sizeof(int) * nk)
  W2_ALLOC(ctx->wtab, sizeof(double) * 4 * nk) W2_ALLOC(ctx->xpart, sizeof(double) * (nx * nx * (3 + nk) + 8 * nx))
  W2_ALLOC(ctx->obs_out, sizeof(double) * (8 + nx + nx * nx))
  W2_ALLOC(ctx->wtab32, sizeof(float) * 4 * nk) W2_ALLOC(ctx->ctab32, sizeof(float) * 8 * nk)
  W2_ALLOC(ctx->wdf, sizeof(float2) * 4 * nk) W2_ALLOC(ctx->zpow, sizeof(float2) * 32)
  W2_ALLOC(ctx->d_err, sizeof(int))
  if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
#undef W2_ALLOC
  if (e == cudaSuccess) e = host_alloc((void **)&ctx->h_obs, sizeof(double) * (8 + nx + nx * nx));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = f64_state(ctx->prec) ? prepare_kernels_f64(nk) : prepare_kernels_f32(nk);
  if (e == cudaSuccess && ctx->prec == W2_F32_BF16X3) e = prepare_kernels_b3(nk);
  if (e == cudaSuccess && ctx->prec == W2_F64_SLICED) e = prepare_kernels_f64s(nk);
  if (e == cudaSuccess && ctx->prec == W2_F64_SLICED && nk == 64) e = prepare_kernels_f64t();
  if (e == cudaSuccess && ctx->prec == W2_F64_SLICED) e = prepare_kernels_adv_df(nk);
  if (e != cudaSuccess) {
    w2_status st = (e == cudaErrorMemoryAllocation) ? W2_ERR_OOM : W2_ERR_CUDA;
    cudaGetLastError();
    free_all(ctx);
    delete ctx;
    return st;
  }
  std::vector<double> sint(M);
  for (int m = 0; m < M; ++m) sint[m] = sin(M_PI * (double)m / nk);
  std::vector<int> k0;
  std::vector<double> wt;
  spline_tables(ctx, k0, wt);
  e = cudaMemcpy(ctx->sintab, sint.data(), sizeof(double) * M, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->k0tab, k0.data(), sizeof(int) * nk, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->wtab, wt.data(), sizeof(double) * 4 * nk, cudaMemcpyHostToDevice);
  // FP32 tables: weights, and the taps of (S - I) merged over offsets -3..3
  // (evaluation weights at k0 + a, a = -1..2, plus z (1, 4, 1) at -1, 0, 1,
  // since f_i = -z (d_{i-1} + 4 d_i + d_{i+1})), usable when k0 in [-2, 1].
  std::vector<float> w32(4 * nk), c32(8 * nk, 0.0f);
  for (int n = 0; n < nk; ++n) {
    for (int q = 0; q < 4; ++q) w32[4 * n + q] = (float)wt[4 * n + q];
    const int k0n = k0[n];
    for (int o = -3; o <= 3; ++o) {
      double t = 0.0;
      const int a = o - k0n;  // weight index a in [-1, 2]
      if (a >= -1 && a <= 2) t += wt[4 * n + a + 1];
      if (o == -1 || o == 1) t += ctx->z;
      if (o == 0) t += 4.0 * ctx->z;
      c32[8 * n + o + 3] = (float)t;
    }
    c32[8 * n + 7] = (k0n >= -2 && k0n <= 1) ? 1.0f : 0.0f;
  }
  if (e == cudaSuccess) e = cudaMemcpy(ctx->wtab32, w32.data(), sizeof(float) * 4 * nk, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->ctab32, c32.data(), sizeof(float) * 8 * nk, cudaMemcpyHostToDevice);
  // double-float tables of the sliced path
  std::vector<float2> wdf(4 * nk), zpow(32);
  for (int q = 0; q < 4 * nk; ++q) wdf[q] = split_df(wt[q]);
  for (int k = 0; k < 32; ++k) zpow[k] = split_df(pow(ctx->z, k));
  if (e == cudaSuccess) e = cudaMemcpy(ctx->wdf, wdf.data(), sizeof(float2) * 4 * nk, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->zpow, zpow.data(), sizeof(float2) * 32, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_all(ctx);
    delete ctx;
    return W2_ERR_CUDA;
  }
  *out = ctx;
  return W2_OK;
}

TabArgs w2::tab_args(w2_ctx *ctx, const double *xsum, int pair_mode) {
  TabArgs a;
  a.nx = ctx->nx;
  a.nk = ctx->nk;
  a.M = ctx->M;
  a.dx = ctx->dx;
  a.dp = ctx->dp;
  a.hbar = ctx->cfg.hbar;
  a.gamma = ctx->gamma;
  a.c_h = ctx->c_h;
  a.c_xc = ctx->c_xc;
  a.xc_kind = ctx->cfg.xc_kind;
  a.pair_mode = pair_mode;
  a.xsum = xsum;
  a.vext_fine = ctx->vext_fine;
  a.w_fine = ctx->w_fine;
  a.d_fine = ctx->d_fine;
  a.sintab = ctx->sintab;
  a.K = pair_mode ? ctx->K12 : ctx->K;
  a.h_fine = ctx->hartree_kind == W2_HARTREE_POISSON ? ctx->h_fine : nullptr;
  return a;
}

extern "C" w2_status w2_set_hartree(w2_ctx *ctx, int32_t kind) {
  if (!ctx || (kind != W2_HARTREE_PAIR && kind != W2_HARTREE_POISSON)) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  const int nx = ctx->nx, M = ctx->M;
  if (kind == W2_HARTREE_POISSON) {
    // G(r) = (1/N_x) [2 sum_{0 < m < N_x/2} cos(k_m r)/k_m^2 + cos(k_{N_x/2} r)/k_{N_x/2}^2 (N_x even)],
    // k_m = 2 pi m / L, at r = d dx + l h'
    std::vector<double> g((size_t)nx * M);
    const double L = ctx->cfg.L;
    for (int d = 0; d < nx; ++d)
      for (int l = 0; l < M; ++l) {
        const double r = d * ctx->dx + l * ctx->hp;
        double v = 0.0;
        for (int m = 1; 2 * m < nx; ++m) {
          const double k = 2.0 * M_PI * m / L;
          v += 2.0 * cos(k * r) / (k * k);
        }
        if (nx % 2 == 0) {
          const double k = M_PI * nx / L;
          v += cos(k * r) / (k * k);
        }
        g[(size_t)d * M + l] = v / nx;
      }
    if (!ctx->h_fine && dev_alloc((void **)&ctx->h_fine, sizeof(double) * nx * M) != cudaSuccess) return W2_ERR_OOM;
    W2_TRY(cudaMemcpy(ctx->h_fine, g.data(), sizeof(double) * nx * M, cudaMemcpyHostToDevice));
  }
  ctx->hartree_kind = kind;
  drop_graphs(ctx);
  return W2_OK;
}

extern "C" w2_status w2_set_potentials(w2_ctx *ctx, w2_fn vext, void *ue, w2_fn vee, void *ui, double gamma,
                                       double c_hartree, double c_xc) {
  if (!ctx) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!isfinite(gamma) || !isfinite(c_hartree) || !isfinite(c_xc)) return W2_ERR_ARG;
  const int nx = ctx->nx, M = ctx->M, nk = ctx->nk;
  const double L = ctx->cfg.L;
  std::vector<double> vf(nx * M), wf(nx * M), df(nx * M, 0.0), vg(nx);
  for (int i = 0; i < nx; ++i) {
    const double xi = -0.5 * L + i * ctx->dx;
    vg[i] = vext ? vext(fold(xi, L), ue) : 0.0;
    for (int l = 0; l < M; ++l) {
      vf[i * M + l] = vext ? vext(fold(xi + l * ctx->hp, L), ue) : 0.0;
      wf[i * M + l] = vee ? vee(fold(i * ctx->dx + l * ctx->hp, L), ui) : 0.0;
      if (!isfinite(vf[i * M + l]) || !isfinite(wf[i * M + l])) return W2_ERR_ARG;
      // trigonometric interpolation weight of the grid density at offset
      // t = d dx + l h' (Nyquist mode halved for even nx)
      if (c_xc != 0.0 && ctx->cfg.xc_kind) {
        const double t = i * ctx->dx + l * ctx->hp;
        double s = 1.0;
        const int half = nx / 2;
        for (int m = 1; m <= (nx - 1) / 2; ++m) s += 2.0 * cos(2.0 * M_PI * m * t / L);
        if (nx % 2 == 0) s += cos(2.0 * M_PI * half * t / L);
        df[i * M + l] = s / nx;
      }
    }
    if (!isfinite(vg[i])) return W2_ERR_ARG;
  }
  // Stability precheck: Theta is skew per X with spectrum inside
  // i [-smax, smax], smax = (1/hbar)(2 max|dV_ext| + gamma max|dW| + Hartree bound).
  double dvmax = 0.0, dwmax = 0.0, wmin = 1e300, wmax = -1e300;
  for (int i = 0; i < nx; ++i)
    for (int l = 1; l < nk; ++l) {
      dvmax = fmax(dvmax, fabs(vf[i * M + l] - vf[i * M + M - l]));
      dwmax = fmax(dwmax, fabs(gamma * (wf[i * M + l] - wf[i * M + M - l])));
    }
  for (int k = 0; k < nx * M; ++k) {
    wmin = fmin(wmin, wf[k]);
    wmax = fmax(wmax, wf[k]);
  }
  // (the neutralised Poisson Hartree term depends on the state's density and
  // has no a-priori bound here; it is left out of the precheck)
  const double hart = ctx->hartree_kind == W2_HARTREE_POISSON ? 0.0 : 2.0 * fabs(c_hartree) * fabs(gamma) * (wmax - wmin);
  const double y = ctx->tau / ctx->cfg.hbar * (2.0 * dvmax + dwmax + hart);
  if (!(y <= 1.0)) return W2_ERR_UNSTABLE;

  W2_TRY(cudaMemcpyAsync(ctx->vext_fine, vf.data(), sizeof(double) * nx * M, cudaMemcpyHostToDevice, ctx->stream));
  W2_TRY(cudaMemcpyAsync(ctx->w_fine, wf.data(), sizeof(double) * nx * M, cudaMemcpyHostToDevice, ctx->stream));
  W2_TRY(cudaMemcpyAsync(ctx->d_fine, df.data(), sizeof(double) * nx * M, cudaMemcpyHostToDevice, ctx->stream));
  W2_TRY(cudaMemcpyAsync(ctx->vext_grid, vg.data(), sizeof(double) * nx, cudaMemcpyHostToDevice, ctx->stream));
  ctx->gamma = gamma;
  ctx->c_h = c_hartree;
  ctx->c_xc = c_xc;
  TabArgs a = tab_args(ctx, nullptr, 1);
  W2_TRY(launch_tables(a, ctx->stream));
  // host vectors are copied by cudaMemcpyAsync from pageable memory before return
  W2_TRY(cudaStreamSynchronize(ctx->stream));
  ctx->have_pot = true;
  drop_graphs(ctx);
  return W2_OK;
}

// The per-X sums of a new state (the time step takes those of f^n from here
// or from the previous step's corrector).
cudaError_t w2::state_sums(w2_ctx *ctx, cudaStream_t s) {
  return f64_state(ctx->prec) ? launch_xsum_f64(ctx->nx, ctx->nk, (const double *)ctx->f, ctx->xsum, s)
                              : launch_xsum_f32(ctx->nx, ctx->nk, (const float *)ctx->f, ctx->xsum, s);
}

extern "C" w2_status w2_set_state(w2_ctx *ctx, const void *f, int32_t on_device) {
  if (!ctx || !f) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot) return W2_ERR_STATE;
  W2_TRY(cudaMemcpyAsync(ctx->f, f, ctx->esz * ctx->npts,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  W2_TRY(state_sums(ctx, ctx->stream));
  W2_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));  // a new state starts without a time-out
  ctx->have_state = true;
  ctx->steps = 0;
  return W2_OK;
}

extern "C" w2_status w2_stage_state(w2_ctx *ctx, const void *f) {
  if (!ctx || !f) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot) return W2_ERR_STATE;
  const size_t bytes = ctx->esz * ctx->npts;
  if (!ctx->stage) {
    if (dev_alloc(&ctx->stage, bytes) != cudaSuccess) {
      ctx->stage = nullptr;
      (void)cudaGetLastError();
      return W2_ERR_OOM;
    }
    W2_TRY(cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking));
    W2_TRY(cudaEventCreateWithFlags(&ctx->ev_staged, cudaEventDisableTiming));
    W2_TRY(cudaEventCreateWithFlags(&ctx->ev_taken, cudaEventDisableTiming));
  }
  // the stage is overwritten only after the previous w2_use_staged_state has read it
  if (ctx->taken_recorded) W2_TRY(cudaStreamWaitEvent(ctx->copy, ctx->ev_taken, 0));
  W2_TRY(cudaMemcpyAsync(ctx->stage, f, bytes, cudaMemcpyHostToDevice, ctx->copy));
  W2_TRY(cudaEventRecord(ctx->ev_staged, ctx->copy));
  ctx->stage_pending = true;
  return W2_OK;
}

extern "C" w2_status w2_use_staged_state(w2_ctx *ctx) {
  if (!ctx) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->stage_pending) return W2_ERR_STATE;
  W2_TRY(cudaStreamWaitEvent(ctx->stream, ctx->ev_staged, 0));
  // no copy: the staged buffer becomes the state, and the old state buffer
  // takes the next staged copy once the work queued on it so far is done
  // (ev_taken; the step graph for each buffer is captured once)
  void *staged = ctx->stage;
  ctx->stage = ctx->f;
  ctx->f = static_cast<double *>(staged);
  W2_TRY(cudaEventRecord(ctx->ev_taken, ctx->stream));
  W2_TRY(state_sums(ctx, ctx->stream));
  W2_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));  // a new state starts without a time-out
  ctx->taken_recorded = true;
  ctx->stage_pending = false;
  ctx->have_state = true;
  ctx->steps = 0;
  return W2_OK;
}

extern "C" w2_status w2_set_tensor_path(w2_ctx *ctx, int32_t tcgen05) {
  if (!ctx || (tcgen05 != 0 && tcgen05 != 1)) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (tcgen05 && ctx->prec != W2_F64_SLICED) return W2_ERR_UNSUPPORTED;
  if (ctx->tc_path != (tcgen05 != 0)) drop_graphs(ctx);
  ctx->tc_path = tcgen05 != 0;
  return W2_OK;
}

extern "C" w2_status w2_debug_sweep_stall(w2_ctx *ctx, int32_t stall, int64_t wait_cycles) {
  if (!ctx || (stall != 0 && stall != 1) || wait_cycles < 0) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  drop_graphs(ctx);
  ctx->dbg_stall = stall;
  ctx->dbg_wait = wait_cycles;
  if (!stall) W2_TRY(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  return W2_OK;
}

extern "C" w2_status w2_set_exchange_symmetry(w2_ctx *ctx, int32_t on) {
  if (!ctx || (on != 0 && on != 1)) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (on && ctx->prec != W2_F64_SLICED) return W2_ERR_UNSUPPORTED;
  if (ctx->exchange_sym != (on != 0)) drop_graphs(ctx);
  ctx->exchange_sym = on != 0;
  return W2_OK;
}

extern "C" w2_status w2_get_state(w2_ctx *ctx, void *f, int32_t on_device) {
  if (!ctx || !f) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_state) return W2_ERR_STATE;
  W2_TRY(cudaMemcpyAsync(f, ctx->f, ctx->esz * ctx->npts,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  if (!on_device) W2_TRY(cudaStreamSynchronize(ctx->stream));
  return W2_OK;
}

// Slope stencil half-width of the patch decomposition: |z|^26 < 2^-52.
static const int kPatchStencil = 26;

extern "C" w2_status w2_set_patches(w2_ctx *ctx, int32_t np1, int32_t np2) {
  if (!ctx || np1 < 1 || np2 < 1) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (ctx->prec != W2_F64) return W2_ERR_UNSUPPORTED;
  const int nx = ctx->nx, nk = ctx->nk, nnb = kPatchStencil;
  std::vector<int> k0;
  std::vector<double> wt;
  spline_tables(ctx, k0, wt);
  int G = 1;
  for (int n = 0; n < nk; ++n) G = std::max(G, std::max(-k0[n], k0[n] + 1));
  const int nps[2] = {np1, np2};
  for (int ax = 0; ax < 2; ++ax)
    if (nps[ax] > 1 && (nx % nps[ax] != 0 || nx / nps[ax] < G + nnb)) return W2_ERR_UNSUPPORTED;
  void *pm[] = {ctx->pm_D, ctx->pm_wb, ctx->pm_tab[0], ctx->pm_tab[1], ctx->pm_xs, ctx->pm_gh};
  for (void *p : pm)
    if (p) cudaFree(p);
  ctx->pm_D = ctx->pm_wb = ctx->pm_tab[0] = ctx->pm_tab[1] = ctx->pm_xs = ctx->pm_gh = nullptr;
  ctx->np_ax[0] = np1;
  ctx->np_ax[1] = np2;
  ctx->pm_G = G;
  drop_graphs(ctx);
  if (np1 == 1 && np2 == 1) return W2_OK;
  // slope of the periodic spline at a point from the samples: the inverse of
  // the (1,4,1)/6 circulant is beta_m = sqrt(3) (z^m + z^(nx-m)) / (1 - z^nx),
  // and D_j = (beta_{j-1} - beta_{j+1}) / (2 dx)
  const double z = ctx->z, zn = pow(z, nx);
  auto beta = [&](int m) {
    m %= nx;
    m += (m < 0) ? nx : 0;
    return sqrt(3.0) * (pow(z, m) + pow(z, nx - m)) / (1.0 - zn);
  };
  std::vector<double> D(2 * nnb + 1), wb(4 * nk);
  for (int j = -nnb; j <= nnb; ++j) D[j + nnb] = (beta(j - 1) - beta(j + 1)) / (2.0 * ctx->dx);
  for (int q = 0; q < 4 * nk; ++q) wb[q] = wt[q] / (-6.0 * z);  // the plain B-spline weights b_a(theta)
  const size_t lines = (size_t)nx * nk * nk;
  const int npmax = std::max(np1, np2);
  cudaError_t e = dev_alloc((void **)&ctx->pm_D, sizeof(double) * D.size());
  if (e == cudaSuccess) e = dev_alloc((void **)&ctx->pm_wb, sizeof(double) * wb.size());
  if (e == cudaSuccess) e = dev_alloc((void **)&ctx->pm_xs, sizeof(double) * 2 * npmax * 2 * lines);
  if (e == cudaSuccess) e = dev_alloc((void **)&ctx->pm_gh, sizeof(double) * 2 * npmax * 2 * G * lines);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->pm_D, D.data(), sizeof(double) * D.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ctx->pm_wb, wb.data(), sizeof(double) * wb.size(), cudaMemcpyHostToDevice);
  for (int ax = 0; ax < 2 && e == cudaSuccess; ++ax) {
    if (nps[ax] < 2) continue;
    // Thomas factors of the (4,2), (1,4,1), (2,4) system on n = M + 2G points
    const int n = nx / nps[ax] + 2 * G;
    std::vector<double> tab(2 * n);  // inv_m [n], then c' [n]
    double cprev = 0.0;
    for (int v = 0; v < n; ++v) {
      const double a = v == 0 ? 0.0 : (v == n - 1 ? 2.0 : 1.0), c = v == 0 ? 2.0 : 1.0;
      const double m = 4.0 - a * cprev;
      tab[v] = 1.0 / m;
      tab[n + v] = cprev = (v < n - 1) ? c / m : 0.0;
    }
    e = dev_alloc((void **)&ctx->pm_tab[ax], sizeof(double) * tab.size());
    if (e == cudaSuccess) e = cudaMemcpy(ctx->pm_tab[ax], tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->np_ax[0] = ctx->np_ax[1] = 1;
    return e == cudaErrorMemoryAllocation ? W2_ERR_OOM : W2_ERR_CUDA;
  }
  return W2_OK;
}

// One FP64 shift pass (DIR 0: x2 lines, DIR 1: x1 lines), through the patch
// decomposition when the context has one on that axis.
static cudaError_t shift_pass64(const w2_ctx *ctx, int dir, int two, const double *in0, const double *in1,
                                double *out0, double *out1, cudaStream_t s) {
  const int np = ctx->np_ax[dir == 1 ? 0 : 1];
  if (np > 1) {
    PatchArgs pa;
    pa.nx = ctx->nx;
    pa.np = np;
    pa.M = ctx->nx / np;
    pa.G = ctx->pm_G;
    pa.nnb = kPatchStencil;
    pa.in0 = in0;
    pa.in1 = in1;
    pa.out0 = out0;
    pa.out1 = out1;
    pa.xs = ctx->pm_xs;
    pa.gh = ctx->pm_gh;
    pa.D = ctx->pm_D;
    const double *tab = ctx->pm_tab[dir == 1 ? 0 : 1];
    pa.inv_m = tab;
    pa.cp = tab + pa.M + 2 * pa.G;
    pa.k0tab = ctx->k0tab;
    pa.wb = ctx->pm_wb;
    pa.h = ctx->dx;
    pa.tau = ctx->tau;
    return launch_adv_pmbc(ctx->nk, dir, two, pa, s);
  }
  AdvArgs av;
  av.nx = ctx->nx;
  av.k0tab = ctx->k0tab;
  av.wtab = ctx->wtab;
  av.z = ctx->z;
  av.zscale = ctx->zscale;
  av.nterm = ctx->nterm;
  av.tau = ctx->tau;
  av.in0 = in0;
  av.in1 = in1;
  av.out0 = out0;
  av.out1 = out1;
  return launch_adv_f64(ctx->nk, dir, two, av, s);
}

static AdvDFArgs adv_df_args(const w2_ctx *ctx) {
  AdvDFArgs a;
  memset(&a, 0, sizeof(a));
  a.nx = ctx->nx;
  a.k0tab = ctx->k0tab;
  a.wdf = ctx->wdf;
  a.zpow = ctx->zpow;
  a.z = split_df(ctx->z);
  a.zscale = split_df(ctx->zscale);
  a.tau = split_df(ctx->tau);
  a.half_tau = split_df(0.5 * ctx->tau);
  a.nterm = ctx->nterm;
  return a;
}

// Optional per-kernel CUDA events around every launch of a step (profiling).
struct StepEvents {
  cudaEvent_t *ev;  // [2 * W2_STEP_KERNELS] or null
};

#define W2_MARK(k, pos)                                                             \
  if (evs && evs->ev) {                                                             \
    if ((e = cudaEventRecord(evs->ev[2 * (k) + (pos)], s)) != cudaSuccess) return e; \
  }

// Feature rows of every spatial point of `f` into ctx->xrows (learned form).
static cudaError_t enqueue_features(w2_ctx *ctx, const void *f, cudaStream_t s) {
  FeatArgs fa;
  fa.nx = ctx->nx;
  fa.nk = ctx->nk;
  fa.din = mlp_din(ctx->mlp);
  fa.dx = ctx->dx;
  fa.dp = ctx->dp;
  fa.s_f = mlp_scale(ctx->mlp, 0);
  fa.s_f1 = mlp_scale(ctx->mlp, 1);
  fa.f1 = ctx->f1;
  fa.f1_src_rows = 1;
  fa.xs = nullptr;
  fa.x = ctx->xrows;
  return launch_features(fa, f, f64_state(ctx->prec), ctx->nx * ctx->nx, s);
}

// The network's two-body term of `f` (in operator units) into the MLP output buffer.
static cudaError_t enqueue_learned_pair(w2_ctx *ctx, const void *f, cudaStream_t s) {
  cudaError_t e = enqueue_features(ctx, f, s);
  if (e != cudaSuccess) return e;
  return mlp_forward(ctx->mlp, ctx->xrows, ctx->nx * ctx->nx, mlp_out(ctx->mlp), 1.0f / mlp_scale(ctx->mlp, 2), s);
}

// One Lawson step on stream s (see w2.h):
//   xsum(f^n) ; K(f^n) ; g = Theta f^n ; (t1, t2) = A_x2 (f, g) ;
//   (f~ -> g, h -> f) = A_x1 (t1, t2) ; xsum(f~) ; K(f~) ; f = h + tau/2 Theta f~
static cudaError_t enqueue_step(w2_ctx *ctx, cudaStream_t s, const StepEvents *evs = nullptr) {
  const int nx = ctx->nx, nk = ctx->nk, W = 2 * nk - 1;
  cudaError_t e;
  TabArgs ta = tab_args(ctx, ctx->xsum, 0);
  // the per-X sums of f^n come from the previous step's corrector or from the
  // state's set-up; both are the same exact fixed-point sums, so a state
  // restored with w2_set_state continues bit-identically
  W2_MARK(0, 0)
  W2_MARK(0, 1)
  W2_MARK(1, 0)
  if ((e = launch_tables(ta, s)) != cudaSuccess) return e;
  W2_MARK(1, 1)
  ThetaArgs th;
  th.nx = nx;
  th.in = ctx->f;
  th.h = nullptr;
  th.out = ctx->g;
  th.xsum = nullptr;
  th.K1 = ctx->K;
  th.K2 = ctx->K + (size_t)nx * W;
  th.K12 = ctx->K12;
  th.half_tau = 0.5 * ctx->tau;
  const bool learned = ctx->mlp && ctx->learned_active;
  const bool learned_kernel = learned && mlp_kind(ctx->mlp) == 1;
  // the network's pair table need not be odd in x1 - x2: no mirrored blocks with it
  th.sym = ctx->exchange_sym && ctx->prec == W2_F64_SLICED && !learned;
  if (learned_kernel) {
    th.K12 = ctx->Klearn;  // the network's pair table, built when it was attached
  } else if (learned) {
    if ((e = enqueue_learned_pair(ctx, ctx->f, s)) != cudaSuccess) return e;
    th.pair = mlp_out(ctx->mlp);
  }
  W2_MARK(2, 0)
  if ((e = theta64(ctx, 0, th, s)) != cudaSuccess) return e;
  W2_MARK(2, 1)
  AdvDFArgs ad = adv_df_args(ctx);  // the sliced path: pairs in t1, t2
  ad.in0 = ctx->f;
  ad.in1 = ctx->g;
  ad.out0 = ctx->t1;
  ad.out1 = ctx->t2;
  const bool df = ctx->prec == W2_F64_SLICED;
  W2_MARK(3, 0)
  if ((e = df ? launch_adv_df(nk, 0, 1, ad, s) : shift_pass64(ctx, 0, 1, ctx->f, ctx->g, ctx->t1, ctx->t2, s)) !=
      cudaSuccess)
    return e;
  W2_MARK(3, 1)
  // x1 pass: f~ -> g, h -> f
  ad.in0 = ctx->t1;
  ad.in1 = ctx->t2;
  ad.out0 = ctx->g;
  ad.out1 = ctx->f;
  W2_MARK(4, 0)
  if ((e = df ? launch_adv_df(nk, 1, 1, ad, s) : shift_pass64(ctx, 1, 1, ctx->t1, ctx->t2, ctx->g, ctx->f, s)) !=
      cudaSuccess)
    return e;
  W2_MARK(4, 1)
  W2_MARK(5, 0)
  if ((e = launch_xsum_f64(nx, nk, ctx->g, ctx->xsum, s)) != cudaSuccess) return e;
  W2_MARK(5, 1)
  W2_MARK(6, 0)
  if ((e = launch_tables(ta, s)) != cudaSuccess) return e;
  W2_MARK(6, 1)
  th.in = ctx->g;
  th.h = ctx->f;
  th.out = ctx->f;
  th.xsum = ctx->xsum;  // the per-X sums of f^{n+1}, for the next step
  if (learned && !learned_kernel && (e = enqueue_learned_pair(ctx, ctx->g, s)) != cudaSuccess) return e;
  W2_MARK(7, 0)
  if ((e = theta64(ctx, 1, th, s)) != cudaSuccess) return e;
  W2_MARK(7, 1)
  return cudaSuccess;
}

Adv32Args w2::adv32_args(w2_ctx *ctx) {
  Adv32Args a;
  memset(&a, 0, sizeof(a));
  a.nx = ctx->nx;
  a.k0tab = ctx->k0tab;
  a.wtab = ctx->wtab32;
  a.ctab = ctx->ctab32;
  a.z = (float)ctx->z;
  a.zscale = (float)ctx->zscale;
  a.nterm = ctx->nterm;
  a.tau = (float)ctx->tau;
  a.nterm_df = ctx->nx <= 28 ? ctx->nx : 28;
  a.zdf = split_df(ctx->z);
  a.zscale_df = split_df(a.nterm_df == ctx->nx ? 1.0 / (1.0 - pow(ctx->z, ctx->nx)) : 1.0);
  a.zpow = ctx->zpow;
  return a;
}

// FP32 precision form of the same step (arrays hold floats):
//   K(f) ; g = Theta f ; (d2 -> t1, g2 -> t2) = A_x2 ;
//   (f~ -> g, dh -> t1) = A_x1 ; xsum(f~) ; K(f~) ; f = f + (dh + tau/2 Theta f~), xsum(f)
// (the per-X sums of f^n come from the previous corrector or from the state's set-up)
static cudaError_t enqueue_step32(w2_ctx *ctx, cudaStream_t s, const StepEvents *evs) {
  const int nx = ctx->nx, nk = ctx->nk, W = 2 * nk - 1;
  float *f = (float *)ctx->f, *g = (float *)ctx->g, *t1 = (float *)ctx->t1, *t2 = (float *)ctx->t2;
  cudaError_t e;
  TabArgs ta = tab_args(ctx, ctx->xsum, 0);
  W2_MARK(0, 0)
  W2_MARK(0, 1)
  W2_MARK(1, 0)
  if ((e = launch_tables(ta, s)) != cudaSuccess) return e;
  W2_MARK(1, 1)
  Theta32Args th;
  th.nx = nx;
  th.in = f;
  th.base = nullptr;
  th.h = nullptr;
  th.out = g;
  th.K1 = ctx->K;
  th.K2 = ctx->K + (size_t)nx * W;
  th.K12 = ctx->K12;
  th.half_tau = (float)(0.5 * ctx->tau);
  W2_MARK(2, 0)
  if ((e = theta32(ctx, 0, th, s)) != cudaSuccess) return e;
  W2_MARK(2, 1)
  Adv32Args av = adv32_args(ctx);
  av.f = f;
  av.g = g;
  av.d2 = t1;
  av.g2 = t2;
  W2_MARK(3, 0)
  if ((e = launch_adv_f32(nk, 0, av, s)) != cudaSuccess) return e;
  W2_MARK(3, 1)
  av.d2in = t1;
  av.g2in = t2;
  av.ft = g;
  av.dh = t1;
  W2_MARK(4, 0)
  if ((e = launch_adv_f32(nk, 1, av, s)) != cudaSuccess) return e;
  W2_MARK(4, 1)
  W2_MARK(5, 0)
  if ((e = launch_xsum_f32(nx, nk, g, ctx->xsum, s)) != cudaSuccess) return e;
  W2_MARK(5, 1)
  W2_MARK(6, 0)
  if ((e = launch_tables(ta, s)) != cudaSuccess) return e;
  W2_MARK(6, 1)
  th.in = g;
  th.base = f;
  th.h = t1;
  th.out = f;
  th.xsum = ctx->xsum;
  W2_MARK(7, 0)
  if ((e = theta32(ctx, 1, th, s)) != cudaSuccess) return e;
  W2_MARK(7, 1)
  return cudaSuccess;
}

static cudaError_t enqueue_any(w2_ctx *ctx, cudaStream_t s, const StepEvents *evs) {
  return f64_state(ctx->prec) ? enqueue_step(ctx, s, evs) : enqueue_step32(ctx, s, evs);
}

static w2_status learned_judge(w2_ctx *ctx);

static w2_status step_graph(w2_ctx *ctx, int32_t nsteps);

extern "C" w2_status w2_step(w2_ctx *ctx, int32_t nsteps) {
  if (!ctx || nsteps < 0) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot || !ctx->have_state) return W2_ERR_STATE;
  if (!(ctx->mlp && ctx->learned_active && ctx->judge_every > 0)) return step_graph(ctx, nsteps);
  // learned form: judge the network against the exact two-body term every
  // judge_every steps and fall back to the exact term when it is off
  int left = nsteps;
  while (left > 0) {
    const int k = std::min(left, ctx->judge_every - ctx->since_judge);
    w2_status st = step_graph(ctx, k);
    if (st != W2_OK) return st;
    left -= k;
    ctx->since_judge += k;
    if (ctx->since_judge >= ctx->judge_every) {
      ctx->since_judge = 0;
      st = learned_judge(ctx);
      if (st != W2_OK) return st;
      if (!ctx->learned_active) return left > 0 ? step_graph(ctx, left) : W2_OK;
    }
  }
  return W2_OK;
}

static w2_status step_graph(w2_ctx *ctx, int32_t nsteps) {
  if (nsteps == 0) return W2_OK;
  int k = -1;
  for (int q = 0; q < 2; ++q)
    if (ctx->graph_ok[q] && ctx->graph_f[q] == ctx->f) k = q;
  if (k < 0) {  // capture for this state buffer, in a free slot or over slot 1
    k = !ctx->graph_ok[0] ? 0 : 1;
    if (ctx->graph_ok[k]) {
      cudaGraphExecDestroy(ctx->graph[k]);
      ctx->graph_ok[k] = false;
    }
    cudaGraph_t graph;
    W2_TRY(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_any(ctx, ctx->cap, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (e2 == cudaSuccess) cudaGraphDestroy(graph);
      ctx->sticky = W2_ERR_CUDA;
      return W2_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&ctx->graph[k], graph, 0);
    cudaGraphDestroy(graph);
    W2_TRY(e);
    ctx->graph_ok[k] = true;
    ctx->graph_f[k] = ctx->f;
  }
  for (int s = 0; s < nsteps; ++s) W2_TRY(cudaGraphLaunch(ctx->graph[k], ctx->stream));
  ctx->steps += nsteps;
  return W2_OK;
}

// Queue the observables' reductions of the current state into ctx->obs_out.
static w2_status enqueue_obs(w2_ctx *ctx) {
  const int nx = ctx->nx;
  ObsArgs a;
  a.nx = nx;
  a.nk = ctx->nk;
  a.M = ctx->M;
  a.dx = ctx->dx;
  a.dp = ctx->dp;
  a.hbar = ctx->cfg.hbar;
  a.mass = ctx->cfg.mass;
  a.gamma = ctx->gamma;
  a.c_h = ctx->c_h;
  a.f = f64_state(ctx->prec) ? ctx->f : nullptr;
  a.f32 = f64_state(ctx->prec) ? nullptr : (const float *)ctx->f;
  a.vext_grid = ctx->vext_grid;
  a.w_fine = ctx->w_fine;
  a.h_fine = ctx->hartree_kind == W2_HARTREE_POISSON ? ctx->h_fine : nullptr;
  a.xpart = ctx->xpart;
  a.out = ctx->obs_out;
  a.err = ctx->d_err;
  W2_TRY(launch_obs(a, ctx->stream));
  return W2_OK;
}

// Unpack a host copy of obs_out.
static w2_status unpack_obs(const w2_ctx *ctx, const double *h, long long steps, w2_obs *out, double *n1,
                            double *n12) {
  const int nx = ctx->nx;
  out->mass = h[0];
  out->energy = h[1];
  out->purity = h[2];
  out->entropy_lin = 1.0 - h[2];
  out->l2norm = h[3];
  out->step = steps;
  if (n1) memcpy(n1, h + 8, sizeof(double) * nx);
  if (n12) memcpy(n12, h + 8 + nx, sizeof(double) * nx * nx);
  if (h[5] != 0.0) return W2_ERR_TIMEOUT;
  return h[4] != 0.0 ? W2_ERR_NONFINITE : W2_OK;
}

extern "C" w2_status w2_observables(w2_ctx *ctx, w2_obs *out, double *n1, double *n12) {
  if (!ctx || !out) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_state) return W2_ERR_STATE;
  w2_status st = enqueue_obs(ctx);
  if (st != W2_OK) return st;
  const size_t nb = sizeof(double) * (8 + ctx->nx + (size_t)ctx->nx * ctx->nx);
  W2_TRY(cudaMemcpyAsync(ctx->h_obs, ctx->obs_out, nb, cudaMemcpyDeviceToHost, ctx->stream));
  W2_TRY(cudaStreamSynchronize(ctx->stream));
  return unpack_obs(ctx, ctx->h_obs, ctx->steps, out, n1, n12);
}

extern "C" w2_status w2_observables_enqueue(w2_ctx *ctx, int32_t slot) {
  if (!ctx || slot < 0 || slot > 1) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_state) return W2_ERR_STATE;
  const size_t nb = sizeof(double) * (8 + ctx->nx + (size_t)ctx->nx * ctx->nx);
  if (!ctx->h_obs_slot[slot]) {
    if (host_alloc((void **)&ctx->h_obs_slot[slot], nb) != cudaSuccess) {
      ctx->h_obs_slot[slot] = nullptr;
      (void)cudaGetLastError();
      return W2_ERR_OOM;
    }
  }
  if (!ctx->ev_obs[slot]) W2_TRY(cudaEventCreateWithFlags(&ctx->ev_obs[slot], cudaEventDisableTiming));
  w2_status st = enqueue_obs(ctx);
  if (st != W2_OK) return st;
  W2_TRY(cudaMemcpyAsync(ctx->h_obs_slot[slot], ctx->obs_out, nb, cudaMemcpyDeviceToHost, ctx->stream));
  W2_TRY(cudaEventRecord(ctx->ev_obs[slot], ctx->stream));
  ctx->obs_pending[slot] = true;
  ctx->obs_steps[slot] = ctx->steps;
  return W2_OK;
}

extern "C" w2_status w2_observables_collect(w2_ctx *ctx, int32_t slot, w2_obs *out, double *n1, double *n12) {
  if (!ctx || !out || slot < 0 || slot > 1) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->obs_pending[slot]) return W2_ERR_STATE;
  W2_TRY(cudaEventSynchronize(ctx->ev_obs[slot]));
  ctx->obs_pending[slot] = false;
  return unpack_obs(ctx, ctx->h_obs_slot[slot], ctx->obs_steps[slot], out, n1, n12);
}

extern "C" w2_status w2_theta(w2_ctx *ctx, const void *f, void *out) {
  if (!ctx || !f || !out || f == out) return W2_ERR_ARG;
  // the sweep moves pairs of doubles / four floats: both arrays must be 16-byte aligned
  if (((uintptr_t)f | (uintptr_t)out) & 15) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot) return W2_ERR_STATE;
  const int nx = ctx->nx, nk = ctx->nk, W = 2 * nk - 1;
  if (f64_state(ctx->prec))
    W2_TRY(launch_xsum_f64(nx, nk, (const double *)f, ctx->xsum2, ctx->stream));
  else
    W2_TRY(launch_xsum_f32(nx, nk, (const float *)f, ctx->xsum2, ctx->stream));
  TabArgs ta = tab_args(ctx, ctx->xsum2, 0);
  W2_TRY(launch_tables(ta, ctx->stream));
  if (f64_state(ctx->prec)) {
    ThetaArgs th;
    th.nx = nx;
    th.in = (const double *)f;
    th.h = nullptr;
    th.out = (double *)out;
    th.xsum = nullptr;
    th.K1 = ctx->K;
    th.K2 = ctx->K + (size_t)nx * W;
    th.K12 = ctx->K12;
    th.half_tau = 0.5 * ctx->tau;
    W2_TRY(theta64(ctx, 0, th, ctx->stream));
  } else {
    Theta32Args th;
    th.nx = nx;
    th.in = (const float *)f;
    th.base = nullptr;
    th.h = nullptr;
    th.out = (float *)out;
    th.K1 = ctx->K;
    th.K2 = ctx->K + (size_t)nx * W;
    th.K12 = ctx->K12;
    th.half_tau = (float)(0.5 * ctx->tau);
    W2_TRY(theta32(ctx, 0, th, ctx->stream));
  }
  return W2_OK;
}

extern "C" w2_status w2_advect(w2_ctx *ctx, const void *f, void *out) {
  if (!ctx || !f || !out || f == out) return W2_ERR_ARG;
  // the FP32 shift stages its lines with 16-byte asynchronous copies
  if (!f64_state(ctx->prec) && (((uintptr_t)f | (uintptr_t)out) & 15)) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot) return W2_ERR_STATE;
  if (ctx->prec == W2_F64_SLICED) {
    AdvDFArgs ad = adv_df_args(ctx);
    ad.in0 = f;
    ad.out0 = ctx->t1;
    W2_TRY(launch_adv_df(ctx->nk, 1, 0, ad, ctx->stream));  // x1 first, into pairs
    ad.in0 = ctx->t1;
    ad.out0 = out;
    W2_TRY(launch_adv_df(ctx->nk, 0, 0, ad, ctx->stream));  // then x2, back to FP64
  } else if (f64_state(ctx->prec)) {
    W2_TRY(shift_pass64(ctx, 1, 0, (const double *)f, nullptr, ctx->t1, nullptr, ctx->stream));  // x1 first
    W2_TRY(shift_pass64(ctx, 0, 0, ctx->t1, nullptr, (double *)out, nullptr, ctx->stream));       // then x2
  } else {
    Adv32Args av = adv32_args(ctx);
    av.f = (const float *)f;
    av.g = nullptr;
    av.d2 = (float *)ctx->t1;
    W2_TRY(launch_adv_f32(ctx->nk, 0, av, ctx->stream));  // increment along x2
    av.d2in = (const float *)ctx->t1;
    av.g2in = nullptr;
    av.ft = (float *)out;
    W2_TRY(launch_adv_f32(ctx->nk, 1, av, ctx->stream));  // then x1: out = S1 (f + d2)
  }
  return W2_OK;
}

extern "C" w2_status w2_step_profile(w2_ctx *ctx, int32_t nsteps, double *kernel_ms) {
  if (!ctx || nsteps <= 0 || !kernel_ms) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot || !ctx->have_state) return W2_ERR_STATE;
  const int NE = 2 * W2_STEP_KERNELS;
  std::vector<cudaEvent_t> ev((size_t)NE * nsteps, nullptr);
  w2_status st = W2_OK;
  for (auto &x : ev)
    if (cudaEventCreate(&x) != cudaSuccess) {
      st = W2_ERR_CUDA;
      break;
    }
  for (int q = 0; q < W2_STEP_KERNELS; ++q) kernel_ms[q] = 0.0;
  for (int s = 0; s < nsteps && st == W2_OK; ++s) {
    StepEvents se{ev.data() + (size_t)NE * s};
    if (enqueue_any(ctx, ctx->stream, &se) != cudaSuccess) st = W2_ERR_CUDA;
  }
  if (st == W2_OK && cudaStreamSynchronize(ctx->stream) != cudaSuccess) st = W2_ERR_CUDA;
  for (int s = 0; s < nsteps && st == W2_OK; ++s)
    for (int q = 0; q < W2_STEP_KERNELS; ++q) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, ev[(size_t)NE * s + 2 * q], ev[(size_t)NE * s + 2 * q + 1]) != cudaSuccess) {
        st = W2_ERR_CUDA;
        break;
      }
      kernel_ms[q] += ms / nsteps;
    }
  for (auto &x : ev)
    if (x) cudaEventDestroy(x);
  if (st != W2_OK) {
    ctx->sticky = st;
    return st;
  }
  ctx->steps += nsteps;
  return W2_OK;
}

// ---------------------------------------------------------------------------
// Learned form
// ---------------------------------------------------------------------------

// Exact two-body term of `f` alone: the sweep with zero one-body tables.
// The pair term alone with the pair table K12 (the exact one by default).
static cudaError_t enqueue_pair_exact(w2_ctx *ctx, const void *f, void *out, cudaStream_t s,
                                      const double *K12 = nullptr) {
  const int nx = ctx->nx, nk = ctx->nk, W = 2 * nk - 1;
  if (!K12) K12 = ctx->K12;
  if (f64_state(ctx->prec)) {
    ThetaArgs th;
    th.nx = nx;
    th.in = (const double *)f;
    th.h = nullptr;
    th.out = (double *)out;
    th.xsum = nullptr;
    th.K1 = ctx->Kzero;
    th.K2 = ctx->Kzero + (size_t)nx * W;
    th.K12 = K12;
    th.half_tau = 0.0;
    return theta64(ctx, 0, th, s);
  }
  Theta32Args th;
  th.nx = nx;
  th.in = (const float *)f;
  th.base = nullptr;
  th.h = nullptr;
  th.out = (float *)out;
  th.K1 = ctx->Kzero;
  th.K2 = ctx->Kzero + (size_t)nx * W;
  th.K12 = K12;
  th.half_tau = 0.0f;
  return theta32(ctx, 0, th, s);
}

static w2_status ensure_pair_buffers(w2_ctx *ctx) {
  const int nx = ctx->nx, W = 2 * ctx->nk - 1;
  if (!ctx->Kzero) {
    if (dev_alloc((void **)&ctx->Kzero, sizeof(double) * 2 * nx * W) != cudaSuccess) return W2_ERR_OOM;
    if (cudaMemset(ctx->Kzero, 0, sizeof(double) * 2 * nx * W) != cudaSuccess) return W2_ERR_CUDA;
  }
  if (!ctx->f1 && dev_alloc((void **)&ctx->f1, sizeof(float) * nx * ctx->nk) != cudaSuccess) return W2_ERR_OOM;
  return W2_OK;
}

extern "C" w2_status w2_theta_pair(w2_ctx *ctx, const void *f, void *out) {
  if (!ctx || !f || !out || f == out) return W2_ERR_ARG;
  if (((uintptr_t)f | (uintptr_t)out) & 15) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot) return W2_ERR_STATE;
  w2_status st = ensure_pair_buffers(ctx);
  if (st != W2_OK) return st;
  W2_TRY(enqueue_pair_exact(ctx, f, out, ctx->stream));
  return W2_OK;
}

extern "C" w2_status w2_features(w2_ctx *ctx, const w2_mlp *m, const void *f, const int32_t *xs, int32_t rows,
                                 void *x) {
  if (!ctx || !m || !f || !x || rows < 1) return W2_ERR_ARG;
  if (mlp_nk(m) != ctx->nk) return W2_ERR_ARG;
  if (!xs && rows != ctx->nx * ctx->nx) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  w2_status st = ensure_pair_buffers(ctx);
  if (st != W2_OK) return st;
  FeatArgs fa;
  fa.nx = ctx->nx;
  fa.nk = ctx->nk;
  fa.din = mlp_din(m);
  fa.dx = ctx->dx;
  fa.dp = ctx->dp;
  fa.s_f = mlp_scale(m, 0);
  fa.s_f1 = mlp_scale(m, 1);
  fa.f1 = ctx->f1;
  fa.f1_src_rows = 1;
  fa.xs = xs;
  fa.x = (uint16_t *)x;
  W2_TRY(launch_features(fa, f, f64_state(ctx->prec), rows, ctx->stream));
  return W2_OK;
}

// Relative L2 error of the network's two-body term against the exact one on
// the current state; falls back to the exact term when above the tolerance.
static w2_status learned_judge(w2_ctx *ctx) {
  cudaStream_t s = ctx->stream;
  W2_TRY(enqueue_pair_exact(ctx, ctx->f, ctx->g, s));
  if (mlp_kind(ctx->mlp) == 1) {  // the network's pair term: the sweep with its table (t1 is free between steps)
    W2_TRY(enqueue_pair_exact(ctx, ctx->f, ctx->t1, s, ctx->Klearn));
    W2_TRY(launch_sqdiff64((const double *)ctx->t1, (const double *)ctx->g, mlp_part(ctx->mlp), ctx->npts, s));
  } else {
    W2_TRY(enqueue_learned_pair(ctx, ctx->f, s));
    W2_TRY(launch_sqdiff(mlp_out(ctx->mlp), ctx->g, f64_state(ctx->prec), mlp_part(ctx->mlp), ctx->npts, 1.0, s));
  }
  W2_TRY(cudaMemcpyAsync(mlp_hpart(ctx->mlp), mlp_part(ctx->mlp), sizeof(double) * 256, cudaMemcpyDeviceToHost, s));
  W2_TRY(cudaStreamSynchronize(s));
  double d = 0.0, r = 0.0;
  for (int q = 0; q < 128; ++q) {
    d += mlp_hpart(ctx->mlp)[2 * q];
    r += mlp_hpart(ctx->mlp)[2 * q + 1];
  }
  ctx->last_err = r > 0.0 ? sqrt(d / r) : (d > 0.0 ? INFINITY : 0.0);
  ctx->judged += 1;
  if (!(ctx->last_err <= ctx->judge_tol)) {
    ctx->learned_active = false;
    drop_graphs(ctx);  // the captured steps used the network
  }
  return W2_OK;
}

extern "C" w2_status w2_learned_attach(w2_ctx *ctx, w2_mlp *m, int32_t judge_every, double tol) {
  if (!ctx) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  drop_graphs(ctx);
  if (!m) {
    ctx->mlp = nullptr;
    ctx->learned_active = false;
    return W2_OK;
  }
  if (!f64_state(ctx->prec)) return W2_ERR_UNSUPPORTED;
  const bool kernel_net = mlp_kind(m) == 1;
  if (mlp_nk(m) != ctx->nk || mlp_maxrows(m) < (kernel_net ? ctx->nx : ctx->nx * ctx->nx) || judge_every < 0 ||
      !(tol >= 0))
    return W2_ERR_ARG;
  w2_status st = ensure_pair_buffers(ctx);
  if (st != W2_OK) return st;
  if (kernel_net) {
    // the network's pair table for every distance d dx, evaluated once: it
    // depends on the distance alone, like the exact table it stands in for
    const int W = 2 * ctx->nk - 1;
    if (!ctx->Klearn && dev_alloc((void **)&ctx->Klearn, sizeof(double) * (size_t)ctx->nx * W) != cudaSuccess)
      return W2_ERR_OOM;
    uint16_t *rows = nullptr;  // the distance features, only for this evaluation
    if (dev_alloc((void **)&rows, sizeof(uint16_t) * (size_t)ctx->nx * mlp_din(m)) != cudaSuccess) return W2_ERR_OOM;
    cudaError_t e = launch_rfeat(rows, ctx->nx, mlp_din(m), ctx->stream);
    if (e == cudaSuccess) e = mlp_forward(m, rows, ctx->nx, mlp_out(m), 1.0f, ctx->stream);
    if (e == cudaSuccess)
      e = launch_pairk_table(mlp_out(m), ctx->nx, ctx->nk, 1.0f / mlp_scale(m, 2), ctx->Klearn, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(rows);
    W2_TRY(e);
  }
  if (!kernel_net && !ctx->xrows &&
      dev_alloc((void **)&ctx->xrows, sizeof(uint16_t) * (size_t)ctx->nx * ctx->nx * mlp_din(m)) != cudaSuccess)
    return W2_ERR_OOM;
  ctx->mlp = m;
  ctx->learned_active = true;
  ctx->judge_every = judge_every;
  ctx->judge_tol = tol;
  ctx->since_judge = 0;
  ctx->judged = 0;
  ctx->last_err = 0.0;
  return W2_OK;
}

extern "C" w2_status w2_learned_report(w2_ctx *ctx, int32_t *active, int32_t *judged, double *last_err) {
  if (!ctx) return W2_ERR_ARG;
  if (active) *active = ctx->mlp && ctx->learned_active ? 1 : 0;
  if (judged) *judged = ctx->judged;
  if (last_err) *last_err = ctx->last_err;
  return W2_OK;
}

// ---------------------------------------------------------------------------
// Occupation numbers and correlation entropy
// ---------------------------------------------------------------------------

extern "C" w2_status w2_occupations(w2_ctx *ctx, double *occ, double *entropy) {
  if (!ctx) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_state) return W2_ERR_STATE;
  const int nx = ctx->nx, nk = ctx->nk;
  if (!ctx->rdm_rho) {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dev_alloc((void **)&ctx->rdm_f1, sizeof(double) * nx * nk);
    if (e == cudaSuccess) e = dev_alloc((void **)&ctx->rdm_fh, sizeof(double) * nx * nk);
    if (e == cudaSuccess) e = dev_alloc((void **)&ctx->rdm_kh, sizeof(double) * nx);
    if (e == cudaSuccess) e = dev_alloc((void **)&ctx->rdm_eig, sizeof(double) * (nx + 1));
    if (e == cudaSuccess) e = dev_alloc((void **)&ctx->rdm_ph, sizeof(double2) * nx * nk);
    if (e == cudaSuccess) e = dev_alloc((void **)&ctx->rdm_rho, sizeof(double2) * nx * nx);
    if (e != cudaSuccess) {  // release the part that was taken, so that a later call starts afresh
      void **bufs[] = {(void **)&ctx->rdm_f1, (void **)&ctx->rdm_fh, (void **)&ctx->rdm_kh,
                       (void **)&ctx->rdm_eig, (void **)&ctx->rdm_ph, (void **)&ctx->rdm_rho};
      for (void **b : bufs) {
        if (*b) cudaFree(*b);
        *b = nullptr;
      }
      (void)cudaGetLastError();
      return W2_ERR_OOM;
    }
    // half-point interpolation kernel: K(j + 1/2), K(t) = (1/N)[1 + 2 sum_{0 < m < N/2} cos(2 pi m t / N)]
    std::vector<double> kh(nx);
    for (int j = 0; j < nx; ++j) {
      double v = 1.0;
      for (int m = 1; 2 * m < nx; ++m) v += 2.0 * cos(2.0 * M_PI * m * (j + 0.5) / nx);
      kh[j] = v / nx;
    }
    // phases dp e^{-2 pi i (n - nk/2)(d/2)/nx}, d = -(nx/2) .. nx - nx/2 - 1
    std::vector<double2> ph((size_t)nx * nk);
    for (int di = 0; di < nx; ++di) {
      const int d = di - nx / 2;
      for (int n = 0; n < nk; ++n) {
        const double a = -2.0 * M_PI * (n - nk / 2) * (0.5 * d) / nx;
        ph[(size_t)di * nk + n] = make_double2(ctx->dp * cos(a), ctx->dp * sin(a));
      }
    }
    W2_TRY(cudaMemcpy(ctx->rdm_kh, kh.data(), sizeof(double) * nx, cudaMemcpyHostToDevice));
    W2_TRY(cudaMemcpy(ctx->rdm_ph, ph.data(), sizeof(double2) * nx * nk, cudaMemcpyHostToDevice));
  }
  cudaStream_t s = ctx->stream;
  W2_TRY(launch_rdm_f1(ctx->f, f64_state(ctx->prec), ctx->rdm_f1, nx, nk, ctx->dx, ctx->dp, s));
  W2_TRY(launch_rdm_rho(ctx->rdm_f1, ctx->rdm_kh, ctx->rdm_fh, ctx->rdm_ph, ctx->rdm_rho, nx, nk, ctx->dx, s));
  W2_TRY(launch_herm_eigvals(ctx->rdm_rho, nx, 1, ctx->rdm_eig, s));
  W2_TRY(launch_corr_entropy(ctx->rdm_eig, nx, ctx->rdm_eig + nx, s));
  if (occ) W2_TRY(cudaMemcpyAsync(occ, ctx->rdm_eig, sizeof(double) * nx, cudaMemcpyDeviceToHost, s));
  if (entropy) W2_TRY(cudaMemcpyAsync(entropy, ctx->rdm_eig + nx, sizeof(double), cudaMemcpyDeviceToHost, s));
  W2_TRY(cudaStreamSynchronize(s));
  return W2_OK;
}

extern "C" w2_status w2_hermitian_eigvals(void *a, int32_t n, int32_t batch, double *eig, void *cuda_stream) {
  if (!a || !eig || n < 1 || n > 4096 || batch < 1) return W2_ERR_ARG;
  if ((uintptr_t)a & 15) return W2_ERR_ARG;
  cudaError_t e = launch_herm_eigvals((double2 *)a, n, batch, eig, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) {
    note_cuda_error(e);
    return W2_ERR_CUDA;
  }
  return W2_OK;
}

