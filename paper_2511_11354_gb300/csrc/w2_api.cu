// C ABI of the w2 library: context, host-side tables, stability precheck,
// step orchestration (one Lawson step captured into a CUDA graph).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "w2_internal.cuh"

using namespace w2;

struct w2_ctx {
  w2_config cfg;
  cudaStream_t stream;       // borrowed
  cudaStream_t cap;          // private stream used only for graph capture
  int dev;
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
  double *xpart, *obs_out, *h_obs;
  double z, zscale;
  int nterm;
  cudaGraphExec_t graph;
  bool graph_ready;
};

#define W2_TRY(call)                                    \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) {                            \
      ctx->sticky = W2_ERR_CUDA;                        \
      return W2_ERR_CUDA;                               \
    }                                                   \
  } while (0)

static double fold(double x, double L) { return x - L * floor((x + 0.5 * L) / L); }

static void free_all(w2_ctx *c) {
  void *ptrs[] = {c->f, c->g, c->t1, c->t2, c->xsum, c->xsum2, c->K, c->K12, c->vext_fine, c->w_fine,
                  c->d_fine, c->sintab, c->vext_grid, c->k0tab, c->wtab, c->xpart, c->obs_out};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (c->h_obs) cudaFreeHost(c->h_obs);
  if (c->graph_ready) cudaGraphExecDestroy(c->graph);
  if (c->cap) cudaStreamDestroy(c->cap);
}

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
  if (cfg->precision != W2_F64) return W2_ERR_UNSUPPORTED;
  if (!nk_supported_f64(cfg->nk) || cfg->nx > 128) return W2_ERR_UNSUPPORTED;
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
  ctx->nx = cfg->nx;
  ctx->nk = cfg->nk;
  ctx->M = 2 * cfg->nk;
  ctx->npts = (size_t)cfg->nx * cfg->nx * cfg->nk * cfg->nk;
  ctx->dx = cfg->L / cfg->nx;
  ctx->dp = M_PI * cfg->hbar / cfg->L;
  ctx->hp = cfg->L / ctx->M;
  ctx->tau = cfg->dt;
  ctx->z = sqrt(3.0) - 2.0;
  ctx->nterm = ctx->nx <= 32 ? ctx->nx : 32;
  ctx->zscale = (ctx->nterm == ctx->nx) ? 1.0 / (1.0 - pow(ctx->z, ctx->nx)) : 1.0;

  const int nx = ctx->nx, nk = ctx->nk, M = ctx->M, W = 2 * nk - 1;
  cudaError_t e = cudaSuccess;
#define W2_ALLOC(ptr, bytes)                                  \
  if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), (bytes));
  const size_t fb = sizeof(double) * ctx->npts;
  W2_ALLOC(ctx->f, fb) W2_ALLOC(ctx->g, fb) W2_ALLOC(ctx->t1, fb) W2_ALLOC(ctx->t2, fb)
  W2_ALLOC(ctx->xsum, sizeof(double) * nx * nx) W2_ALLOC(ctx->xsum2, sizeof(double) * nx * nx)
  W2_ALLOC(ctx->K, sizeof(double) * 2 * nx * W) W2_ALLOC(ctx->K12, sizeof(double) * nx * W)
  W2_ALLOC(ctx->vext_fine, sizeof(double) * nx * M) W2_ALLOC(ctx->w_fine, sizeof(double) * nx * M)
  W2_ALLOC(ctx->d_fine, sizeof(double) * nx * M) W2_ALLOC(ctx->sintab, sizeof(double) * M)
  W2_ALLOC(ctx->vext_grid, sizeof(double) * nx) W2_ALLOC(ctx->k0tab, sizeof(int) * nk)
  W2_ALLOC(ctx->wtab, sizeof(double) * 4 * nk) W2_ALLOC(ctx->xpart, sizeof(double) * nx * nx * (3 + nk))
  W2_ALLOC(ctx->obs_out, sizeof(double) * (8 + nx + nx * nx))
#undef W2_ALLOC
  if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->h_obs, sizeof(double) * (8 + nx + nx * nx));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = prepare_kernels_f64(nk);
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
  if (e != cudaSuccess) {
    free_all(ctx);
    delete ctx;
    return W2_ERR_CUDA;
  }
  *out = ctx;
  return W2_OK;
}

static TabArgs tab_args(w2_ctx *ctx, const double *xsum, int pair_mode) {
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
  return a;
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
  const double hart = 2.0 * fabs(c_hartree) * fabs(gamma) * (wmax - wmin);
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
  if (ctx->graph_ready) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph_ready = false;
  }
  return W2_OK;
}

extern "C" w2_status w2_set_state(w2_ctx *ctx, const void *f, int32_t on_device) {
  if (!ctx || !f) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot) return W2_ERR_STATE;
  W2_TRY(cudaMemcpyAsync(ctx->f, f, sizeof(double) * ctx->npts,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  W2_TRY(launch_xsum_f64(ctx->nx, ctx->nk, ctx->f, ctx->xsum, ctx->stream));
  ctx->have_state = true;
  ctx->steps = 0;
  return W2_OK;
}

extern "C" w2_status w2_get_state(w2_ctx *ctx, void *f, int32_t on_device) {
  if (!ctx || !f) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_state) return W2_ERR_STATE;
  W2_TRY(cudaMemcpyAsync(f, ctx->f, sizeof(double) * ctx->npts,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  if (!on_device) W2_TRY(cudaStreamSynchronize(ctx->stream));
  return W2_OK;
}

// Optional per-kernel CUDA events around every launch of a step (profiling).
struct StepEvents {
  cudaEvent_t *ev;  // [2 * W2_STEP_KERNELS] or null
};

#define W2_MARK(k, pos)                                                             \
  if (evs && evs->ev) {                                                             \
    if ((e = cudaEventRecord(evs->ev[2 * (k) + (pos)], s)) != cudaSuccess) return e; \
  }

// One Lawson step on stream s (see w2.h):
//   xsum(f^n) ; K(f^n) ; g = Theta f^n ; (t1, t2) = A_x2 (f, g) ;
//   (f~ -> g, h -> f) = A_x1 (t1, t2) ; xsum(f~) ; K(f~) ; f = h + tau/2 Theta f~
static cudaError_t enqueue_step(w2_ctx *ctx, cudaStream_t s, const StepEvents *evs = nullptr) {
  const int nx = ctx->nx, nk = ctx->nk, W = 2 * nk - 1;
  cudaError_t e;
  TabArgs ta = tab_args(ctx, ctx->xsum, 0);
  // per-X sums of f^n always from the same fixed-order reduction, so a state
  // restored with w2_set_state continues bit-identically
  W2_MARK(0, 0)
  if ((e = launch_xsum_f64(nx, nk, ctx->f, ctx->xsum, s)) != cudaSuccess) return e;
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
  W2_MARK(2, 0)
  if ((e = launch_theta_f64(nk, 0, th, s)) != cudaSuccess) return e;
  W2_MARK(2, 1)
  AdvArgs av;
  av.nx = nx;
  av.k0tab = ctx->k0tab;
  av.wtab = ctx->wtab;
  av.z = ctx->z;
  av.zscale = ctx->zscale;
  av.nterm = ctx->nterm;
  av.tau = ctx->tau;
  av.in0 = ctx->f;
  av.in1 = ctx->g;
  av.out0 = ctx->t1;
  av.out1 = ctx->t2;
  W2_MARK(3, 0)
  if ((e = launch_adv_f64(nk, 0, 1, av, s)) != cudaSuccess) return e;
  W2_MARK(3, 1)
  av.in0 = ctx->t1;
  av.in1 = ctx->t2;
  av.out0 = ctx->g;  // f~
  av.out1 = ctx->f;  // h
  W2_MARK(4, 0)
  if ((e = launch_adv_f64(nk, 1, 1, av, s)) != cudaSuccess) return e;
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
  th.xsum = nullptr;
  W2_MARK(7, 0)
  if ((e = launch_theta_f64(nk, 1, th, s)) != cudaSuccess) return e;
  W2_MARK(7, 1)
  return cudaSuccess;
}

extern "C" w2_status w2_step(w2_ctx *ctx, int32_t nsteps) {
  if (!ctx || nsteps < 0) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot || !ctx->have_state) return W2_ERR_STATE;
  if (nsteps == 0) return W2_OK;
  if (!ctx->graph_ready) {
    cudaGraph_t graph;
    W2_TRY(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_step(ctx, ctx->cap);
    cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (e2 == cudaSuccess) cudaGraphDestroy(graph);
      ctx->sticky = W2_ERR_CUDA;
      return W2_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&ctx->graph, graph, 0);
    cudaGraphDestroy(graph);
    W2_TRY(e);
    ctx->graph_ready = true;
  }
  for (int s = 0; s < nsteps; ++s) W2_TRY(cudaGraphLaunch(ctx->graph, ctx->stream));
  ctx->steps += nsteps;
  return W2_OK;
}

extern "C" w2_status w2_observables(w2_ctx *ctx, w2_obs *out, double *n1, double *n12) {
  if (!ctx || !out) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_state) return W2_ERR_STATE;
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
  a.f = ctx->f;
  a.vext_grid = ctx->vext_grid;
  a.w_fine = ctx->w_fine;
  a.xpart = ctx->xpart;
  a.out = ctx->obs_out;
  W2_TRY(launch_obs_f64(a, ctx->stream));
  const size_t nb = sizeof(double) * (8 + nx + (size_t)nx * nx);
  W2_TRY(cudaMemcpyAsync(ctx->h_obs, ctx->obs_out, nb, cudaMemcpyDeviceToHost, ctx->stream));
  W2_TRY(cudaStreamSynchronize(ctx->stream));
  const double *h = ctx->h_obs;
  out->mass = h[0];
  out->energy = h[1];
  out->purity = h[2];
  out->entropy_lin = 1.0 - h[2];
  out->l2norm = h[3];
  out->step = ctx->steps;
  if (n1) memcpy(n1, h + 8, sizeof(double) * nx);
  if (n12) memcpy(n12, h + 8 + nx, sizeof(double) * nx * nx);
  return h[4] != 0.0 ? W2_ERR_NONFINITE : W2_OK;
}

extern "C" w2_status w2_theta(w2_ctx *ctx, const double *f, double *out) {
  if (!ctx || !f || !out || f == out) return W2_ERR_ARG;
  // the sweep moves pairs of doubles: both arrays must be 16-byte aligned
  if (((uintptr_t)f | (uintptr_t)out) & 15) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot) return W2_ERR_STATE;
  const int nx = ctx->nx, nk = ctx->nk, W = 2 * nk - 1;
  W2_TRY(launch_xsum_f64(nx, nk, f, ctx->xsum2, ctx->stream));
  TabArgs ta = tab_args(ctx, ctx->xsum2, 0);
  W2_TRY(launch_tables(ta, ctx->stream));
  ThetaArgs th;
  th.nx = nx;
  th.in = f;
  th.h = nullptr;
  th.out = out;
  th.xsum = nullptr;
  th.K1 = ctx->K;
  th.K2 = ctx->K + (size_t)nx * W;
  th.K12 = ctx->K12;
  th.half_tau = 0.5 * ctx->tau;
  W2_TRY(launch_theta_f64(nk, 0, th, ctx->stream));
  return W2_OK;
}

extern "C" w2_status w2_advect(w2_ctx *ctx, const double *f, double *out) {
  if (!ctx || !f || !out || f == out) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot) return W2_ERR_STATE;
  AdvArgs av;
  av.nx = ctx->nx;
  av.k0tab = ctx->k0tab;
  av.wtab = ctx->wtab;
  av.z = ctx->z;
  av.zscale = ctx->zscale;
  av.nterm = ctx->nterm;
  av.tau = ctx->tau;
  av.in0 = f;
  av.in1 = nullptr;
  av.out0 = ctx->t1;
  av.out1 = nullptr;
  W2_TRY(launch_adv_f64(ctx->nk, 1, 0, av, ctx->stream));  // x1 first
  av.in0 = ctx->t1;
  av.out0 = out;
  W2_TRY(launch_adv_f64(ctx->nk, 0, 0, av, ctx->stream));  // then x2
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
    if (enqueue_step(ctx, ctx->stream, &se) != cudaSuccess) st = W2_ERR_CUDA;
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
