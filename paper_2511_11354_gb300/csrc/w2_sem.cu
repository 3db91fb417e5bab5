// C ABI of the non-periodic path (include/w2_sem.h): context, set-up of the
// static tables, and the orchestration of the operator (Sec. 3.2), the
// natural-boundary spline shift and the Lawson step (Sec. 4.1).
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "w2_internal.cuh"
#include "w2_sem.cuh"

using namespace w2sem;

struct w2_sem_ctx {
  int nx, M, Q, np, h, Ny, Nyh, xc_kind, C, bx;
  double L, Lp, dx, width, tau, hbar, mass, gamma = 0.0, c_h = 0.0, c_xc = 0.0;
  long long npts;
  bool have_pot = false, have_state = false;
  w2_status sticky = W2_OK;
  int64_t step = 0;
  cudaStream_t stream;
  std::vector<double> hp, hw;
  // device
  double *f = nullptr, *g = nullptr, *a = nullptr, *b = nullptr, *t = nullptr;
  double *p = nullptr, *w = nullptr, *centre = nullptr, *cheb = nullptr, *osc = nullptr, *psi = nullptr;
  double *phir = nullptr, *phii = nullptr, *ph = nullptr, *eh = nullptr, *eier = nullptr;
  double *cp = nullptr, *wts = nullptr, *vext = nullptr, *wgrid = nullptr;
  double *xs = nullptr, *n = nullptr, *U = nullptr, *ut = nullptr, *G = nullptr;
  double *cT = nullptr, *cA = nullptr, *cS = nullptr, *xpart = nullptr, *obs = nullptr, *h_obs = nullptr;
  int *k0 = nullptr;
};

#define SEM_TRY(call)                   \
  do {                                  \
    cudaError_t e_ = (call);            \
    if (e_ != cudaSuccess) {            \
      w2::note_cuda_error(e_);          \
      ctx->sticky = W2_ERR_CUDA;        \
      return W2_ERR_CUDA;               \
    }                                   \
  } while (0)

static void sem_free(w2_sem_ctx *c) {
  double *d[] = {c->f, c->g, c->a, c->b, c->t, c->p, c->w, c->centre, c->cheb, c->osc, c->psi, c->phir,
                 c->phii, c->ph, c->eh, c->eier, c->cp, c->wts, c->vext, c->wgrid, c->xs, c->n, c->U,
                 c->ut, c->G, c->cT, c->cA, c->cS, c->xpart, c->obs};
  for (double *q : d)
    if (q) cudaFree(q);
  if (c->k0) cudaFree(c->k0);
  if (c->h_obs) cudaFreeHost(c->h_obs);
}

extern "C" w2_status w2_sem_create(const w2_sem_config *cfg, void *cuda_stream, w2_sem_ctx **out) {
  if (!cfg || !out) return W2_ERR_ARG;
  *out = nullptr;
  const int nx = cfg->nx, M = cfg->ncell, Q = cfg->nq;
  if (nx < 8 || nx > 1024 || M < 1 || Q < 2 || Q > 32 || (long long)M * Q > 256) return W2_ERR_ARG;
  if (!(cfg->L > 0) || !(cfg->Lp > 0) || !(cfg->dt > 0) || !(cfg->hbar > 0) || !(cfg->mass > 0)) return W2_ERR_ARG;
  if (cfg->xc_kind < 0 || cfg->xc_kind > 2) return W2_ERR_ARG;
  // the Bessel recurrence of the oscillatory integrals runs to about z + 20 z^(1/3) + 40 terms
  if (cfg->Lp / M * cfg->L / cfg->hbar > 4096.0) return W2_ERR_ARG;
  w2_sem_ctx *ctx = new (std::nothrow) w2_sem_ctx();
  if (!ctx) return W2_ERR_OOM;
  ctx->nx = nx; ctx->M = M; ctx->Q = Q; ctx->np = M * Q;
  ctx->h = (nx - 1) / 2; ctx->Ny = 2 * ctx->h + 1; ctx->Nyh = ctx->h + 1;
  ctx->L = cfg->L; ctx->Lp = cfg->Lp; ctx->dx = cfg->L / (nx - 1); ctx->width = cfg->Lp / M;
  ctx->tau = cfg->dt; ctx->hbar = cfg->hbar; ctx->mass = cfg->mass; ctx->xc_kind = cfg->xc_kind;
  ctx->stream = (cudaStream_t)cuda_stream;
  const int np = ctx->np, Ny = ctx->Ny, Nyh = ctx->Nyh;
  ctx->npts = (long long)nx * nx * np * np;
  ctx->C = sem_adv_cols(nx, np);
  // two-body chain chunk: about 256 MB of intermediates
  const double per_x = 8.0 * (2.0 * np * Ny + 2.0 * Nyh * Ny + 2.0 * np * Ny);
  long long bx = (long long)(256.0 * 1024 * 1024 / per_x);
  if (bx < 1) bx = 1;
  if (bx > (long long)nx * nx) bx = (long long)nx * nx;
  ctx->bx = (int)bx;

  // host geometry: nodes, cell centres, Chebyshev transform, weights, spline tables
  std::vector<double> centre(M), eta(Q), cheb(Q * Q), p(np), w(np), cp(nx, 0.0), wts(4 * np);
  std::vector<int> k0(np);
  for (int s = 0; s < M; ++s) centre[s] = -0.5 * cfg->Lp + ctx->width * (s + 0.5);
  for (int q = 0; q < Q; ++q) eta[q] = -cos((2 * q + 1) * M_PI / (2 * Q));
  for (int l = 0; l < Q; ++l)
    for (int q = 0; q < Q; ++q) cheb[l * Q + q] = (l == 0 ? 1.0 : 2.0) / Q * cos(l * acos(eta[q]));
  std::vector<double> wq(Q, 0.0);
  for (int q = 0; q < Q; ++q)
    for (int l = 0; l < Q; l += 2) wq[q] += 2.0 / (1.0 - (double)l * l) * cheb[l * Q + q];
  for (int s = 0; s < M; ++s)
    for (int q = 0; q < Q; ++q) {
      p[s * Q + q] = centre[s] + 0.5 * ctx->width * eta[q];
      w[s * Q + q] = 0.5 * ctx->width * wq[q];
    }
  for (int i = 1; i < nx - 1; ++i) cp[i] = 1.0 / (4.0 - cp[i - 1]);
  for (int j = 0; j < np; ++j) {
    const double sh = -ctx->tau * p[j] / (ctx->mass * ctx->dx);  // foot offset in cells
    const double kf = floor(sh), th = sh - kf;
    k0[j] = (int)kf;
    wts[4 * j + 0] = (1.0 - th) * (1.0 - th) * (1.0 - th) / 6.0;
    wts[4 * j + 1] = (3.0 * th * th * th - 6.0 * th * th + 4.0) / 6.0;
    wts[4 * j + 2] = (-3.0 * th * th * th + 3.0 * th * th + 3.0 * th + 1.0) / 6.0;
    wts[4 * j + 3] = th * th * th / 6.0;
  }
  ctx->hp = p;
  ctx->hw = w;

  cudaError_t e = cudaSuccess;
#define SEM_ALLOC(ptr, count) \
  if (e == cudaSuccess) e = cudaMalloc((void **)&(ptr), sizeof(*(ptr)) * (size_t)(count));
  const long long N = ctx->npts;
  SEM_ALLOC(ctx->f, N) SEM_ALLOC(ctx->g, N) SEM_ALLOC(ctx->a, N) SEM_ALLOC(ctx->b, N) SEM_ALLOC(ctx->t, N)
  SEM_ALLOC(ctx->p, np) SEM_ALLOC(ctx->w, np) SEM_ALLOC(ctx->centre, M) SEM_ALLOC(ctx->cheb, Q * Q)
  SEM_ALLOC(ctx->osc, 2LL * nx * Q) SEM_ALLOC(ctx->psi, (2LL * nx - 1) * np * np)
  SEM_ALLOC(ctx->phir, (long long)Ny * np) SEM_ALLOC(ctx->phii, (long long)Ny * np)
  SEM_ALLOC(ctx->ph, 4LL * Nyh * np) SEM_ALLOC(ctx->eh, 4LL * np * Nyh) SEM_ALLOC(ctx->eier, 2LL * np * Ny)
  SEM_ALLOC(ctx->cp, nx) SEM_ALLOC(ctx->wts, 4 * np) SEM_ALLOC(ctx->k0, np) SEM_ALLOC(ctx->vext, nx)
  SEM_ALLOC(ctx->wgrid, 4 * nx - 3) SEM_ALLOC(ctx->xs, (long long)nx * nx) SEM_ALLOC(ctx->n, 2 * nx)
  SEM_ALLOC(ctx->U, 2 * nx) SEM_ALLOC(ctx->ut, 2LL * nx * (2 * nx - 1)) SEM_ALLOC(ctx->G, 2LL * nx * np * np)
  SEM_ALLOC(ctx->cT, bx * 2 * np * Ny) SEM_ALLOC(ctx->cA, bx * 2 * Nyh * Ny) SEM_ALLOC(ctx->cS, bx * 2 * np * Ny)
  SEM_ALLOC(ctx->xpart, (long long)nx * nx * (4 + np)) SEM_ALLOC(ctx->obs, 8 + nx)
#undef SEM_ALLOC
  if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->h_obs, sizeof(double) * (8 + nx));
  auto up = [&](void *dst, const void *src, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
  };
  up(ctx->p, p.data(), sizeof(double) * np);
  up(ctx->w, w.data(), sizeof(double) * np);
  up(ctx->centre, centre.data(), sizeof(double) * M);
  up(ctx->cheb, cheb.data(), sizeof(double) * Q * Q);
  up(ctx->cp, cp.data(), sizeof(double) * nx);
  up(ctx->wts, wts.data(), sizeof(double) * 4 * np);
  up(ctx->k0, k0.data(), sizeof(int) * np);
  SemTabArgs ta{nx, M, Q, np, ctx->h, ctx->dx, ctx->width, ctx->hbar, ctx->Lp, ctx->p, ctx->centre, ctx->cheb,
                ctx->osc, ctx->psi, ctx->phir, ctx->phii, ctx->ph, ctx->eh, ctx->eier};
  if (e == cudaSuccess) e = launch_sem_osc(ta, ctx->stream);
  if (e == cudaSuccess) e = launch_sem_tables(ta, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    w2::note_cuda_error(e);
    const w2_status st = (e == cudaErrorMemoryAllocation) ? W2_ERR_OOM : W2_ERR_CUDA;
    cudaGetLastError();
    sem_free(ctx);
    delete ctx;
    return st;
  }
  *out = ctx;
  return W2_OK;
}

extern "C" w2_status w2_sem_set_potentials(w2_sem_ctx *ctx, w2_fn vext, void *ue, w2_fn vee, void *ui,
                                           double gamma, double c_h, double c_xc) {
  if (!ctx || !vext || !vee) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!isfinite(gamma) || !isfinite(c_h) || !isfinite(c_xc)) return W2_ERR_ARG;
  const int nx = ctx->nx, W0 = 2 * (nx - 1);
  std::vector<double> v(nx), wg(4 * nx - 3);
  for (int i = 0; i < nx; ++i) v[i] = vext(-0.5 * ctx->L + ctx->dx * i, ue);
  for (int k = -W0; k <= W0; ++k) wg[k + W0] = vee(k * ctx->dx, ui);
  for (double x : v)
    if (!isfinite(x)) return W2_ERR_ARG;
  for (double x : wg)
    if (!isfinite(x)) return W2_ERR_ARG;
  SEM_TRY(cudaMemcpyAsync(ctx->vext, v.data(), sizeof(double) * nx, cudaMemcpyHostToDevice, ctx->stream));
  SEM_TRY(cudaMemcpyAsync(ctx->wgrid, wg.data(), sizeof(double) * wg.size(), cudaMemcpyHostToDevice, ctx->stream));
  SEM_TRY(cudaStreamSynchronize(ctx->stream));
  ctx->gamma = gamma; ctx->c_h = c_h; ctx->c_xc = c_xc;
  ctx->have_pot = true;
  return W2_OK;
}

extern "C" w2_status w2_sem_momenta(const w2_sem_ctx *ctx, double *p, double *w) {
  if (!ctx) return W2_ERR_ARG;
  if (p) memcpy(p, ctx->hp.data(), sizeof(double) * ctx->np);
  if (w) memcpy(w, ctx->hw.data(), sizeof(double) * ctx->np);
  return W2_OK;
}

extern "C" w2_status w2_sem_set_state(w2_sem_ctx *ctx, const double *f, int32_t on_device) {
  if (!ctx || !f) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  SEM_TRY(cudaMemcpyAsync(ctx->f, f, sizeof(double) * ctx->npts,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  if (!on_device) SEM_TRY(cudaStreamSynchronize(ctx->stream));
  ctx->have_state = true;
  ctx->step = 0;
  return W2_OK;
}

extern "C" w2_status w2_sem_get_state(w2_sem_ctx *ctx, double *f, int32_t on_device) {
  if (!ctx || !f) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_state) return W2_ERR_STATE;
  SEM_TRY(cudaMemcpyAsync(f, ctx->f, sizeof(double) * ctx->npts,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  if (!on_device) SEM_TRY(cudaStreamSynchronize(ctx->stream));
  return W2_OK;
}

// out = Theta[in]: densities -> potentials -> one-body tables G(x) =
// sum_n U(x_n) psi[n - m] -> G1(x1) F_X + F_X G2(x2)^T, then the two-body chain
// per chunk of X: T = F Phi^T, [Ar; Ai] = Ph T, B = w D (.) A,
// [Sr | Si] = Eh B, out += c Im(S E^T).
static w2_status sem_theta(w2_sem_ctx *ctx, const double *in, double *out) {
  const int nx = ctx->nx, np = ctx->np, Ny = ctx->Ny, Nyh = ctx->Nyh;
  const long long np2 = (long long)np * np, nX = (long long)nx * nx;
  cudaStream_t s = ctx->stream;
  SEM_TRY(launch_sem_marginal(nx, np, ctx->dx, in, ctx->w, ctx->xs, ctx->n, s));
  SemPotArgs pa{nx, ctx->xc_kind, ctx->dx, ctx->c_h, ctx->c_xc, ctx->n, ctx->vext, ctx->wgrid, ctx->U, ctx->ut};
  SEM_TRY(launch_sem_potential(pa, s));
  Gemm64 g{};
  // G[2 nx][np*np] = ut[2 nx][2 nx - 1] psi[2 nx - 1][np*np]
  g = Gemm64{2 * nx, (int)np2, 2 * nx - 1, ctx->ut, 2 * nx - 1, 0, ctx->psi, np2, 0, ctx->G, np2, 1.0, 0.0, 1, 1,
             0, 0, 0, 0, 0, 0};
  SEM_TRY(launch_gemm64(g, s));
  // out_X = G1[i1] F_X
  g = Gemm64{np, np, np, ctx->G, np, 0, in, np, 0, out, np, 1.0, 0.0, (int)nX, nx, np2, 0, nx * np2, np2,
             nx * np2, np2};
  SEM_TRY(launch_gemm64(g, s));
  // out_X += F_X G2[i2]^T
  g = Gemm64{np, np, np, in, np, 0, ctx->G + nx * np2, np, 1, out, np, 1.0, 1.0, (int)nX, nx, nx * np2, np2, 0,
             np2, nx * np2, np2};
  SEM_TRY(launch_gemm64(g, s));
  if (ctx->gamma == 0.0) return W2_OK;
  const double alpha = ctx->gamma * ctx->dx * ctx->dx / (M_PI * M_PI * ctx->hbar * ctx->hbar * ctx->hbar);
  const long long sT = 2LL * np * Ny, sA = 2LL * Nyh * Ny, sS = 2LL * np * Ny;
  for (long long x0 = 0; x0 < nX; x0 += ctx->bx) {
    const int nb = (int)((nX - x0) < ctx->bx ? (nX - x0) : ctx->bx);
    const double *F = in + x0 * np2;
    // [Tr; Ti]_X = F_X [Phr^T, Phi^T] (two products into the two row blocks)
    g = Gemm64{np, Ny, np, F, np, 0, ctx->phir, np, 1, ctx->cT, Ny, 1.0, 0.0, nb, 1, np2, 0, 0, 0, sT, 0};
    SEM_TRY(launch_gemm64(g, s));
    g.B = ctx->phii;
    g.C = ctx->cT + (long long)np * Ny;
    SEM_TRY(launch_gemm64(g, s));
    // [Ar; Ai]_X = Ph [Tr; Ti]_X
    g = Gemm64{2 * Nyh, Ny, 2 * np, ctx->ph, 2 * np, 0, ctx->cT, Ny, 0, ctx->cA, Ny, 1.0, 0.0, nb, 1, 0, 0, sT, 0,
               sA, 0};
    SEM_TRY(launch_gemm64(g, s));
    SEM_TRY(launch_sem_dmul(nx, ctx->h, (int)x0, nb, ctx->wgrid, ctx->cA, s));
    // [Sr | Si]_X = [[Er_h | -Ei_h] B, [Ei_h | Er_h] B]
    g = Gemm64{np, Ny, 2 * Nyh, ctx->eh, 2 * Nyh, 0, ctx->cA, Ny, 0, ctx->cS, 2 * Ny, 1.0, 0.0, nb, 1, 0, 0, sA, 0,
               sS, 0};
    SEM_TRY(launch_gemm64(g, s));
    g.A = ctx->eh + 2LL * np * Nyh;
    g.C = ctx->cS + Ny;
    SEM_TRY(launch_gemm64(g, s));
    // out_X += alpha [Sr | Si]_X [Ei | Er]^T
    g = Gemm64{np, np, 2 * Ny, ctx->cS, 2 * Ny, 0, ctx->eier, 2 * Ny, 1, out + x0 * np2, np, alpha, 1.0, nb, 1,
               sS, 0, 0, 0, np2, 0};
    SEM_TRY(launch_gemm64(g, s));
  }
  return W2_OK;
}

static w2_status sem_advect(w2_sem_ctx *ctx, const double *in, double *out) {
  SemAdvArgs aa{ctx->nx, ctx->np, ctx->C, in, ctx->t, ctx->cp, ctx->k0, ctx->wts};
  SEM_TRY(launch_sem_adv(0, aa, ctx->stream));
  aa.in = ctx->t;
  aa.out = out;
  SEM_TRY(launch_sem_adv(1, aa, ctx->stream));
  return W2_OK;
}

static bool overlaps(const double *a, const double *b, long long n) { return a < b + n && b < a + n; }

extern "C" w2_status w2_sem_theta(w2_sem_ctx *ctx, const double *in, double *out) {
  if (!ctx || !in || !out || overlaps(in, out, ctx->npts)) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot) return W2_ERR_STATE;
  return sem_theta(ctx, in, out);
}

extern "C" w2_status w2_sem_advect(w2_sem_ctx *ctx, const double *in, double *out) {
  if (!ctx || !in || !out || overlaps(in, out, ctx->npts)) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  return sem_advect(ctx, in, out);
}

extern "C" w2_status w2_sem_step(w2_sem_ctx *ctx, int32_t nsteps) {
  if (!ctx || nsteps < 0) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot || !ctx->have_state) return W2_ERR_STATE;
  const long long N = ctx->npts;
  for (int st = 0; st < nsteps; ++st) {
    w2_status r;
    if ((r = sem_theta(ctx, ctx->f, ctx->g)) != W2_OK) return r;        // g = Theta f
    if ((r = sem_advect(ctx, ctx->f, ctx->a)) != W2_OK) return r;       // a = S f
    if ((r = sem_advect(ctx, ctx->g, ctx->b)) != W2_OK) return r;       // b = S g
    SEM_TRY(launch_sem_axpy(N, ctx->a, ctx->tau, ctx->b, nullptr, ctx->t, ctx->stream));  // f~ = a + tau b
    if ((r = sem_theta(ctx, ctx->t, ctx->g)) != W2_OK) return r;        // c = Theta f~
    SEM_TRY(launch_sem_axpy(N, ctx->a, 0.5 * ctx->tau, ctx->b, ctx->g, ctx->f, ctx->stream));  // a + tau/2 (b + c)
    ++ctx->step;
  }
  return W2_OK;
}

extern "C" w2_status w2_sem_observables(w2_sem_ctx *ctx, w2_obs *out, double *n1) {
  if (!ctx || !out) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_pot || !ctx->have_state) return W2_ERR_STATE;
  const int nx = ctx->nx;
  SEM_TRY(launch_sem_marginal(nx, ctx->np, ctx->dx, ctx->f, ctx->w, ctx->xs, ctx->n, ctx->stream));
  SemObsArgs oa{nx, ctx->np, ctx->dx, ctx->hbar, ctx->mass, ctx->gamma, ctx->c_h, ctx->f, ctx->p, ctx->w,
                ctx->vext, ctx->wgrid, ctx->n, ctx->xpart, ctx->obs};
  SEM_TRY(launch_sem_obs(oa, ctx->stream));
  SEM_TRY(cudaMemcpyAsync(ctx->h_obs, ctx->obs, sizeof(double) * (8 + nx), cudaMemcpyDeviceToHost, ctx->stream));
  SEM_TRY(cudaStreamSynchronize(ctx->stream));
  out->mass = ctx->h_obs[0];
  out->energy = ctx->h_obs[1];
  out->purity = ctx->h_obs[2];
  out->entropy_lin = ctx->h_obs[3];
  out->l2norm = ctx->h_obs[4];
  out->step = ctx->step;
  if (n1) memcpy(n1, ctx->h_obs + 8, sizeof(double) * nx);
  return W2_OK;
}

extern "C" void w2_sem_destroy(w2_sem_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  sem_free(ctx);
  delete ctx;
}
