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
  float2 *cpdf = nullptr, *wtsdf = nullptr;  // spline tables as double-float pairs (sliced context)
  float2 *fwdc = nullptr, *bwdc = nullptr;   // start-sum coefficients of the piecewise recursion
  // S'^T = E B form of the last two products: slices of [Er | -Ei], [Ei | Er] (rows
  // over 2 Ny) and of alpha [Ei_h | Er_h] (rows over 2 Nyh)
  double *erm = nullptr, *eha = nullptr;
  uint16_t *ermP = nullptr, *eiP = nullptr, *ehaP = nullptr;
  int *ermE = nullptr, *eiE = nullptr, *ehaE = nullptr, ldq = 0;
  long long bsz = 0;  // per-X size of the B slices
  double *dtab = nullptr;  // [2][2nx-1][4h+1] w (W(rho + u) - W(rho - u)), w = 1, 2 (sliced context)
  uint16_t *psiP = nullptr, *utP = nullptr;  // slices of psi (columns) and of the U-Toeplitz rows
  uint16_t *phP2 = nullptr;                  // slices of Ph' (Ph with its last np columns negated)
  double *ph2 = nullptr;
  int *phE2 = nullptr;
  int *psiE = nullptr, *utE = nullptr, Kp5 = 0;
  long long ldpsi = 0;  // row stride of the psi slices: np^2 rounded up to a multiple of 8
  // occupation numbers (allocated by the first w2_sem_occupations)
  double *rf1 = nullptr, *reta = nullptr, *rg = nullptr, *rosc = nullptr, *rphr = nullptr, *rphi = nullptr,
         *reig = nullptr;
  double2 *rrho = nullptr;
  // tensor-core products (W2_F64_SLICED): digit planes and line exponents
  int prec = W2_F64, Kp1 = 0, Kp2 = 0, Kp3 = 0, Kp4 = 0, ldp = 0;
  uint16_t *phrP = nullptr, *phiP = nullptr, *phP = nullptr, *gP = nullptr;
  uint16_t *frP = nullptr, *fcP = nullptr, *tP = nullptr, *bP = nullptr, *sP = nullptr;
  int *phrE = nullptr, *phiE = nullptr, *phE = nullptr, *gE = nullptr;
  int *frE = nullptr, *fcE = nullptr, *tE = nullptr, *bE = nullptr, *sE = nullptr;
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
  void *v[] = {c->erm, c->eha, c->ermP, c->eiP, c->ehaP, c->ermE, c->eiE, c->ehaE, c->fwdc, c->bwdc, c->phP2, c->ph2, c->phE2, c->rf1, c->reta, c->rg, c->rosc, c->rphr, c->rphi, c->reig, c->rrho, c->psiP, c->utP, c->psiE, c->utE, c->dtab, c->cpdf, c->wtsdf, c->phrP, c->phiP, c->phP, c->gP, c->frP, c->fcP, c->tP, c->bP, c->sP,
               c->phrE, c->phiE, c->phE, c->gE, c->frE, c->fcE, c->tE, c->bE, c->sE};
  for (void *q : v)
    if (q) cudaFree(q);
  if (c->h_obs) cudaFreeHost(c->h_obs);
}

extern "C" w2_status w2_sem_create(const w2_sem_config *cfg, void *cuda_stream, w2_sem_ctx **out) {
  if (!cfg || !out) return W2_ERR_ARG;
  *out = nullptr;
  const int nx = cfg->nx, M = cfg->ncell, Q = cfg->nq;
  if (nx < 8 || nx > 1024 || M < 1 || Q < 2 || Q > 32 || (long long)M * Q > 256) return W2_ERR_ARG;
  if (!(cfg->L > 0) || !(cfg->Lp > 0) || !(cfg->dt > 0) || !(cfg->hbar > 0) || !(cfg->mass > 0)) return W2_ERR_ARG;
  if (cfg->xc_kind < 0 || cfg->xc_kind > 2) return W2_ERR_ARG;
  if (cfg->precision != W2_F64 && cfg->precision != W2_F64_SLICED) return W2_ERR_ARG;
  if (cfg->precision == W2_F64_SLICED && nx > 256) return W2_ERR_ARG;  // sliced lines of 2 N_y <= 512 values
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
  ctx->prec = cfg->precision;
  const bool sliced = ctx->prec == W2_F64_SLICED;
  ctx->Kp1 = slice_kp(np); ctx->Kp2 = slice_kp(2 * np); ctx->Kp3 = slice_kp(2 * Nyh); ctx->Kp4 = slice_kp(2 * Ny);
  ctx->ldp = (np + 7) / 8 * 8;
  ctx->Kp5 = slice_kp(2 * nx - 1);
  ctx->ldq = (Nyh + 7) / 8 * 8;
  ctx->bsz = 6LL * ((long long)slice_kp(2 * Ny) * ctx->ldq > (long long)Ny * slice_kp(2 * Nyh)
                        ? (long long)slice_kp(2 * Ny) * ctx->ldq
                        : (long long)Ny * slice_kp(2 * Nyh));
  ctx->ldpsi = ((long long)np * np + 7) / 8 * 8;
  const int Kp1 = ctx->Kp1, Kp2 = ctx->Kp2, Kp3 = ctx->Kp3, Kp4 = ctx->Kp4, ldp = ctx->ldp;
  // two-body chain chunk: about 256 MB of FP64 intermediates (4 GB with the
  // slices, in whole rows of x1 so that a chunk's x1 index is affine in X;
  // large chunks keep the tail of each product's last wave small)
  const double per_x = 8.0 * (2.0 * np * Ny + 2.0 * Nyh * Ny + 2.0 * np * Ny);
  const double per_xs = per_x + 12.0 * ((double)np * Kp1 + (double)Kp1 * ldp + (double)Ny * Kp2 + (double)Ny * Kp3 +
                                        (double)np * Kp4) + 4.0 * (3.0 * np + 2.0 * Ny);
  long long bx;
  if (!sliced) {
    bx = (long long)(256.0 * 1024 * 1024 / per_x);
  } else {
    bx = (long long)(4096.0 * 1024 * 1024 / (per_xs * nx));
    if (bx < 1) bx = 1;
    bx *= nx;
    while (bx > 65535) bx -= nx;
  }
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
  if (e == cudaSuccess) e = w2::dev_alloc((void **)&(ptr), sizeof(*(ptr)) * (size_t)(count));
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
  SEM_ALLOC(ctx->xpart, (long long)nx * nx * (4 + np) + 5 * nx) SEM_ALLOC(ctx->obs, 8 + nx)
  if (sliced) {
    SEM_ALLOC(ctx->psiP, 6LL * ctx->Kp5 * ctx->ldpsi) SEM_ALLOC(ctx->psiE, (long long)np * np)
    SEM_ALLOC(ctx->utP, 6LL * 2 * nx * ctx->Kp5) SEM_ALLOC(ctx->utE, 2 * nx)
    SEM_ALLOC(ctx->phP2, 6LL * 2 * Nyh * Kp2) SEM_ALLOC(ctx->ph2, 4LL * Nyh * np) SEM_ALLOC(ctx->phE2, 2 * Nyh)
    SEM_ALLOC(ctx->cpdf, nx) SEM_ALLOC(ctx->wtsdf, 4 * np) SEM_ALLOC(ctx->fwdc, 28) SEM_ALLOC(ctx->bwdc, 28) SEM_ALLOC(ctx->dtab, 2LL * (2 * nx - 1) * (4 * ctx->h + 1))
    SEM_ALLOC(ctx->phrP, 6LL * Ny * Kp1) SEM_ALLOC(ctx->phiP, 6LL * Ny * Kp1) SEM_ALLOC(ctx->phP, 6LL * 2 * Nyh * Kp2)
    SEM_ALLOC(ctx->gP, 6LL * 2 * nx * np * Kp1)
    SEM_ALLOC(ctx->frP, bx * 6 * np * Kp1) SEM_ALLOC(ctx->fcP, bx * 6 * Kp1 * ldp) SEM_ALLOC(ctx->tP, bx * 6 * Ny * Kp2)
    SEM_ALLOC(ctx->bP, bx * ctx->bsz) SEM_ALLOC(ctx->sP, bx * 6 * np * Kp4)
    SEM_ALLOC(ctx->erm, 2LL * np * Ny) SEM_ALLOC(ctx->eha, 2LL * np * Nyh)
    SEM_ALLOC(ctx->ermP, 6LL * np * Kp4) SEM_ALLOC(ctx->eiP, 6LL * np * Kp4) SEM_ALLOC(ctx->ehaP, 6LL * np * Kp3)
    SEM_ALLOC(ctx->ermE, np) SEM_ALLOC(ctx->eiE, np) SEM_ALLOC(ctx->ehaE, np)
    SEM_ALLOC(ctx->phrE, Ny) SEM_ALLOC(ctx->phiE, Ny) SEM_ALLOC(ctx->phE, 2 * Nyh)
    SEM_ALLOC(ctx->gE, 2LL * nx * np) SEM_ALLOC(ctx->frE, bx * np) SEM_ALLOC(ctx->fcE, bx * np)
    SEM_ALLOC(ctx->tE, bx * Ny) SEM_ALLOC(ctx->bE, bx * Ny) SEM_ALLOC(ctx->sE, bx * np)
  }
#undef SEM_ALLOC
  if (e == cudaSuccess) e = w2::host_alloc((void **)&ctx->h_obs, sizeof(double) * (8 + nx));
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
  std::vector<float2> cpdf(nx), wtsdf(4 * np);
  auto pair = [](double v) { const float h = (float)v; return make_float2(h, (float)(v - (double)h)); };
  for (int i = 0; i < nx; ++i) cpdf[i] = pair(cp[i]);
  for (int j = 0; j < 4 * np; ++j) wtsdf[j] = pair(6.0 * wts[j]);  // the double-float solve runs on eta / 6
  std::vector<float2> fwdc(28), bwdc(28);
  {
    const double cs = 2.0 - sqrt(3.0);
    double pw = 1.0;  // c*^k
    for (int k = 0; k < 28; ++k) {
      bwdc[k] = pair((k & 1) ? -pw : pw);
      fwdc[k] = pair((k & 1) ? -pw * cs : pw * cs);
      pw *= cs;
    }
  }
  if (sliced) {
    up(ctx->fwdc, fwdc.data(), sizeof(float2) * 28);
    up(ctx->bwdc, bwdc.data(), sizeof(float2) * 28);
    up(ctx->cpdf, cpdf.data(), sizeof(float2) * nx);
    up(ctx->wtsdf, wtsdf.data(), sizeof(float2) * 4 * np);
  }
  SemTabArgs ta{nx, M, Q, np, ctx->h, ctx->dx, ctx->width, ctx->hbar, ctx->Lp, ctx->p, ctx->centre, ctx->cheb,
                ctx->osc, ctx->psi, ctx->phir, ctx->phii, ctx->ph, ctx->eh, ctx->eier};
  if (e == cudaSuccess) e = launch_sem_osc(ta, ctx->stream);
  if (e == cudaSuccess) e = launch_sem_tables(ta, ctx->stream);
  if (sliced) {  // static slices: Phi rows (K = np), Ph and Ph' rows (K = 2 np), [Er | -Ei] and [Ei | Er] rows (K = 2 Ny)
    auto rows = [&](const double *in, int L, int K, int Kp, uint16_t *P, int *E) {
      SliceArgs sa{L, K, Kp, 0, in, K, 1, 0, 0, P, (long long)L * Kp, 0, E, 0, 1, 1, nullptr, nx, ctx->h, 0};
      if (e == cudaSuccess) e = launch_slice(0, 0, sa, ctx->stream);
    };
    rows(ctx->phir, Ny, np, Kp1, ctx->phrP, ctx->phrE);
    rows(ctx->phii, Ny, np, Kp1, ctx->phiP, ctx->phiE);
    rows(ctx->ph, 2 * Nyh, 2 * np, Kp2, ctx->phP, ctx->phE);
    if (e == cudaSuccess) e = launch_sem_negcols(2 * Nyh, 2 * np, np, ctx->ph, ctx->ph2, ctx->stream);
    rows(ctx->ph2, 2 * Nyh, 2 * np, Kp2, ctx->phP2, ctx->phE2);
    if (e == cudaSuccess) e = launch_sem_erm(np, Ny, ctx->eier, ctx->erm, ctx->stream);
    rows(ctx->erm, np, 2 * Ny, Kp4, ctx->ermP, ctx->ermE);
    rows(ctx->eier, np, 2 * Ny, Kp4, ctx->eiP, ctx->eiE);
    // psi as columns (i, j) over the offset d: the B operand of the table product
    SliceArgs sp{np * np, 2 * nx - 1, ctx->Kp5, (int)ctx->ldpsi, ctx->psi, 1, (long long)np * np, 0, 0, ctx->psiP,
                 (long long)ctx->Kp5 * ctx->ldpsi, 0, ctx->psiE, 0, 1, 1, nullptr, nx, ctx->h, 0};
    if (e == cudaSuccess) e = launch_slice(1, 0, sp, ctx->stream);
  }
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
  if (ctx->prec == W2_F64_SLICED) {
    const double alpha = gamma * ctx->dx * ctx->dx / (M_PI * M_PI * ctx->hbar * ctx->hbar * ctx->hbar);
    const long long n = 2LL * ctx->np * ctx->Nyh;
    SEM_TRY(launch_sem_scale(n, alpha, ctx->eh + (long long)ctx->np * 2 * ctx->Nyh, ctx->eha, ctx->stream));
    SliceArgs sa{ctx->np, 2 * ctx->Nyh, ctx->Kp3, 0, ctx->eha, 2 * ctx->Nyh, 1, 0, 0, ctx->ehaP,
                 (long long)ctx->np * ctx->Kp3, 0, ctx->ehaE, 0, 1, 1, nullptr, nx, ctx->h, 0};
    SEM_TRY(launch_slice(0, 0, sa, ctx->stream));
    // D_V weights of the two-body chain, w (W(rho + u) - W(rho - u)) for w = 1 and 2
    const int nr = 2 * nx - 1, nu = 4 * ctx->h + 1;
    std::vector<double> dt(2LL * nr * nu);
    for (int ir = 0; ir < nr; ++ir)
      for (int iu = 0; iu < nu; ++iu) {
        const int rho = ir - (nx - 1), u = iu - 2 * ctx->h;
        const double D = wg[rho + u + W0] - wg[rho - u + W0];
        dt[(long long)ir * nu + iu] = D;
        dt[(long long)nr * nu + (long long)ir * nu + iu] = 2.0 * D;
      }
    SEM_TRY(cudaMemcpyAsync(ctx->dtab, dt.data(), sizeof(double) * dt.size(), cudaMemcpyHostToDevice, ctx->stream));
    SEM_TRY(cudaStreamSynchronize(ctx->stream));
  }
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
static w2_status sem_theta_sliced(w2_sem_ctx *ctx, const double *in, double *out);

static w2_status sem_theta(w2_sem_ctx *ctx, const double *in, double *out) {
  if (ctx->prec == W2_F64_SLICED) return sem_theta_sliced(ctx, in, out);
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

// The same operator from exact slices on the BF16 tensor cores (w2_gemms.cu).
// Layouts chosen so that every sliced line runs along the contraction index:
// T^T = Phi F^T ([Nyh][2np]: [Tr | Ti] for y2 >= 0), A^T = T^T Ph^T and
// T^T Ph'^T ([Ny][2Nyh]), B = w D (.) A sliced along [re | im] x y2,
// S'^T = [[Er | -Ei] B | [Ei | Er] B] ([np][2Nyh]), out += alpha [Ei_h | Er_h] S'
// -- the sums over y2 before those over y1, which halves the last product;
// the one-body products use F's row slices (F G2^T, and T^T) and its column
// slices (G1 F).
static w2_status sem_theta_sliced(w2_sem_ctx *ctx, const double *in, double *out) {
  const int nx = ctx->nx, np = ctx->np, Ny = ctx->Ny, Nyh = ctx->Nyh;
  const int Kp1 = ctx->Kp1, Kp2 = ctx->Kp2, Kp3 = ctx->Kp3, Kp4 = ctx->Kp4, ldp = ctx->ldp;
  const long long np2 = (long long)np * np, nX = (long long)nx * nx;
  cudaStream_t s = ctx->stream;
  SEM_TRY(launch_sem_marginal(nx, np, ctx->dx, in, ctx->w, ctx->xs, ctx->n, s));
  SemPotArgs pa{nx, ctx->xc_kind, ctx->dx, ctx->c_h, ctx->c_xc, ctx->n, ctx->vext, ctx->wgrid, ctx->U, ctx->ut};
  SEM_TRY(launch_sem_potential(pa, s));
  // products over K in pieces of at most 256 (multiples of 32), adding after the first
  auto gemm_k = [&](GemmSArgs a, int K, int b_kn) -> cudaError_t {
    const int beta0 = a.beta;
    for (int k0 = 0; k0 < K; k0 += 256) {
      a.k0 = k0;
      a.K = K - k0 < 256 ? K - k0 : 256;
      a.beta = k0 ? 1 : beta0;
      const cudaError_t e = launch_gemms(b_kn, a, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  {  // G[2 nx][np*np] = ut[2 nx][2 nx - 1] psi[2 nx - 1][np*np], from slices
    const int Kp5 = ctx->Kp5;
    SliceArgs su{2 * nx, 2 * nx - 1, Kp5, 0, ctx->ut, 2 * nx - 1, 1, 0, 0, ctx->utP, 2LL * nx * Kp5, 0, ctx->utE, 0,
                 1, 1, nullptr, nx, ctx->h, 0};
    SEM_TRY(launch_slice(0, 0, su, s));
    GemmSArgs gt{2 * nx, (int)np2, 2 * nx - 1, 0, ctx->utP, Kp5, 2LL * nx * Kp5, 0, 0, ctx->utE, 0, 0, ctx->psiP,
                 ctx->ldpsi, (long long)Kp5 * ctx->ldpsi, 0, 0, ctx->psiE, 0, 0, ctx->G, np2, 0, 0, 0, 1, 1};
    SEM_TRY(gemm_k(gt, 2 * nx - 1, 1));
    SliceArgs sa{2 * nx * np, np, Kp1, 0, ctx->G, np, 1, 0, 0, ctx->gP, 2LL * nx * np * Kp1, 0, ctx->gE, 0, 1, 1,
                 nullptr, nx, ctx->h, 0};
    SEM_TRY(launch_slice(0, 0, sa, s));
  }
  const long long frS = 6LL * np * Kp1, fcS = 6LL * Kp1 * ldp, tS = 6LL * Ny * Kp2,
                  sS = 6LL * np * Kp4;
  for (long long x0 = 0; x0 < nX; x0 += ctx->bx) {
    const int nb = (int)((nX - x0) < ctx->bx ? (nX - x0) : ctx->bx);
    const long long i10 = x0 / nx;
    const double *F = in + x0 * np2;
    SliceArgs fr{np, np, Kp1, 0, F, np, 1, np2, 0, ctx->frP, (long long)np * Kp1, frS, ctx->frE, np, nb, 1,
                 nullptr, nx, ctx->h, 0};
    SEM_TRY(launch_slice(0, 0, fr, s));
    SliceArgs fc{np, np, Kp1, ldp, F, 1, np, np2, 0, ctx->fcP, (long long)Kp1 * ldp, fcS, ctx->fcE, np, nb, 1,
                 nullptr, nx, ctx->h, 0};
    SEM_TRY(launch_slice(1, 0, fc, s));
    // out_X = G1[i1] F_X  (B = F's column slices, row-major planes)
    GemmSArgs a1{np, np, np, 0, ctx->gP + i10 * np * Kp1, Kp1, 2LL * nx * np * Kp1, (long long)np * Kp1, 0,
                 ctx->gE + i10 * np, np, 0, ctx->fcP, ldp, (long long)Kp1 * ldp, nx * fcS, fcS, ctx->fcE,
                 (long long)nx * np, np, out + x0 * np2, np, nx * np2, np2, 0, nb, nx};
    SEM_TRY(gemm_k(a1, np, 1));
    // out_X += F_X G2[i2]^T
    GemmSArgs a2{np, np, np, 0, ctx->frP, Kp1, (long long)np * Kp1, nx * frS, frS, ctx->frE, (long long)nx * np, np,
                 ctx->gP + (long long)nx * np * Kp1, Kp1, 2LL * nx * np * Kp1, 0, (long long)np * Kp1,
                 ctx->gE + (long long)nx * np, 0, np, out + x0 * np2, np, nx * np2, np2, 1, nb, nx};
    SEM_TRY(gemm_k(a2, np, 0));
    if (ctx->gamma == 0.0) continue;
    // T^T_X = [Phr F_X^T | Phi F_X^T] on the rows y2 >= 0 only: F is real, so
    // the row -y2 is the conjugate [Tr | -Ti] of the row y2
    const long long hK1 = (long long)ctx->h * Kp1;
    GemmSArgs t{Nyh, np, np, 0, ctx->phrP + hK1, Kp1, (long long)Ny * Kp1, 0, 0, ctx->phrE + ctx->h, 0, 0, ctx->frP,
                Kp1, (long long)np * Kp1, frS, 0, ctx->frE, np, 0, ctx->cT, 2 * np, (long long)Nyh * 2 * np, 0, 0, nb,
                1};
    SEM_TRY(gemm_k(t, np, 0));
    t.A = ctx->phiP + hK1;
    t.Ae = ctx->phiE + ctx->h;
    t.C = ctx->cT + np;
    SEM_TRY(gemm_k(t, np, 0));
    SliceArgs ts{Nyh, 2 * np, Kp2, 0, ctx->cT, 2 * np, 1, (long long)Nyh * 2 * np, 0, ctx->tP, (long long)Nyh * Kp2,
                 tS, ctx->tE, Nyh, nb, 1, nullptr, nx, ctx->h, 0};
    SEM_TRY(launch_slice(0, 0, ts, s));
    // A^T_X rows y2 >= 0: T^T Ph^T; rows y2 = -y < 0: [Tr | -Ti](y) Ph^T = T^T(y) Ph'^T
    // (Ph' = Ph with its last np columns negated), written upwards from row h - 1
    GemmSArgs aa{Nyh, 2 * Nyh, 2 * np, 0, ctx->tP, Kp2, (long long)Nyh * Kp2, tS, 0, ctx->tE, Nyh, 0, ctx->phP, Kp2,
                 2LL * Nyh * Kp2, 0, 0, ctx->phE, 0, 0, ctx->cA + (long long)ctx->h * 2 * Nyh, 2 * Nyh,
                 (long long)Ny * 2 * Nyh, 0, 0, nb, 1};
    SEM_TRY(gemm_k(aa, 2 * np, 0));
    if (ctx->h > 0) {
      GemmSArgs an{ctx->h, 2 * Nyh, 2 * np, 0, ctx->tP + Kp2, Kp2, (long long)Nyh * Kp2, tS, 0, ctx->tE + 1, Nyh, 0,
                   ctx->phP2, Kp2, 2LL * Nyh * Kp2, 0, 0, ctx->phE2, 0, 0,
                   ctx->cA + (long long)(ctx->h - 1) * 2 * Nyh, -2LL * Nyh, (long long)Ny * 2 * Nyh, 0, 0, nb, 1};
      SEM_TRY(gemm_k(an, 2 * np, 0));
    }
    // B(k, y1) = w D (.) A over k = [re | im] x y2, sliced along k (columns y1)
    SliceArgs bs{Nyh, 2 * Ny, Kp4, ctx->ldq, ctx->cA, 2 * Nyh, 1, (long long)Ny * 2 * Nyh, 0, ctx->bP,
                 (long long)Kp4 * ctx->ldq, ctx->bsz, ctx->bE, Nyh, nb, 1, ctx->dtab, nx, ctx->h, (int)x0};
    SEM_TRY(launch_slice_dstack(bs, s));
    // S'^T_X = [[Er | -Ei] B | [Ei | Er] B]  ([np][2 Nyh]: S'r^T, S'i^T)
    for (int blk = 0; blk < 2; ++blk) {
      GemmSArgs sg{np, Nyh, 2 * Ny, 0, blk ? ctx->eiP : ctx->ermP, Kp4, (long long)np * Kp4, 0, 0,
                   blk ? ctx->eiE : ctx->ermE, 0, 0, ctx->bP, ctx->ldq, (long long)Kp4 * ctx->ldq, ctx->bsz, 0,
                   ctx->bE, Nyh, 0, ctx->cS + blk * Nyh, 2 * Nyh, (long long)np * 2 * Nyh, 0, 0, nb, 1};
      SEM_TRY(gemm_k(sg, 2 * Ny, 1));
    }
    SliceArgs ss{np, 2 * Nyh, Kp3, 0, ctx->cS, 2 * Nyh, 1, (long long)np * 2 * Nyh, 0, ctx->sP, (long long)np * Kp3,
                 sS, ctx->sE, np, nb, 1, nullptr, nx, ctx->h, 0};
    SEM_TRY(launch_slice(0, 0, ss, s));
    // out_X += alpha [Ei_h | Er_h] S'_X
    GemmSArgs fo{np, np, 2 * Nyh, 0, ctx->ehaP, Kp3, (long long)np * Kp3, 0, 0, ctx->ehaE, 0, 0, ctx->sP, Kp3,
                 (long long)np * Kp3, sS, 0, ctx->sE, np, 0, out + x0 * np2, np, np2, 0, 1, nb, 1};
    SEM_TRY(gemm_k(fo, 2 * Nyh, 0));
  }
  return W2_OK;
}

// The sliced context shifts in double-float pairs (k_sem_adv_df), the
// FP64-pipe context in FP64.
static w2_status sem_advect(w2_sem_ctx *ctx, const double *in, double *out) {
  const int df = ctx->prec == W2_F64_SLICED;
  SemAdvArgs aa{ctx->nx, ctx->np, ctx->C, in, ctx->t, ctx->cp, ctx->k0, ctx->wts, ctx->cpdf, ctx->wtsdf, ctx->fwdc,
                ctx->bwdc};
  SEM_TRY(launch_sem_adv(0, aa, ctx->stream, df));
  aa.in = ctx->t;
  aa.out = out;
  SEM_TRY(launch_sem_adv(1, aa, ctx->stream, df));
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
  SemObsArgs oa{nx, ctx->np, ctx->dx, ctx->hbar, ctx->mass, ctx->gamma, ctx->c_h, ctx->f, ctx->p, ctx->w,
                ctx->vext, ctx->wgrid, ctx->xpart, ctx->obs};
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

extern "C" w2_status w2_sem_occupations(w2_sem_ctx *ctx, double *occ, double *entropy) {
  if (!ctx) return W2_ERR_ARG;
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->have_state) return W2_ERR_STATE;
  const int nx = ctx->nx, np = ctx->np, Q = ctx->Q;
  cudaStream_t s = ctx->stream;
  if (!ctx->rrho) {
    cudaError_t e = cudaSuccess;
#define SEM_ALLOC(ptr, count) \
  if (e == cudaSuccess) e = w2::dev_alloc((void **)&(ptr), sizeof(*(ptr)) * (size_t)(count));
    SEM_ALLOC(ctx->rf1, (long long)nx * np) SEM_ALLOC(ctx->reta, (long long)(nx + 2) * np)
    SEM_ALLOC(ctx->rg, (long long)(2 * nx - 1) * np) SEM_ALLOC(ctx->rosc, 2LL * nx * Q)
    SEM_ALLOC(ctx->rphr, (long long)(2 * nx - 1) * np) SEM_ALLOC(ctx->rphi, (long long)(2 * nx - 1) * np)
    SEM_ALLOC(ctx->reig, nx + 1) SEM_ALLOC(ctx->rrho, (long long)nx * nx)
#undef SEM_ALLOC
    if (e != cudaSuccess) {
      cudaGetLastError();
      return W2_ERR_OOM;
    }
    // transform rows at half steps: Phi_j(m dx / 2), m = -(nx - 1) .. nx - 1
    SemTabArgs ta{nx, ctx->M, Q, np, nx - 1, 0.5 * ctx->dx, ctx->width, ctx->hbar, ctx->Lp, ctx->p, ctx->centre,
                  ctx->cheb, ctx->rosc, nullptr, ctx->rphr, ctx->rphi, nullptr, nullptr, nullptr};
    SEM_TRY(launch_sem_osc(ta, s));
    SEM_TRY(launch_sem_phi(ta, s));
  }
  SEM_TRY(launch_sem_rdm(nx, np, ctx->dx, ctx->f, ctx->w, ctx->cp, ctx->rf1, ctx->reta, ctx->rg, ctx->rphr, ctx->rphi,
                         ctx->rrho, s));
  SEM_TRY(w2::launch_herm_eigvals(ctx->rrho, nx, 1, ctx->reig, s));
  SEM_TRY(w2::launch_corr_entropy(ctx->reig, nx, ctx->reig + nx, s));
  if (occ) SEM_TRY(cudaMemcpyAsync(occ, ctx->reig, sizeof(double) * nx, cudaMemcpyDeviceToHost, s));
  if (entropy) SEM_TRY(cudaMemcpyAsync(entropy, ctx->reig + nx, sizeof(double), cudaMemcpyDeviceToHost, s));
  SEM_TRY(cudaStreamSynchronize(s));
  return W2_OK;
}

extern "C" void w2_sem_destroy(w2_sem_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  sem_free(ctx);
  delete ctx;
}
