// Learned form, host side: the MLP object (parameters, Adam state,
// activations) and its C entry points; the step integration lives in
// w2_api.cu.  Kernels in w2_mlp.cu.
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "w2_internal.cuh"

using namespace w2;

struct w2_mlp {
  int nk = 0, din = 0, H = 0, dout = 0, maxrows = 0;
  int kind = 0;  // 0: the pair term per point; 1: the pair kernel per distance
  // kernel-network training scratch (allocated by the first training step)
  uint16_t *kx = nullptr;
  float *ky = nullptr, *kt = nullptr;
  double *kres = nullptr, *kg = nullptr, *kpart = nullptr, *h_kpart = nullptr;
  double *kd = nullptr;  // dL/dy of w2_pair_kernel_loss_grad [maxrows][nk]
  int krows = 0;
  cudaStream_t stream = nullptr;
  size_t np = 0, offW[4] = {}, offb[4] = {};
  int fin[4] = {}, fout[4] = {};
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  uint16_t *pb = nullptr;
  float *Z[3] = {}, *dZ[3] = {};
  uint16_t *A[3] = {}, *dZb[3] = {};
  float *Y = nullptr, *dY = nullptr;
  uint16_t *dYb = nullptr;
  double *part = nullptr, *h_part = nullptr;
  float s_f = 1.f, s_f1 = 1.f, s_y = 1.f;
  int t = 0;
};

namespace w2 {
int mlp_din(const w2_mlp *m) { return m->din; }
int mlp_kind(const w2_mlp *m) { return m->kind; }
int mlp_nk(const w2_mlp *m) { return m->nk; }
int mlp_maxrows(const w2_mlp *m) { return m->maxrows; }
float mlp_scale(const w2_mlp *m, int which) { return which == 0 ? m->s_f : which == 1 ? m->s_f1 : m->s_y; }
float *mlp_out(w2_mlp *m) { return m->Y; }
double *mlp_part(w2_mlp *m) { return m->part; }
double *mlp_hpart(w2_mlp *m) { return m->h_part; }

// y[rows][dout] = s * MLP(x), x bf16 [rows][din]: each layer one pipelined
// GEMM with the bias / SiLU / scale epilogue fused; with keep_z the FP32
// pre-activations of the hidden layers stay in m->Z for the backward pass.
static cudaError_t mlp_forward_impl(w2_mlp *m, const uint16_t *x, int rows, float *y, float s, bool keep_z,
                                    cudaStream_t st) {
  const void *in = x;
  for (int l = 0; l < 4; ++l) {
    GemmArgs a;
    memset(&a, 0, sizeof(a));
    a.A = in;
    a.sam = m->fin[l];
    a.sak = 1;
    a.B = m->pb + m->offW[l];
    a.sbk = m->fout[l];
    a.sbn = 1;
    a.M = rows;
    a.N = m->fout[l];
    a.K = m->fin[l];
    a.bias = m->p + m->offb[l];
    if (l < 3) {
      a.epi = GEMM_BIAS_SILU;
      a.out_f32 = keep_z ? m->Z[l] : nullptr;
      a.out_bf16 = m->A[l];
    } else {
      a.epi = GEMM_BIAS_SCALE;
      a.scale = s;
      a.out_f32 = y;
    }
    cudaError_t e = launch_gemm_fwd(a, st);
    if (e != cudaSuccess) return e;
    in = m->A[l < 3 ? l : 2];
  }
  return cudaSuccess;
}

cudaError_t mlp_forward(w2_mlp *m, const uint16_t *x, int rows, float *y, float s, cudaStream_t st) {
  return mlp_forward_impl(m, x, rows, y, s, false, st);
}

static cudaError_t mlp_forward_train(w2_mlp *m, const uint16_t *x, int rows, float *y, float s, cudaStream_t st) {
  return mlp_forward_impl(m, x, rows, y, s, true, st);
}
}  // namespace w2

#define WM_TRY(call)                 \
  do {                               \
    cudaError_t e_ = (call);         \
    if (e_ != cudaSuccess) {         \
      w2::note_cuda_error(e_);       \
      return W2_ERR_CUDA;            \
    }                                \
  } while (0)

static void mlp_free(w2_mlp *m) {
  void *ptrs[] = {m->p, m->g, m->m, m->v, m->pb, m->Y, m->dY, m->dYb, m->part, m->kx, m->ky, m->kt, m->kres, m->kg,
                  m->kpart, m->kd};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  for (int l = 0; l < 3; ++l) {
    if (m->Z[l]) cudaFree(m->Z[l]);
    if (m->dZ[l]) cudaFree(m->dZ[l]);
    if (m->A[l]) cudaFree(m->A[l]);
    if (m->dZb[l]) cudaFree(m->dZb[l]);
  }
  if (m->h_part) cudaFreeHost(m->h_part);
  if (m->h_kpart) cudaFreeHost(m->h_kpart);
}

extern "C" void w2_mlp_destroy(w2_mlp *m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  mlp_free(m);
  delete m;
}

// Counter-based uniform in [-1, 1) (SplitMix64 finaliser) for the default init.
static double hash_uniform(uint64_t i) {
  uint64_t z = (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return 2.0 * (double)(z >> 11) * (1.0 / 9007199254740992.0) - 1.0;
}

static w2_status mlp_create(int kind, int32_t nk, int32_t hidden, int32_t max_rows, void *cuda_stream, w2_mlp **out) {
  if (!out) return W2_ERR_ARG;
  *out = nullptr;
  if (nk < 2 || nk > 128 || hidden < 16 || hidden > 4096 || (hidden & 15) || max_rows < 1 || max_rows > (1 << 20))
    return W2_ERR_ARG;
  w2_mlp *m = new (std::nothrow) w2_mlp();
  if (!m) return W2_ERR_OOM;
  m->kind = kind;
  m->nk = nk;
  m->H = hidden;
  if (kind == 0) {
    m->dout = nk * nk;
    m->din = ((nk * nk + 2 * nk + 2 * kMlpHarmonics) + 31) / 32 * 32;
  } else {
    m->dout = nk;
    m->din = (2 * kMlpHarmonics + 31) / 32 * 32;
  }
  m->maxrows = max_rows;
  m->stream = (cudaStream_t)cuda_stream;
  const int fin[4] = {m->din, hidden, hidden, hidden}, fout[4] = {hidden, hidden, hidden, m->dout};
  size_t off = 0;
  for (int l = 0; l < 4; ++l) {
    m->fin[l] = fin[l];
    m->fout[l] = fout[l];
    m->offW[l] = off;
    off += (size_t)fin[l] * fout[l];
    m->offb[l] = off;
    off += fout[l];
  }
  m->np = off;
  cudaError_t e = cudaSuccess;
  const size_t R = (size_t)max_rows;
#define WM_ALLOC(ptr, bytes) \
  if (e == cudaSuccess) e = dev_alloc((void **)&(ptr), (bytes));
  WM_ALLOC(m->p, 4 * m->np) WM_ALLOC(m->g, 4 * m->np) WM_ALLOC(m->m, 4 * m->np) WM_ALLOC(m->v, 4 * m->np)
  WM_ALLOC(m->pb, 2 * m->np)
  for (int l = 0; l < 3; ++l) {
    WM_ALLOC(m->Z[l], 4 * R * hidden) WM_ALLOC(m->dZ[l], 4 * R * hidden)
    WM_ALLOC(m->A[l], 2 * R * hidden) WM_ALLOC(m->dZb[l], 2 * R * hidden)
  }
  WM_ALLOC(m->Y, 4 * R * m->dout) WM_ALLOC(m->dY, 4 * R * m->dout) WM_ALLOC(m->dYb, 2 * R * m->dout)
  WM_ALLOC(m->part, sizeof(double) * 512)
#undef WM_ALLOC
  if (e == cudaSuccess) e = host_alloc((void **)&m->h_part, sizeof(double) * 512);
  if (e == cudaSuccess) e = cudaMemset(m->m, 0, 4 * m->np);
  if (e == cudaSuccess) e = cudaMemset(m->v, 0, 4 * m->np);
  if (e != cudaSuccess) {
    mlp_free(m);
    delete m;
    return e == cudaErrorMemoryAllocation ? W2_ERR_OOM : W2_ERR_CUDA;
  }
  // default initialisation: weights uniform in +-sqrt(3 / fan_in) (unit
  // variance through each layer), biases zero
  std::vector<float> h(m->np, 0.0f);
  for (int l = 0; l < 4; ++l) {
    const double a = sqrt(3.0 / fin[l]);
    for (size_t i = 0; i < (size_t)fin[l] * fout[l]; ++i) h[m->offW[l] + i] = (float)(a * hash_uniform(m->offW[l] + i));
  }
  w2_status st = w2_mlp_set_params(m, h.data());
  if (st != W2_OK) {
    mlp_free(m);
    delete m;
    return st;
  }
  *out = m;
  return W2_OK;
}

extern "C" w2_status w2_mlp_create(int32_t nk, int32_t hidden, int32_t max_rows, void *cuda_stream, w2_mlp **out) {
  return mlp_create(0, nk, hidden, max_rows, cuda_stream, out);
}

extern "C" w2_status w2_mlp_create_kernel(int32_t nk, int32_t hidden, int32_t max_nx, void *cuda_stream,
                                          w2_mlp **out) {
  if (max_nx > 1024) return W2_ERR_ARG;
  return mlp_create(1, nk, hidden, max_nx, cuda_stream, out);
}

extern "C" size_t w2_mlp_param_count(const w2_mlp *m) { return m ? m->np : 0; }
extern "C" int32_t w2_mlp_input_dim(const w2_mlp *m) { return m ? m->din : 0; }

extern "C" w2_status w2_mlp_set_params(w2_mlp *m, const float *params) {
  if (!m || !params) return W2_ERR_ARG;
  WM_TRY(cudaMemcpyAsync(m->p, params, 4 * m->np, cudaMemcpyHostToDevice, m->stream));
  WM_TRY(launch_f2bf(m->p, m->pb, m->np, m->stream));
  WM_TRY(cudaStreamSynchronize(m->stream));
  return W2_OK;
}

extern "C" w2_status w2_mlp_get_params(w2_mlp *m, float *params) {
  if (!m || !params) return W2_ERR_ARG;
  WM_TRY(cudaMemcpyAsync(params, m->p, 4 * m->np, cudaMemcpyDeviceToHost, m->stream));
  WM_TRY(cudaStreamSynchronize(m->stream));
  return W2_OK;
}

extern "C" w2_status w2_mlp_set_scales(w2_mlp *m, float s_f, float s_f1, float s_y) {
  if (!m || !(s_f > 0) || !(s_f1 > 0) || !(s_y > 0) || !isfinite(s_f) || !isfinite(s_f1) || !isfinite(s_y))
    return W2_ERR_ARG;
  m->s_f = s_f;
  m->s_f1 = s_f1;
  m->s_y = s_y;
  return W2_OK;
}

extern "C" w2_status w2_mlp_forward(w2_mlp *m, const void *x, int32_t rows, float *y) {
  if (!m || !x || !y || rows < 1 || rows > m->maxrows) return W2_ERR_ARG;
  WM_TRY(mlp_forward(m, (const uint16_t *)x, rows, y, 1.0f, m->stream));
  return W2_OK;
}

// Forward and backward of the mean squared error 1/(rows dout) sum (y - t)^2;
// leaves the gradient in m->g and the loss in *loss (synchronises).
static w2_status forward_backward(w2_mlp *m, const uint16_t *x, const float *target, int rows, double *loss) {
  cudaStream_t s = m->stream;
  WM_TRY(mlp_forward_train(m, x, rows, m->Y, 1.0f, s));
  const size_t ny = (size_t)rows * m->dout;
  WM_TRY(launch_mse(m->Y, target, m->dY, m->part, ny, (float)(2.0 / (double)ny), s));
  WM_TRY(launch_f2bf(m->dY, m->dYb, ny, s));
  const float *dz = m->dY;
  const uint16_t *dzb = m->dYb;
  for (int l = 3; l >= 0; --l) {
    const int fi = m->fin[l], fo = m->fout[l];
    const void *act = l == 0 ? (const void *)x : (const void *)m->A[l - 1];
    const long long ld_act = l == 0 ? m->din : m->H;
    // dW_l[k][n] = sum_r act[r][k] dZ_l[r][n]
    GemmArgs gw;
    memset(&gw, 0, sizeof(gw));
    gw.A = act;
    gw.sam = 1;
    gw.sak = ld_act;
    gw.B = dzb;
    gw.sbk = fo;
    gw.sbn = 1;
    gw.M = fi;
    gw.N = fo;
    gw.K = rows;
    gw.epi = GEMM_STORE;
    gw.out_f32 = m->g + m->offW[l];
    WM_TRY(launch_gemm(gw, s));
    WM_TRY(launch_colsum(dz, m->g + m->offb[l], rows, fo, s));
    if (l == 0) break;
    // dZ_{l-1}[r][k] = (sum_n dZ_l[r][n] W_l[k][n]) silu'(Z_{l-1}[r][k])
    GemmArgs gb;
    memset(&gb, 0, sizeof(gb));
    gb.A = dzb;
    gb.sam = fo;
    gb.sak = 1;
    gb.B = m->pb + m->offW[l];
    gb.sbk = 1;
    gb.sbn = fo;
    gb.M = rows;
    gb.N = fi;
    gb.K = fo;
    gb.epi = GEMM_DSILU;
    gb.aux = m->Z[l - 1];
    gb.out_f32 = m->dZ[l - 1];
    gb.out_bf16 = m->dZb[l - 1];
    WM_TRY(launch_gemm(gb, s));
    dz = m->dZ[l - 1];
    dzb = m->dZb[l - 1];
  }
  WM_TRY(cudaMemcpyAsync(m->h_part, m->part, sizeof(double) * 256, cudaMemcpyDeviceToHost, s));
  WM_TRY(cudaStreamSynchronize(s));
  double L = 0.0;
  for (int q = 0; q < 256; ++q) L += m->h_part[q];
  if (loss) *loss = L / (double)ny;
  return isfinite(L) ? W2_OK : W2_ERR_NONFINITE;
}

extern "C" w2_status w2_mlp_gradients(w2_mlp *m, const void *x, const float *target, int32_t rows, float *grads,
                                      double *loss) {
  if (!m || !x || !target || rows < 1 || rows > m->maxrows) return W2_ERR_ARG;
  w2_status st = forward_backward(m, (const uint16_t *)x, target, rows, loss);
  if (st != W2_OK) return st;
  if (grads) {
    WM_TRY(cudaMemcpyAsync(grads, m->g, 4 * m->np, cudaMemcpyDeviceToHost, m->stream));
    WM_TRY(cudaStreamSynchronize(m->stream));
  }
  return W2_OK;
}

extern "C" w2_status w2_mlp_train_step(w2_mlp *m, const void *x, const float *target, int32_t rows, float lr,
                                       double *loss) {
  if (!m || !x || !target || rows < 1 || rows > m->maxrows || !(lr > 0)) return W2_ERR_ARG;
  w2_status st = forward_backward(m, (const uint16_t *)x, target, rows, loss);
  if (st != W2_OK) return st;
  m->t += 1;
  WM_TRY(launch_adam(m->p, m->g, m->m, m->v, m->pb, m->np, lr, 0.9f, 0.999f, m->t, 1e-8f, m->stream));
  return W2_OK;
}

// The kernel network's outputs y for every distance, the residuals of its
// predicted term on the rows, their per-row sums and the per-row gradients
// with respect to the kernel (everything the loss and its gradient need);
// *loss and *inv_p2 = 1 / sum |P|^2 on the host.  Synchronises.
static w2_status pairk_forward(w2_ctx *ctx, w2_mlp *m, const double *f, const double *p, const int32_t *dr,
                               int32_t rows, double *loss, double *inv_p2) {
  const int nx = ctx->nx, nk = ctx->nk;
  cudaStream_t s = m->stream;
  if (rows > m->krows) {
    void *old[] = {m->kres, m->kg, m->kpart};
    for (void *q : old)
      if (q) cudaFree(q);
    if (m->h_kpart) cudaFreeHost(m->h_kpart);
    m->kres = m->kg = m->kpart = m->h_kpart = nullptr;
    m->krows = 0;
    cudaError_t e = dev_alloc((void **)&m->kres, sizeof(double) * (size_t)rows * nk * nk);
    if (e == cudaSuccess) e = dev_alloc((void **)&m->kg, sizeof(double) * (size_t)rows * nk);
    if (e == cudaSuccess) e = dev_alloc((void **)&m->kpart, sizeof(double) * 2 * (size_t)rows);
    if (e == cudaSuccess) e = host_alloc((void **)&m->h_kpart, sizeof(double) * 2 * (size_t)rows);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return W2_ERR_OOM;
    }
    m->krows = rows;
  }
  if (!m->kx) {
    cudaError_t e = dev_alloc((void **)&m->kx, sizeof(uint16_t) * (size_t)m->maxrows * m->din);
    if (e == cudaSuccess) e = dev_alloc((void **)&m->ky, sizeof(float) * (size_t)m->maxrows * m->dout);
    if (e == cudaSuccess) e = dev_alloc((void **)&m->kt, sizeof(float) * (size_t)m->maxrows * m->dout);
    if (e != cudaSuccess) {  // all three or none: a later call tests kx alone
      void *part[] = {m->kx, m->ky, m->kt};
      for (void *q : part)
        if (q) cudaFree(q);
      m->kx = nullptr;
      m->ky = m->kt = nullptr;
      cudaGetLastError();
      return W2_ERR_OOM;
    }
  }
  const float inv_sy = 1.0f / m->s_y;
  WM_TRY(launch_rfeat(m->kx, nx, m->din, s));
  WM_TRY(mlp_forward(m, m->kx, nx, m->ky, 1.0f, s));
  WM_TRY(launch_pairk_grad(f, p, (const int *)dr, rows, m->ky, nx, nk, inv_sy, m->kres, m->kg, m->kpart, s));
  WM_TRY(cudaMemcpyAsync(m->h_kpart, m->kpart, sizeof(double) * 2 * rows, cudaMemcpyDeviceToHost, s));
  WM_TRY(cudaStreamSynchronize(s));
  double r2 = 0.0, p2 = 0.0;
  for (int b = 0; b < rows; ++b) {
    r2 += m->h_kpart[2 * b];
    p2 += m->h_kpart[2 * b + 1];
  }
  if (!(p2 > 0.0) || !isfinite(r2)) return W2_ERR_NONFINITE;
  *loss = r2 / p2;
  *inv_p2 = 1.0 / p2;
  return W2_OK;
}

static bool pairk_args_ok(const w2_ctx *ctx, const w2_mlp *m, const void *f, const void *p, const void *dr,
                          int32_t rows) {
  return ctx && m && f && p && dr && rows >= 1 && m->kind == 1 && m->nk == ctx->nk && ctx->nx <= m->maxrows;
}

extern "C" w2_status w2_pair_kernel_train_step(w2_ctx *ctx, w2_mlp *m, const double *f, const double *p,
                                               const int32_t *dr, int32_t rows, float lr, double *loss) {
  if (!pairk_args_ok(ctx, m, f, p, dr, rows) || !(lr > 0)) return W2_ERR_ARG;
  double L = 0.0, inv_p2 = 0.0;
  w2_status st = pairk_forward(ctx, m, f, p, dr, rows, &L, &inv_p2);
  if (st != W2_OK) return st;
  if (loss) *loss = L;
  WM_TRY(launch_pairk_target(m->ky, m->kg, (const int *)dr, rows, ctx->nx, ctx->nk, 1.0f / m->s_y, inv_p2, m->kt,
                             nullptr, m->stream));
  return w2_mlp_train_step(m, m->kx, m->kt, ctx->nx, lr, nullptr);
}

extern "C" w2_status w2_pair_kernel_loss_grad(w2_ctx *ctx, w2_mlp *m, const double *f, const double *p,
                                              const int32_t *dr, int32_t rows, double *loss, float *y, double *dldy) {
  if (!pairk_args_ok(ctx, m, f, p, dr, rows) || !loss) return W2_ERR_ARG;
  const int nx = ctx->nx, nk = ctx->nk;
  double L = 0.0, inv_p2 = 0.0;
  w2_status st = pairk_forward(ctx, m, f, p, dr, rows, &L, &inv_p2);
  if (st != W2_OK) return st;
  *loss = L;
  cudaStream_t s = m->stream;
  if (dldy) {
    if (!m->kd && dev_alloc((void **)&m->kd, sizeof(double) * (size_t)m->maxrows * nk) != cudaSuccess) {
      m->kd = nullptr;
      cudaGetLastError();
      return W2_ERR_OOM;
    }
    WM_TRY(launch_pairk_target(m->ky, m->kg, (const int *)dr, rows, nx, nk, 1.0f / m->s_y, inv_p2, m->kt, m->kd, s));
    WM_TRY(cudaMemcpyAsync(dldy, m->kd, sizeof(double) * (size_t)nx * nk, cudaMemcpyDeviceToHost, s));
  }
  if (y) WM_TRY(cudaMemcpyAsync(y, m->ky, sizeof(float) * (size_t)nx * nk, cudaMemcpyDeviceToHost, s));
  WM_TRY(cudaStreamSynchronize(s));
  return W2_OK;
}
