// Allocation-free variant of the pseudo-difference sweep.
//
// w2_theta_noalloc applies the same operator as w2_theta, but the caller hands
// over the potentials already sampled on the fine points, and the shift-kernel
// tables that w2_theta keeps in its context live in one fixed array in device
// memory that is part of this library image.  Nothing is allocated on any
// call: no cudaMalloc / cudaFree, no host heap.
#include <math.h>

#include <mutex>

#include "w2_internal.cuh"

namespace {

constexpr int kMaxNx = W2_NOALLOC_MAX_NX;
constexpr int kMaxNk = W2_NOALLOC_MAX_NK;
// three kernel tables [nx][2nk-1] (particle 1, particle 2, pair) + sin(pi m/nk), m < 2nk
constexpr size_t kScratchDoubles = (size_t)3 * kMaxNx * (2 * kMaxNk - 1) + 2 * kMaxNk;

// The scratch.  Every device that loads the library holds it until the process
// exits.  In host code its name is only a host-side stand-in: the device
// address comes from cudaGetSymbolAddress in scratch_for_current_device().
static __device__ __align__(256) double g_w2_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_ptr[kMaxDevices];
bool g_ready[kMaxDevices];

__global__ void k_sin_table(double *sintab, int nk) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < 2 * nk) sintab[m] = sinpi((double)m / nk);
}

// Once per device, with that device current: resolve the scratch address and
// set the kernels' shared-memory limits.  Returns nullptr on failure.
double *scratch_for_current_device(w2_status *st) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *st = W2_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ready[dev]) {
    double *p = nullptr;
    if (cudaGetSymbolAddress((void **)&p, g_w2_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      *st = W2_ERR_CUDA;
      return nullptr;
    }
    for (int nk = 8; nk <= kMaxNk; nk += 8)
      if (w2::prepare_kernels_f64(nk) != cudaSuccess) {
        cudaGetLastError();
        *st = W2_ERR_CUDA;
        return nullptr;
      }
    g_ptr[dev] = p;
    g_ready[dev] = true;
  }
  return g_ptr[dev];
}

}  // namespace

extern "C" w2_status w2_theta_noalloc(const w2_config *cfg, const double *u1, const double *u2, const double *u12,
                                      const double *f, double *out, void *cuda_stream) {
  if (!cfg || !u1 || !u2 || !u12 || !f || !out || f == out) return W2_ERR_ARG;
  if (((uintptr_t)f | (uintptr_t)out) & 15) return W2_ERR_ARG;
  if (cfg->nx < 4 || cfg->nk < 2 || (cfg->nk & 1) || !(cfg->L > 0) || !(cfg->hbar > 0) || !isfinite(cfg->L) ||
      !isfinite(cfg->hbar))
    return W2_ERR_ARG;
  if (cfg->precision != W2_F64) return W2_ERR_UNSUPPORTED;
  // sizes beyond the fixed scratch are refused, never truncated
  if (cfg->nx > kMaxNx || cfg->nk > kMaxNk || !w2::nk_supported_f64(cfg->nk)) return W2_ERR_UNSUPPORTED;

  w2_status st = W2_OK;
  double *scratch = scratch_for_current_device(&st);
  if (!scratch) return st;

  const int nx = cfg->nx, nk = cfg->nk, W = 2 * nk - 1;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double *K1 = scratch, *K2 = K1 + (size_t)nx * W, *K12 = K2 + (size_t)nx * W, *sintab = K12 + (size_t)nx * W;

  // Every entry of the tables is rewritten below on each call, so nothing left
  // by an earlier call can leak into this one.
  k_sin_table<<<(2 * nk + 127) / 128, 128, 0, s>>>(sintab, nk);
  if (cudaGetLastError() != cudaSuccess) return W2_ERR_CUDA;

  w2::TabArgs ta;
  ta.nx = nx;
  ta.nk = nk;
  ta.M = 2 * nk;
  ta.dx = cfg->L / nx;
  ta.dp = M_PI * cfg->hbar / cfg->L;
  ta.hbar = cfg->hbar;
  ta.gamma = 1.0;  // the samples are taken as they are
  ta.c_h = 0.0;
  ta.c_xc = 0.0;
  ta.xc_kind = 0;
  ta.pair_mode = 1;  // U(row, l) read straight from the given samples
  ta.xsum = nullptr;
  ta.vext_fine = nullptr;
  ta.d_fine = nullptr;
  ta.sintab = sintab;
  const double *src[3] = {u1, u2, u12};
  double *dst[3] = {K1, K2, K12};
  for (int q = 0; q < 3; ++q) {
    ta.w_fine = src[q];
    ta.K = dst[q];
    if (w2::launch_tables(ta, s) != cudaSuccess) return W2_ERR_CUDA;
  }

  w2::ThetaArgs th;
  th.nx = nx;
  th.in = f;
  th.h = nullptr;
  th.out = out;
  th.xsum = nullptr;
  th.K1 = K1;
  th.K2 = K2;
  th.K12 = K12;
  th.half_tau = 0.0;
  if (w2::launch_theta_f64(nk, 0, th, s) != cudaSuccess) return W2_ERR_CUDA;
  return W2_OK;
}
