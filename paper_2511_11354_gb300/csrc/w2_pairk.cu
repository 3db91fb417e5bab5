// Learned form with the two-body term's structure: the network predicts the
// shift kernel of the pair term instead of the term itself.
//
// The two-body term of Eq. two_body_FSM is linear in f with a kernel that
// depends only on the pair distance r = x1 - x2:
//   Theta_12 f(X, n1, n2) = sum_{j >= 1} K(r, j) [F(n1 + j, n2 - j) - F(n1 - j, n2 + j)],
// F = f(X, ., .), zero outside the momentum window.  A kernel network maps
// the harmonics of r (sin, cos (2 pi m r / L), m = 1..8) to s_y K^(r, j),
// j = 0 .. nk - 1 (j = 0 unused).  It is trained on snapshots of exact
// trajectories: the loss is the relative squared error of Theta_K^ F against
// the exact term over a batch of spatial points, and its gradient with
// respect to the network's outputs is handed to the network's own backward
// and Adam kernels (w2_learned.cu) as a target.  In the step, the predicted
// table K^[d][2 nk - 1] (d = r / dx) takes the place of the exact pair table
// in the ordinary pseudo-difference sweep.
#include "w2_internal.cuh"

namespace w2 {
namespace {

__device__ __forceinline__ uint16_t f2bf_rn(float v) {
  const uint32_t u = __float_as_uint(v);
  return (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

// x[d][e]: sin(2 pi m d / nx) (e = 2 (m - 1)), cos (e = 2 (m - 1) + 1), m = 1..8, then zeros.
__global__ void k_rfeat(uint16_t *x, int nx, int din) {
  const int d = blockIdx.x;
  for (int e = threadIdx.x; e < din; e += blockDim.x) {
    float v = 0.f;
    if (e < 2 * kMlpHarmonics) {
      const int m = e / 2 + 1;
      const float u = 2.f * (float)(m * d) / (float)nx;
      v = (e & 1) ? cospif(u) : sinpif(u);
    }
    x[(size_t)d * din + e] = f2bf_rn(v);
  }
}

// The kernel of row b's distance: k[j] = y[d][j] / s_y, j = 1 .. nk - 1 (k[0] = 0).
__device__ __forceinline__ void load_kernel(double *k, const float *y, int d, int nk, float inv_sy) {
  for (int j = threadIdx.x; j < nk; j += blockDim.x) k[j] = j ? (double)y[(size_t)d * nk + j] * inv_sy : 0.0;
}

// Theta_K F (n1, n2) for the kernel k and the block F in shared memory.
__device__ __forceinline__ double pair_apply(const double *F, const double *k, int nk, int n1, int n2) {
  double s = 0.0;
  for (int j = 1; j < nk; ++j) {
    const double a = (n1 + j < nk && n2 - j >= 0) ? F[(n1 + j) * nk + n2 - j] : 0.0;
    const double b = (n1 - j >= 0 && n2 + j < nk) ? F[(n1 - j) * nk + n2 + j] : 0.0;
    s = fma(k[j], a - b, s);
  }
  return s;
}

// Row b: res = Theta_K^ F - P, and the row's sums of res^2 and P^2 (fixed order).
__global__ void k_pairk_resid(const double *f, const double *p, const int *dr, const float *y, float inv_sy, int nk,
                              double *res, double *part) {
  extern __shared__ double shp[];
  const int b = blockIdx.x, P = nk * nk;
  double *F = shp, *k = shp + P;
  __shared__ double r2[256], p2[256];
  for (int e = threadIdx.x; e < P; e += blockDim.x) F[e] = f[(size_t)b * P + e];
  load_kernel(k, y, dr[b], nk, inv_sy);
  __syncthreads();
  double a2 = 0.0, b2 = 0.0;
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    const double t = p[(size_t)b * P + e];
    const double v = pair_apply(F, k, nk, e / nk, e % nk) - t;
    res[(size_t)b * P + e] = v;
    a2 = fma(v, v, a2);
    b2 = fma(t, t, b2);
  }
  r2[threadIdx.x] = a2;
  p2[threadIdx.x] = b2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int q = 0; q < (int)blockDim.x; ++q) {
      sa += r2[q];
      sb += p2[q];
    }
    part[2 * b] = sa;
    part[2 * b + 1] = sb;
  }
}

// Row b: g[b][j] = sum_{n1, n2} res(n1, n2) [F(n1 + j, n2 - j) - F(n1 - j, n2 + j)], j = 1..nk-1.
__global__ void k_pairk_rowgrad(const double *f, const double *res, int nk, double *g) {
  extern __shared__ double shp[];
  const int b = blockIdx.x, P = nk * nk;
  double *F = shp, *R = shp + P;
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    F[e] = f[(size_t)b * P + e];
    R[e] = res[(size_t)b * P + e];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nk; j += blockDim.x) {
    double s = 0.0;
    if (j > 0)
      for (int n1 = 0; n1 < nk; ++n1)
        for (int n2 = 0; n2 < nk; ++n2) {
          const double a = (n1 + j < nk && n2 - j >= 0) ? F[(n1 + j) * nk + n2 - j] : 0.0;
          const double c = (n1 - j >= 0 && n2 + j < nk) ? F[(n1 - j) * nk + n2 + j] : 0.0;
          s = fma(R[n1 * nk + n2], a - c, s);
        }
    g[(size_t)b * nk + j] = s;
  }
}

// The network's target for its mean squared error 1/(nx nk) sum (y - t)^2,
// whose gradient is then 2 (y - t) / (nx nk) = dL/dy:
//   t[d][j] = y[d][j] - (nx nk / 2) dL/dy[d][j],
//   dL/dy = (1 / s_y) 2 / sum P^2 * sum_{rows b with distance d} g[b][j]  (rows in order).
// With dldy given, dL/dy itself is written there (FP64) as well.
__global__ void k_pairk_target(const float *y, const double *g, const int *dr, int rows, int nx, int nk, float inv_sy,
                               double inv_p2, float *t, double *dldy) {
  const int d = blockIdx.x;
  for (int j = threadIdx.x; j < nk; j += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < rows; ++b)
      if (dr[b] == d) s += g[(size_t)b * nk + j];
    const double v = 2.0 * s * inv_p2 * (double)inv_sy;
    t[(size_t)d * nk + j] = y[(size_t)d * nk + j] - (float)(0.5 * nx * nk * v);
    if (dldy) dldy[(size_t)d * nk + j] = v;
  }
}

// The predicted pair table K^[d][nk - 1 + j] = y[d][j] / s_y, odd in j, 0 at j = 0.
__global__ void k_pairk_table(const float *y, int nk, float inv_sy, double *K) {
  const int d = blockIdx.x, W = 2 * nk - 1;
  for (int j = threadIdx.x; j < nk; j += blockDim.x) {
    const double v = j ? (double)y[(size_t)d * nk + j] * inv_sy : 0.0;
    K[(size_t)d * W + nk - 1 + j] = v;
    K[(size_t)d * W + nk - 1 - j] = -v;
  }
}

}  // namespace

cudaError_t launch_rfeat(uint16_t *x, int nx, int din, cudaStream_t s) {
  k_rfeat<<<nx, 32, 0, s>>>(x, nx, din);
  return cudaGetLastError();
}

cudaError_t launch_pairk_table(const float *y, int nx, int nk, float inv_sy, double *K, cudaStream_t s) {
  k_pairk_table<<<nx, 64, 0, s>>>(y, nk, inv_sy, K);
  return cudaGetLastError();
}

cudaError_t launch_pairk_grad(const double *f, const double *p, const int *dr, int rows, const float *y, int nx, int nk,
                              float inv_sy, double *res, double *g, double *part, cudaStream_t s) {
  const size_t P = (size_t)nk * nk;
  if (sizeof(double) * (2 * P) > 64 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_pairk_resid, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_pairk_rowgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  if (e != cudaSuccess) return e;
  k_pairk_resid<<<rows, 256, sizeof(double) * (P + nk), s>>>(f, p, dr, y, inv_sy, nk, res, part);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_pairk_rowgrad<<<rows, 64, sizeof(double) * 2 * P, s>>>(f, res, nk, g);
  (void)nx;
  return cudaGetLastError();
}

cudaError_t launch_pairk_target(const float *y, const double *g, const int *dr, int rows, int nx, int nk, float inv_sy,
                                double inv_p2, float *t, double *dldy, cudaStream_t s) {
  k_pairk_target<<<nx, 64, 0, s>>>(y, g, dr, rows, nx, nk, inv_sy, inv_p2, t, dldy);
  return cudaGetLastError();
}

}  // namespace w2
