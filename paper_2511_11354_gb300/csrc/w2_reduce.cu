// Reductions of the phase-space state (FP64 or FP32 storage): per-X momentum
// sums for the densities (exact fixed-point sums) and the observables (FP64,
// fixed order).  Repeated calls give identical bits.
#include <math.h>

#include "w2_df.cuh"
#include "w2_internal.cuh"

namespace w2 {

// Fixed-point image of v: round(|v| 2^(49 - E)) (FP64) or |v| 2^(48 - E)
// (FP32), with sign, where 2^E bounds the block (emax its largest biased
// exponent); the unit is 2^(emax - 1071) for FP64 and 2^(emax - 174) for FP32,
// so that up to 4096 (FP64) or 16384 (FP32) images add up below 2^62.
// Integer operations only.
__device__ __forceinline__ long long fixed_image(double v, int emax) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = (b & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
  const int sh = emax - (e ? e : 1) + 4;  // >= 4
  const long long q = sh < 64 ? (long long)((m + (1ull << (sh - 1))) >> sh) : 0;
  return (b >> 63) ? -q : q;
}

__device__ __forceinline__ long long fixed_image(float v, int emax) {
  const unsigned b = __float_as_uint(v);
  const int e = (int)((b >> 23) & 0xff);
  const unsigned long long m = (unsigned long long)((b & 0x7fffffu) | (e ? 0x800000u : 0u)) << 24;
  const int sh = emax - (e ? e : 1);  // >= 0
  const long long q = sh == 0 ? (long long)m : sh < 64 ? (long long)((m + (1ull << (sh - 1))) >> sh) : 0;
  return (b >> 31) ? -q : q;
}

__device__ __forceinline__ int expo_of(double v) {
  return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff);
}
__device__ __forceinline__ int expo_of(float v) { return (int)((__float_as_uint(v) >> 23) & 0xff); }

// Block maximum exponent and exact fixed-point sum of the n values at base,
// with up to K values per thread held in registers between the two steps
// (the rest, if any, read a second time).
template <typename T, int K>
__device__ __forceinline__ void xsum_hold(const T *f, size_t base, int n, int &em_out, long long &acc_out, int *ired) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  T v[K];
  int em = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int e = tid + i * (int)blockDim.x;
    v[i] = e < n ? f[base + e] : (T)0;
    em = max(em, expo_of(v[i]));
  }
  for (int e = tid + K * (int)blockDim.x; e < n; e += blockDim.x) em = max(em, expo_of(f[base + e]));
  em = __reduce_max_sync(0xffffffffu, em);
  if (lane == 0) ired[w] = em;
  __syncthreads();
  em = 0;
  for (int q = 0; q < nw; ++q) em = max(em, ired[q]);
  em = max(em, 1);
  long long acc = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) acc += fixed_image(v[i], em);
  for (int e = tid + K * (int)blockDim.x; e < n; e += blockDim.x) acc += fixed_image(f[base + e], em);
  em_out = em;
  acc_out = acc;
}

// xsum[X] = sum_P f(X, P), one block per X, as an exact sum of fixed-point
// images (each rounded to 2^-49 / 2^-48 of the block bound, then added
// without rounding): the result does not depend on the order of the
// additions, and neither the FP64 pipe nor a floating-point reduction tree is
// involved.  A block holding Inf or NaN gives NaN.  red: 256 doubles of
// shared memory (used as 32 ints and 32 int64).
// (The sum is exact, so every kernel that uses this gives the same bits.)
template <typename T, int K>
__device__ __forceinline__ void xsum_block(const T *f, double *xsum, int nk, int X, double *red) {
  constexpr int EMAX_NONFINITE = sizeof(T) == 8 ? 2047 : 255;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  const size_t base = (size_t)X * nk * nk;
  const int n = nk * nk;
  int *ired = reinterpret_cast<int *>(red);
  long long *lred = reinterpret_cast<long long *>(red) + 32;
  int em;
  long long acc;
  xsum_hold<T, K>(f, base, n, em, acc, ired);  // one read of the block when n <= K * blockDim
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) lred[w] = acc;
  __syncthreads();
  if (tid == 0) {
    long long tot = 0;
    for (int q = 0; q < nw; ++q) tot += lred[q];
    xsum[X] = em == EMAX_NONFINITE ? __longlong_as_double(0x7ff8000000000000ll)
                                   : ll_to_double_scaled(tot, em - (sizeof(T) == 8 ? 1071 : 174));
  }
  __syncthreads();  // red is reused by the next item of a persistent caller
}

template <typename T, int K>
__global__ void __launch_bounds__(256) k_xsum(const T *f, double *xsum, int nk) {
  __shared__ double red[256];
  xsum_block<T, K>(f, xsum, nk, blockIdx.x, red);
}

// Batched per-X sums over the FP32 states of several instances.
__global__ void k_bxsum(const BXsum *args, const int *off, int n) {
  __shared__ double red[256];
  const int total = off[n];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    int k = 0;
    while (k + 1 < n && off[k + 1] <= item) ++k;
    const BXsum a = args[k];
    xsum_block<float, 16>(a.f, a.xsum, a.nk, item - off[k], red);
    __syncthreads();
  }
}

cudaError_t launch_bxsum(const BXsum *args, const int *off, int n, int grid, cudaStream_t s) {
  k_bxsum<<<grid, 256, 0, s>>>(args, off, n);
  return cudaGetLastError();
}

cudaError_t launch_xsum_f64(int nx, int nk, const double *f, double *xsum, cudaStream_t s) {
  k_xsum<double, 16><<<nx * nx, 256, 0, s>>>(f, xsum, nk);  // nk <= 64: one read
  return cudaGetLastError();
}

cudaError_t launch_xsum_f32(int nx, int nk, const float *f, double *xsum, cudaStream_t s) {
  if (nk * nk > 16 * 256)
    k_xsum<float, 64><<<nx * nx, 256, 0, s>>>(f, xsum, nk);
  else
    k_xsum<float, 16><<<nx * nx, 256, 0, s>>>(f, xsum, nk);
  return cudaGetLastError();
}

// Per-X partials: [0] sum f, [1] sum f (p1^2 + p2^2), [2] sum f^2, [3 + n1] sum_{n2} f.
template <typename T>
__global__ void k_obs_x(ObsArgs a, const T *f) {
  __shared__ double red[3][128];
  const int nk = a.nk, X = blockIdx.x, tid = threadIdx.x;
  const size_t base = (size_t)X * nk * nk;
  double *xp = a.xpart + (size_t)X * (3 + nk);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int r = 0; r < nk; ++r) {
    // row sums: thread tid handles column block; reduce per row below
    double rv = 0.0;
    for (int c = tid; c < nk; c += blockDim.x) {
      const double v = (double)f[base + (size_t)r * nk + c];
      const double p1 = (r - nk / 2) * a.dp, p2 = (c - nk / 2) * a.dp;
      rv += v;
      s1 += v * (p1 * p1 + p2 * p2);
      s2 += v * v;
    }
    s0 += rv;
    red[0][tid] = rv;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
      if (tid < h) red[0][tid] += red[0][tid + h];
      __syncthreads();
    }
    if (tid == 0) xp[3 + r] = red[0][0];
    __syncthreads();
  }
  red[0][tid] = s0;
  red[1][tid] = s1;
  red[2][tid] = s2;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (tid < h) {
      red[0][tid] += red[0][tid + h];
      red[1][tid] += red[1][tid + h];
      red[2][tid] += red[2][tid + h];
    }
    __syncthreads();
  }
  if (tid == 0) {
    xp[0] = red[0][0];
    xp[1] = red[1][0];
    xp[2] = red[2][0];
  }
}

// Single block: fixed-order final reductions.
// out: [0] mass [1] energy [2] purity [3] l2norm [4] nonfinite flag
//      [8 .. 8+nx) n_1 ; [8+nx .. 8+nx+nx*nx) n_12
__global__ void k_obs_final(ObsArgs a) {
  __shared__ double red[6][256];
  extern __shared__ double dyn[];  // n1[nx], n2[nx]
  const int nx = a.nx, nk = a.nk, M = a.M, tid = threadIdx.x, nt = blockDim.x;
  const double dV = a.dx * a.dx * a.dp * a.dp;
  double *n1 = dyn, *n2 = dyn + nx;
  double m0 = 0, ek = 0, ep = 0, l2 = 0, bad = 0;
  for (int X = tid; X < nx * nx; X += nt) {
    const double *xp = a.xpart + (size_t)X * (3 + nk);
    const int i1 = X / nx, i2 = X % nx;
    int d = i1 - i2;
    d += (d < 0) ? nx : 0;
    const double vx = a.vext_grid[i1] + a.vext_grid[i2] + a.gamma * a.w_fine[(size_t)d * M];
    m0 += xp[0];
    ek += xp[1];
    l2 += xp[2];
    ep += xp[0] * vx;
    if (!isfinite(xp[0]) || !isfinite(xp[1]) || !isfinite(xp[2])) bad = 1.0;
    a.out[8 + nx + X] = xp[0] * a.dp * a.dp;
  }
  for (int i = tid; i < nx; i += nt) {
    double s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < nx; ++k) {
      s1 += a.xpart[((size_t)i * nx + k) * (3 + nk)];
      s2 += a.xpart[((size_t)k * nx + i) * (3 + nk)];
    }
    n1[i] = s1 * a.dx * a.dp * a.dp;
    n2[i] = s2 * a.dx * a.dp * a.dp;
    a.out[8 + i] = n1[i];
  }
  __syncthreads();
  // Hartree energy and purity
  double eh = 0.0, pur = 0.0;
  if (a.c_h != 0.0) {
    for (int i = tid; i < nx; i += nt) {
      double va = 0.0, vb = 0.0;
      for (int q = 0; q < nx; ++q) {
        int d = i - q;
        d += (d < 0) ? nx : 0;
        va += (a.h_fine ? a.h_fine : a.w_fine)[(size_t)d * M] * n1[q];
        vb += (a.h_fine ? a.h_fine : a.w_fine)[(size_t)d * M] * n2[q];
      }
      eh += 0.5 * a.c_h * (a.h_fine ? 1.0 : a.gamma * a.dx) * (va * n1[i] + vb * n2[i]) * a.dx;
    }
  }
  for (int e = tid; e < nx * nk; e += nt) {
    const int i1 = e / nk, r = e % nk;
    double s = 0.0;
    for (int i2 = 0; i2 < nx; ++i2) s += a.xpart[((size_t)i1 * nx + i2) * (3 + nk) + 3 + r];
    const double f1 = s * a.dx * a.dp;
    pur += f1 * f1;
  }
  red[0][tid] = m0;
  red[1][tid] = ek;
  red[2][tid] = ep;
  red[3][tid] = l2;
  red[4][tid] = eh;
  red[5][tid] = pur + bad * 0.0;
  __shared__ int sbad;
  if (tid == 0) sbad = 0;
  __syncthreads();
  if (bad != 0.0) sbad = 1;
  for (int h = nt / 2; h > 0; h >>= 1) {
    if (tid < h)
      for (int q = 0; q < 6; ++q) red[q][tid] += red[q][tid + h];
    __syncthreads();
  }
  if (tid == 0) {
    const double mass = red[0][0] * dV;
    const double energy = red[1][0] * dV / (2.0 * a.mass) + red[2][0] * dV + red[4][0];
    const double purity = 2.0 * 3.14159265358979323846 * a.hbar * red[5][0] * a.dx * a.dp;
    const double l2n = sqrt(red[3][0] * dV);
    a.out[0] = mass;
    a.out[1] = energy;
    a.out[2] = purity;
    a.out[3] = l2n;
    a.out[4] = (sbad || !isfinite(mass) || !isfinite(energy) || !isfinite(purity) || !isfinite(l2n)) ? 1.0 : 0.0;
  }
}

cudaError_t launch_obs(const ObsArgs &a, cudaStream_t s) {
  if (a.f32)
    k_obs_x<float><<<a.nx * a.nx, 128, 0, s>>>(a, a.f32);
  else
    k_obs_x<double><<<a.nx * a.nx, 128, 0, s>>>(a, a.f);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_obs_final<<<1, 256, sizeof(double) * 2 * a.nx, s>>>(a);
  return cudaGetLastError();
}

}  // namespace w2
