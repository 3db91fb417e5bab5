// Reductions of the phase-space state (FP64 or FP32 storage): per-X momentum
// sums for the densities (exact fixed-point sums) and the observables (exact
// fixed-point per-X partials for FP64 states, FP64 in a fixed order
// otherwise).  Repeated calls give identical bits.
#include <math.h>

#include "w2_df.cuh"
#include "w2_blocks.cuh"
#include "w2_internal.cuh"

namespace w2 {

template <typename T, int K>
__global__ void __launch_bounds__(256) k_xsum(const T *f, double *xsum, int nk) {
  __shared__ double red[256];
  xsum_block<T, K>(f, xsum, nk, blockIdx.x, red);
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
// One block per X, one thread per row n1 (lanes on neighbouring rows; each
// thread walks its row in pairs).  p2^2 comes from a table and p1^2 multiplies
// the row sum: three FP64 operations per element, no per-row reductions.
__device__ __forceinline__ void load_pair(const double *p, double &a, double &b) {
  const double2 v = *reinterpret_cast<const double2 *>(p);
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void load_pair(const float *p, double &a, double &b) {
  const float2 v = *reinterpret_cast<const float2 *>(p);
  a = v.x;
  b = v.y;
}

// The same per-X partials for an FP64 state without the FP64 pipe's
// accumulations: every value becomes its exact fixed-point image (integer
// operations, rounded to 2^-49 of the block's largest power of two, as in
// xsum_block), the row sums sum_{n2} f and column sums sum_{n1} f are exact
// int64 sums (so they do not depend on the order), and
//   [0] = sum of the rows,  [1] = sum_n1 p1^2 row(n1) + sum_n2 p2^2 col(n2),
//   [2] = sum f^2 (FP64 squares, exact fixed-point sum).
// One FP64 multiply per element (the square) instead of three operations.
// A block holding Inf or NaN gives NaN partials.  256 threads, nk <= 64.
__global__ void __launch_bounds__(256) k_obs_x_exact(ObsArgs a, const double *f) {
  constexpr int K = 16;  // values per thread (nk^2 <= 16 * 256)
  __shared__ long long img[64 * 65];
  __shared__ long long lred[2][8];
  __shared__ int ired[8];
  __shared__ double dred[8];
  const int nk = a.nk, X = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int n = nk * nk, S = nk + 1;
  const double *fx = f + (size_t)X * n;
  double v[K];
  int e1 = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int e = tid + i * 256;
    v[i] = e < n ? fx[e] : 0.0;
    e1 = max(e1, expo_of(v[i]));
  }
  e1 = __reduce_max_sync(0xffffffffu, e1);
  if (lane == 0) ired[w] = e1;
  __syncthreads();
  e1 = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) e1 = max(e1, ired[k]);
  // |f| < 2^(e1 - 1022), so every square's biased exponent is at most
  // 2 e1 - 1022: the squares' images take that bound as their scale
  const int e2 = max(2 * e1 - 1022, 1);
  const bool bad = e1 == 2047 || e2 > 2046;
  e1 = max(e1, 1);
  long long sq = 0;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int e = tid + i * 256;
    if (e < n) {
      const int r = e / nk, c = e - r * nk;
      img[r * S + c] = fixed_image(v[i], e1);
      sq += fixed_image(v[i] * v[i], e2);
    }
  }
  __syncthreads();
  // rows and columns: four threads (neighbouring lanes) per row or column,
  // each summing every fourth element, then two exchanges
  const int k = tid >> 2, part = tid & 3;
  long long rs = 0, cs = 0;
  if (k < nk) {
    for (int c = part; c < nk; c += 4) rs += img[k * S + c];
    for (int r = part; r < nk; r += 4) cs += img[r * S + k];
  }
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    rs += __shfl_xor_sync(0xffffffffu, rs, o);
    cs += __shfl_xor_sync(0xffffffffu, cs, o);
  }
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  double *xp = a.xpart + (size_t)X * (3 + nk);
  double t1 = 0.0;  // this row's and column's share of sum f p^2
  long long tot = 0;
  if (k < nk && part == 0) {
    const double drow = bad ? nan : ll_to_double_scaled(rs, e1 - 1071);
    const double dcol = bad ? nan : ll_to_double_scaled(cs, e1 - 1071);
    xp[3 + k] = drow;
    const double p = (k - nk / 2) * a.dp;
    t1 = p * p * (drow + dcol);
    tot = rs;
  }
  // block totals: exact for the integers, a fixed tree for the FP64 share
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    t1 += __shfl_xor_sync(0xffffffffu, t1, o);
  }
  if (lane == 0) {
    lred[0][w] = tot;
    lred[1][w] = sq;
    dred[w] = t1;
  }
  __syncthreads();
  if (tid == 0) {
    long long T = 0, Q = 0;
    double s1 = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      T += lred[0][q];
      Q += lred[1][q];
      s1 += dred[q];
    }
    xp[0] = bad ? nan : ll_to_double_scaled(T, e1 - 1071);
    xp[1] = bad ? nan : s1;
    xp[2] = bad ? nan : ll_to_double_scaled(Q, e2 - 1071);
  }
}

// k_obs_x_exact for nk = 64 without the shared-memory image: thread t holds
// column c = t % 64 at rows t / 64 + 4 i (i < 16), so its column sum is its
// own; the row sums come from a transposing butterfly across the warp (after
// it, lane l holds the sum of row index l / 2 over the warp's 32 columns) and
// the two warps of a row group.  The integers are those of k_obs_x_exact; the
// FP64 share of [1] is summed in a fixed order, so repeated calls agree.
__global__ void __launch_bounds__(256) k_obs_x_exact64(ObsArgs a, const double *f) {
  __shared__ long long colp[4][64];
  __shared__ long long rowp[8][16];
  __shared__ long long lred[2][8];
  __shared__ int ired[8];
  __shared__ double dred[8];
  const int X = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5, g = tid >> 6, c = tid & 63;
  const double *fx = f + (size_t)X * 4096;
  long long im[16];
  int e1 = 0;
  {
    double v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      v[i] = fx[tid + 256 * i];
      e1 = max(e1, expo_of(v[i]));
    }
    e1 = __reduce_max_sync(0xffffffffu, e1);
    if (lane == 0) ired[w] = e1;
    __syncthreads();
    e1 = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) e1 = max(e1, ired[k]);
    // |f| < 2^(e1 - 1022): every square's biased exponent is at most 2 e1 - 1022
    const int e2 = max(2 * e1 - 1022, 1);
    const int eb = max(e1, 1);
    long long sq = 0, cs = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      im[i] = fixed_image(v[i], eb);
      cs += im[i];
      sq += fixed_image(v[i] * v[i], e2);
    }
    colp[g][c] = cs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) lred[1][w] = sq;
  }
  // butterfly: at offset o each lane keeps one half of its entries (by lane
  // bit o) and adds the partner's copy of that half
#pragma unroll
  for (int o = 16, h = 8; o >= 2; o >>= 1, h >>= 1) {
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const long long send = hi ? im[j] : im[h + j], keep = hi ? im[h + j] : im[j];
      im[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  im[0] += __shfl_xor_sync(0xffffffffu, im[0], 1);
  if ((lane & 1) == 0) rowp[w][lane >> 1] = im[0];  // row g + 4 (lane / 2), this warp's 32 columns
  __syncthreads();
  const bool bad = e1 == 2047 || 2 * e1 - 1022 > 2046;
  const int eb = max(e1, 1), e2 = max(2 * e1 - 1022, 1);
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  double *xp = a.xpart + (size_t)X * 67;
  double t1 = 0.0;
  long long tot = 0;
  if (tid < 64) {  // row k and column k
    const int k = tid, rg = k & 3, ri = k >> 2;
    const long long rs = rowp[2 * rg][ri] + rowp[2 * rg + 1][ri];
    const long long cl = colp[0][k] + colp[1][k] + colp[2][k] + colp[3][k];
    const double drow = bad ? nan : ll_to_double_scaled(rs, eb - 1071);
    const double dcol = bad ? nan : ll_to_double_scaled(cl, eb - 1071);
    xp[3 + k] = drow;
    const double p = (k - 32) * a.dp;
    t1 = p * p * (drow + dcol);
    tot = rs;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    t1 += __shfl_xor_sync(0xffffffffu, t1, o);
  }
  if (lane == 0) {
    lred[0][w] = tot;
    dred[w] = t1;
  }
  __syncthreads();
  if (tid == 0) {
    long long T = 0, Q = 0;
    double s1 = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      T += lred[0][q];
      Q += lred[1][q];
      s1 += dred[q];
    }
    xp[0] = bad ? nan : ll_to_double_scaled(T, eb - 1071);
    xp[1] = bad ? nan : s1;
    xp[2] = bad ? nan : ll_to_double_scaled(Q, e2 - 1071);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_obs_x(ObsArgs a, const T *f) {
  __shared__ double red[3][8];
  extern __shared__ double psq[];  // [nk] (p_n)^2
  const int nk = a.nk, X = blockIdx.x, nt = blockDim.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = threadIdx.x; c < nk; c += nt) {
    const double p = (c - nk / 2) * a.dp;
    psq[c] = p * p;
  }
  __syncthreads();
  const T *fx = f + (size_t)X * nk * nk;
  double *xp = a.xpart + (size_t)X * (3 + nk);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int r = threadIdx.x; r < nk; r += nt) {
    const T *row = fx + (size_t)r * nk;  // nk is even: pairs stay aligned
    double rv = 0.0;
    for (int c = 0; c < nk; c += 2) {
      double v0, v1;
      load_pair(row + c, v0, v1);
      rv += v0;
      rv += v1;
      s1 = fma(psq[c], v0, s1);
      s1 = fma(psq[c + 1], v1, s1);
      s2 = fma(v0, v0, s2);
      s2 = fma(v1, v1, s2);
    }
    xp[3 + r] = rv;
    s0 += rv;
    s1 = fma(psq[r], rv, s1);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) {
    red[0][w] = s0;
    red[1][w] = s1;
    red[2][w] = s2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int q = 0; q < nt / 32; ++q) t += red[threadIdx.x][q];
    xp[threadIdx.x] = t;
  }
}

// One block per i (256 threads), over the partials of X = (i, i2):
// mid[i][0..7] = sum f, sum f p^2, sum f (V(x_i) + V(x_i2) + gamma W), sum f^2,
// a non-finite flag, n1 and n2 sums at x_i (raw), sum_n f1(x_i, p_n)^2; and
// out[8 + nx + X] = n12.
__global__ void __launch_bounds__(256) k_obs_mid(ObsArgs a, double *mid) {
  __shared__ double red[8][8];
  const int nx = a.nx, nk = a.nk, M = a.M, i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const size_t ld = 3 + (size_t)nk;
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i2 = tid; i2 < nx; i2 += 256) {
    const double *xp = a.xpart + ((size_t)i * nx + i2) * ld;
    int d = i - i2;
    d += (d < 0) ? nx : 0;
    const double vx = a.vext_grid[i] + a.vext_grid[i2] + a.gamma * a.w_fine[(size_t)d * M];
    v[0] += xp[0];
    v[1] += xp[1];
    v[2] += xp[0] * vx;
    v[3] += xp[2];
    if (!isfinite(xp[0]) || !isfinite(xp[1]) || !isfinite(xp[2])) v[4] = 1.0;
    v[5] += xp[0];
    a.out[8 + nx + (size_t)i * nx + i2] = xp[0] * a.dp * a.dp;
  }
  for (int i1 = tid; i1 < nx; i1 += 256) v[6] += a.xpart[((size_t)i1 * nx + i) * ld];
  for (int b = 0; b < nk; b += 64) {  // a quad of lanes per momentum row r
    const int r = b + (tid >> 2);
    const double sr = quad_sum(r < nk, nx, [&](int i2) { return a.xpart[((size_t)i * nx + i2) * ld + 3 + r]; });
    if ((tid & 3) == 0 && r < nk) {
      const double f1 = sr * a.dx * a.dp;
      v[7] += f1 * f1;
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const double t = __shfl_xor_sync(0xffffffffu, v[q], o);
      v[q] = q == 4 ? fmax(v[q], t) : v[q] + t;
    }
    if (lane == 0) red[q][w] = v[q];
  }
  __syncthreads();
  if (tid < 8) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t = tid == 4 ? fmax(t, red[tid][q]) : t + red[tid][q];
    mid[(size_t)i * 8 + tid] = t;
  }
}

// Single block: the Hartree energy and fixed-order sums of the per-i partials.
// out: [0] mass [1] energy [2] purity [3] l2norm [4] nonfinite flag
//      [8 .. 8+nx) n_1 ; [8+nx .. 8+nx+nx*nx) n_12 (written by k_obs_mid)
__global__ void k_obs_final(ObsArgs a, const double *mid) {
  __shared__ double red[6][256];
  extern __shared__ double dyn[];  // n1[nx], n2[nx]
  const int nx = a.nx, M = a.M, tid = threadIdx.x, nt = blockDim.x;
  const double dV = a.dx * a.dx * a.dp * a.dp;
  double *n1 = dyn, *n2 = dyn + nx;
  double m0 = 0, ek = 0, ep = 0, l2 = 0, bad = 0, pur = 0;
  for (int i = tid; i < nx; i += nt) {
    const double *m = mid + (size_t)i * 8;
    m0 += m[0];
    ek += m[1];
    ep += m[2];
    l2 += m[3];
    bad = fmax(bad, m[4]);
    pur += m[7];
    n1[i] = m[5] * a.dx * a.dp * a.dp;
    n2[i] = m[6] * a.dx * a.dp * a.dp;
    a.out[8 + i] = n1[i];
  }
  __syncthreads();
  // Hartree energy
  double eh = 0.0;
  if (a.c_h != 0.0) {
    const double *ker = a.h_fine ? a.h_fine : a.w_fine;
    for (int b = 0; b < nx; b += nt >> 2) {  // a quad of lanes per point i
      const int i = b + (tid >> 2);
      auto conv = [&](const double *n) {
        return quad_sum(i < nx, nx, [&](int q) {
          int d = i - q;
          d += (d < 0) ? nx : 0;
          return ker[(size_t)d * M] * n[q];
        });
      };
      const double va = conv(n1), vb = conv(n2);
      if ((tid & 3) == 0 && i < nx)
        eh += 0.5 * a.c_h * (a.h_fine ? 1.0 : a.gamma * a.dx) * (va * n1[i] + vb * n2[i]) * a.dx;
    }
  }
  red[0][tid] = m0;
  red[1][tid] = ek;
  red[2][tid] = ep;
  red[3][tid] = l2;
  red[4][tid] = eh;
  red[5][tid] = pur;
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
    a.out[5] = a.err ? (double)*a.err : 0.0;
  }
}

cudaError_t launch_obs(const ObsArgs &a, cudaStream_t s) {
  const int nt = a.nk >= 256 ? 256 : 32 * ((a.nk + 31) / 32);  // a thread per row
  if (a.f32)
    k_obs_x<float><<<a.nx * a.nx, nt, sizeof(double) * a.nk, s>>>(a, a.f32);
  else if (a.nk == 64)
    k_obs_x_exact64<<<a.nx * a.nx, 256, 0, s>>>(a, a.f);
  else if (a.nk <= 64)
    k_obs_x_exact<<<a.nx * a.nx, 256, 0, s>>>(a, a.f);
  else
    k_obs_x<double><<<a.nx * a.nx, nt, sizeof(double) * a.nk, s>>>(a, a.f);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double *mid = a.xpart + (size_t)a.nx * a.nx * (3 + a.nk);
  k_obs_mid<<<a.nx, 256, 0, s>>>(a, mid);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_obs_final<<<1, 256, sizeof(double) * 2 * a.nx, s>>>(a, mid);
  return cudaGetLastError();
}

}  // namespace w2
