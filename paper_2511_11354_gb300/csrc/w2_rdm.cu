// Occupation numbers of the one-body density matrix and the correlation
// entropy (the paper's appendix on the correlation entropy through the Wigner
// function), and a batched eigensolver for complex Hermitian matrices.
//
//  k_rdm_f1   : f1[a][n] = dx dp sum_{x2, p2} f (FP64 from an FP64 or FP32 state).
//  k_rdm_half : f1 at the half points x_a + dx/2 from its periodic
//               trigonometric interpolant (kernel table from the host).
//  k_rdm_rho  : rho1 dx on the grid by the inverse Wigner transform on the half
//               grid: rho1(x_{mu - nu}, x_{mu + nu}) = dp sum_n f1(x_mu, p_n)
//               e^{-2 pi i (n - nk/2) nu / nx}, nu = (c - b)/2 with c - b the
//               minimal image, mu = b + nu (a half point when b + c is odd);
//               made Hermitian as (rho + rho^H)/2.
//  k_jacobi_herm : one CTA per matrix (in global memory, L2-resident): cyclic
//               Jacobi with the round-robin ordering, n/2 disjoint rotations
//               per round applied as A <- A J then A <- J^H A, at most 40
//               sweeps (it stops when the off-diagonal part falls below 1e-14
//               of the matrix); eigenvalues sorted, largest first.
#include <math.h>

#include "w2_internal.cuh"

namespace w2 {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

template <typename T>
__global__ void k_rdm_f1(const T *f, double *f1, int nx, int nk, double w) {
  const int groups = (nk + 7) / 8, lane = threadIdx.x & 31;
  const int i = blockIdx.x / groups, n = (blockIdx.x % groups) * 8 + (threadIdx.x >> 5);
  if (n >= nk) return;  // whole warp
  double s = 0.0;
  for (int i2 = 0; i2 < nx; ++i2) {
    const T *row = f + (((size_t)i * nx + i2) * nk + n) * nk;
    for (int n2 = lane; n2 < nk; n2 += 32) s += (double)row[n2];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) f1[(size_t)i * nk + n] = s * w;
}

// fh[a][n] = sum_q f1[q][n] kh[(a - q) mod nx]
__global__ void k_rdm_half(const double *f1, const double *kh, double *fh, int nx, int nk) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nx * nk) return;
  const int a = e / nk, n = e - a * nk;
  double s = 0.0;
  for (int q = 0; q < nx; ++q) {
    int j = a - q;
    j += (j < 0) ? nx : 0;
    s += f1[(size_t)q * nk + n] * kh[j];
  }
  fh[e] = s;
}

// One thread per pair b <= c; ph[(d + nx/2) * nk + n] = dp e^{-2 pi i (n - nk/2)(d/2)/nx} for
// d in [-(nx/2), nx - nx/2); rho = dx (raw + raw^H) / 2.
__global__ void k_rdm_rho(const double *f1, const double *fh, const double2 *ph, double2 *rho, int nx, int nk,
                          double dx) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nx * nx) return;
  const int b = e / nx, c = e - b * nx;
  if (c < b) return;
  double2 v[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int r = k ? c : b, s = k ? b : c;  // raw entry (r, s)
    int d = s - r;
    d += (d < 0) ? nx : 0;
    if (d >= (nx + 1) / 2) d -= nx;
    const int s2 = 2 * r + d;
    const double *row;
    if ((s2 & 1) == 0) {
      int mu = s2 / 2;
      mu = ((mu % nx) + nx) % nx;
      row = f1 + (size_t)mu * nk;
    } else {
      int mu = (s2 - 1) / 2;
      mu = ((mu % nx) + nx) % nx;
      row = fh + (size_t)mu * nk;
    }
    const double2 *pr = ph + (size_t)(d + nx / 2) * nk;
    double2 acc = make_double2(0.0, 0.0);
    for (int n = 0; n < nk; ++n) acc = cadd(acc, cscale(row[n], pr[n]));
    v[k] = acc;
  }
  const double2 h = cscale(0.5 * dx, cadd(v[0], cconj(v[1])));
  rho[(size_t)b * nx + c] = h;
  rho[(size_t)c * nx + b] = cconj(h);
}

// Rotation of the Hermitian 2 x 2 block [[app, apq], [conj(apq), aqq]]:
// J = [[c, s e], [-s conj(e), c]] with e = apq / |apq| annihilates the
// off-diagonal entry of J^H A J.
__device__ __forceinline__ void jacobi_rotation(double app, double aqq, double2 apq, double &c, double &s, double2 &e) {
  const double r = hypot(apq.x, apq.y);
  if (r == 0.0) {
    c = 1.0;
    s = 0.0;
    e = make_double2(1.0, 0.0);
    return;
  }
  e = make_double2(apq.x / r, apq.y / r);
  const double tau = (aqq - app) / (2.0 * r);
  const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  c = 1.0 / sqrt(1.0 + t * t);
  s = t * c;
}

constexpr int kMaxSweeps = 40;

// Player at position k of round r of the round-robin over m (even) players.
__device__ __forceinline__ int rr_player(int k, int r, int m) {
  return k == 0 ? 0 : 1 + ((k - 1 - r) % (m - 1) + (m - 1)) % (m - 1);
}

__global__ void __launch_bounds__(512) k_jacobi_herm(double2 *mats, int n, double *eig) {
  extern __shared__ double jsm[];  // m/2 x (c, s, e.x, e.y) and 2 x 32 reduction slots
  double2 *A = mats + (size_t)blockIdx.x * n * n;
  const int m = n + (n & 1), half = m / 2;
  double *rot = jsm, *red = jsm + 4 * half;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    // convergence: off-diagonal vs total Frobenius norm
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < n * n; e += blockDim.x) {
      const double2 a = A[e];
      const double v = a.x * a.x + a.y * a.y;
      tot += v;
      if (e / n != e % n) off += v;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (lane == 0) {
      red[w] = off;
      red[32 + w] = tot;
    }
    __syncthreads();
    off = tot = 0.0;
    for (int q = 0; q < nw; ++q) {
      off += red[q];
      tot += red[32 + q];
    }
    __syncthreads();
    if (!(off > 1e-28 * tot)) break;  // also leaves on NaN
    for (int r = 0; r < m - 1; ++r) {
      for (int k = tid; k < half; k += blockDim.x) {
        int p = rr_player(k, r, m), q = rr_player(m - 1 - k, r, m);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, s = 0.0;
        double2 e = make_double2(1.0, 0.0);
        if (q < n) jacobi_rotation(A[(size_t)p * n + p].x, A[(size_t)q * n + q].x, A[(size_t)p * n + q], c, s, e);
        rot[4 * k] = c;
        rot[4 * k + 1] = s;
        rot[4 * k + 2] = e.x;
        rot[4 * k + 3] = e.y;
      }
      __syncthreads();
      // A <- A J: columns p, q of every row
      for (int it = tid; it < n * half; it += blockDim.x) {
        const int row = it / half, k = it - row * half;
        int p = rr_player(k, r, m), q = rr_player(m - 1 - k, r, m);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        if (q >= n) continue;
        const double c = rot[4 * k], s = rot[4 * k + 1];
        const double2 e = make_double2(rot[4 * k + 2], rot[4 * k + 3]);
        const double2 ap = A[(size_t)row * n + p], aq = A[(size_t)row * n + q];
        A[(size_t)row * n + p] = cadd(cscale(c, ap), cscale(-s, cmul(cconj(e), aq)));
        A[(size_t)row * n + q] = cadd(cscale(s, cmul(e, ap)), cscale(c, aq));
      }
      __syncthreads();
      // A <- J^H A: rows p, q of every column
      for (int it = tid; it < n * half; it += blockDim.x) {
        const int col = it / half, k = it - col * half;
        int p = rr_player(k, r, m), q = rr_player(m - 1 - k, r, m);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        if (q >= n) continue;
        const double c = rot[4 * k], s = rot[4 * k + 1];
        const double2 e = make_double2(rot[4 * k + 2], rot[4 * k + 3]);
        const double2 ap = A[(size_t)p * n + col], aq = A[(size_t)q * n + col];
        A[(size_t)p * n + col] = cadd(cscale(c, ap), cscale(-s, cmul(e, aq)));
        A[(size_t)q * n + col] = cadd(cscale(s, cmul(cconj(e), ap)), cscale(c, aq));
      }
      __syncthreads();
    }
  }
  // eigenvalues, largest first (rank of each diagonal entry; ties by index)
  for (int i = tid; i < n; i += blockDim.x) {
    const double li = A[(size_t)i * n + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = A[(size_t)j * n + j].x;
      rank += (lj > li) || (lj == li && j < i);
    }
    eig[(size_t)blockIdx.x * n + rank] = li;
  }
}

// entropy[0] = sum_{lam > 1e-14 max} lam ln lam / sum lam over the sorted eigenvalues.
__global__ void k_corr_entropy(const double *eig, int n, double *entropy) {
  __shared__ double r0[256], r1[256];
  const double cut = 1e-14 * eig[0];
  double s = 0.0, t = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double l = eig[i];
    t += l;
    if (l > cut && l > 0.0) s += l * log(l);
  }
  r0[threadIdx.x] = s;
  r1[threadIdx.x] = t;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      r0[threadIdx.x] += r0[threadIdx.x + h];
      r1[threadIdx.x] += r1[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) entropy[0] = r0[0] / r1[0];
}

}  // namespace

cudaError_t launch_corr_entropy(const double *eig, int n, double *entropy, cudaStream_t s) {
  k_corr_entropy<<<1, 256, 0, s>>>(eig, n, entropy);
  return cudaGetLastError();
}

cudaError_t launch_rdm_f1(const void *f, int f64, double *f1, int nx, int nk, double dx, double dp, cudaStream_t s) {
  const int grid = nx * ((nk + 7) / 8);
  if (f64)
    k_rdm_f1<double><<<grid, 256, 0, s>>>((const double *)f, f1, nx, nk, dx * dp);
  else
    k_rdm_f1<float><<<grid, 256, 0, s>>>((const float *)f, f1, nx, nk, dx * dp);
  return cudaGetLastError();
}

cudaError_t launch_rdm_rho(const double *f1, const double *kh, double *fh, const double2 *ph, double2 *rho, int nx,
                           int nk, double dx, cudaStream_t s) {
  k_rdm_half<<<(nx * nk + 255) / 256, 256, 0, s>>>(f1, kh, fh, nx, nk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_rdm_rho<<<(nx * nx + 255) / 256, 256, 0, s>>>(f1, fh, ph, rho, nx, nk, dx);
  return cudaGetLastError();
}

cudaError_t launch_jacobi_herm(double2 *mats, int n, int batch, double *eig, cudaStream_t s) {
  if (n < 1 || n > 4096 || batch < 1) return cudaErrorInvalidValue;
  const int half = (n + (n & 1)) / 2;
  const size_t smem = sizeof(double) * (4 * (size_t)half + 64);
  k_jacobi_herm<<<batch, 512, smem, s>>>(mats, n, eig);
  return cudaGetLastError();
}

}  // namespace w2
