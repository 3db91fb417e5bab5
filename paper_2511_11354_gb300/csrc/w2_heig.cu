// Eigenvalues of complex Hermitian matrices for the occupation numbers (the
// paper's appendix on the correlation entropy: the occupations are the
// eigenvalues of the one-body density matrix on the grid).
//
//  k_hh_tridiag : one cluster of 8 CTAs per matrix, the rows dealt out
//                 cyclically (row r lives in the shared memory of CTA r % 8).
//                 Householder reduction to tridiagonal form: at step k the
//                 column x = A[k+1:, k] is sent to every CTA, the reflector
//                 H = I - beta u u^H, u = x + e^{i arg x_0} |x| e_1,
//                 beta = 1 / (|x| (|x| + |x_0|)), maps x to a multiple of e_1
//                 of modulus |x|, and the trailing block becomes
//                 H A H = A - u w^H - w u^H with p = beta A u,
//                 w = p - (beta u^H p / 2) u.  Two cluster barriers a step.
//                 A Hermitian tridiagonal matrix with off-diagonals e_k has the
//                 eigenvalues of the real one with |e_k| (a diagonal unitary
//                 similarity), so only the moduli are kept: d and |e| are left
//                 in the first row of the matrix's storage.
//  k_tridiag_eigs : one warp per eigenvalue: multisection of the Gershgorin
//                 interval, 32 Sturm counts a round (the number of negative
//                 pivots of T - x I = L D L^T counts the eigenvalues below x),
//                 until the bracket is a few ulps wide.
#include <cooperative_groups.h>
#include <math.h>

#include "w2_internal.cuh"

namespace cg = cooperative_groups;

namespace w2 {
namespace {

constexpr int kHhCluster = 8;
constexpr int kHhThreads = 512;
constexpr int kHhWarps = kHhThreads / 32;
constexpr int kBisectRounds = 64;  // 33-fold shrink a round: 11 reach FP64 resolution

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Sum over the block in a fixed order (every CTA of a cluster that runs it on
// the same data gets the same bits).  All threads call it; all get the sum.
__device__ __forceinline__ double block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < kHhWarps; ++q) s += red[q];
  __syncthreads();
  return s;
}

// Shared memory: rows [nlmax][n], xb, pb, ub, wb [n] (double2); dd [n],
// ee [n], part [8], red [32] (double).
__global__ void __cluster_dims__(kHhCluster, 1, 1) __launch_bounds__(kHhThreads, 1)
    k_hh_tridiag(double2 *mats, int n) {
  extern __shared__ __align__(16) double2 hsm[];
  cg::cluster_group cl = cg::this_cluster();
  constexpr int G = kHhCluster;
  const int g = (int)cl.block_rank();
  double2 *A = mats + (size_t)(blockIdx.x / G) * n * n;
  const int nl = (n - g + G - 1) / G, nlmax = (n + G - 1) / G;
  double2 *R = hsm, *xb = R + (size_t)nlmax * n, *pb = xb + n, *ub = pb + n, *wb = ub + n;
  double *dd = reinterpret_cast<double *>(wb + n), *ee = dd + n, *part = ee + n, *red = part + G;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

  for (int i = tid; i < nl * n; i += kHhThreads) {
    const int j = i / n, c = i - j * n;
    R[i] = A[(size_t)(g + j * G) * n + c];
  }
  cl.sync();  // every CTA of the cluster has started before the first remote store

  for (int k = 0; k < n; ++k) {
    // column k, rows k .. n-1, to every CTA
    const int j0 = k > g ? (k - g + G - 1) / G : 0;
    for (int i = tid; i < (nl - j0) * G; i += kHhThreads) {
      const int j = j0 + i / G, dst = i % G;
      cl.map_shared_rank(xb, dst)[g + j * G] = R[(size_t)j * n + k];
    }
    cl.sync();

    const int m = n - 1 - k;
    double s = 0.0;
    for (int c = k + 1 + tid; c < n; c += kHhThreads) s += xb[c].x * xb[c].x + xb[c].y * xb[c].y;
    s = block_sum(s, red);
    const double nrm = sqrt(s);
    if (tid == 0) {
      dd[k] = xb[k].x;
      if (m >= 1) ee[k] = nrm;
    }
    // below 1e-150 the column is left as it is: the dropped part is below
    // 1e-150 of an entry, and beta stays finite
    const bool refl = m >= 2 && nrm > 1e-150;
    const int j1 = k + 1 > g ? (k + 1 - g + G - 1) / G : 0;  // first local row >= k + 1
    double beta = 0.0;
    if (refl) {
      const double2 x0 = xb[k + 1];
      const double a0 = hypot(x0.x, x0.y);
      const double2 ph = a0 > 0.0 ? make_double2(x0.x / a0, x0.y / a0) : make_double2(1.0, 0.0);
      beta = 1.0 / (nrm * (nrm + a0));
      for (int c = k + 1 + tid; c < n; c += kHhThreads) {
        double2 u = xb[c];
        if (c == k + 1) u = make_double2(u.x + ph.x * nrm, u.y + ph.y * nrm);
        ub[c] = u;
      }
      __syncthreads();
      // p_r = beta sum_c A[r][c] u_c over the local rows, sent to every CTA
      double dot = 0.0;
      for (int j = j1 + wid; j < nl; j += kHhWarps) {
        const double2 *row = R + (size_t)j * n;
        double2 acc = make_double2(0.0, 0.0);
        for (int c = k + 1 + lane; c < n; c += 32) {
          const double2 t = cmul(row[c], ub[c]);
          acc.x += t.x;
          acc.y += t.y;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
          acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        const int r = g + j * G;
        const double2 p = make_double2(beta * acc.x, beta * acc.y);
        if (lane < G) cl.map_shared_rank(pb, lane)[r] = p;
        if (lane == 0) dot += ub[r].x * p.x + ub[r].y * p.y;  // Re(conj(u_r) p_r)
      }
      dot = block_sum(dot, red);
      if (tid < G) cl.map_shared_rank(part, tid)[g] = dot;
    }
    cl.sync();

    if (refl) {
      double upu = 0.0;
      for (int q = 0; q < G; ++q) upu += part[q];
      const double K = 0.5 * beta * upu;
      for (int c = k + 1 + tid; c < n; c += kHhThreads)
        wb[c] = make_double2(pb[c].x - K * ub[c].x, pb[c].y - K * ub[c].y);
      __syncthreads();
      // A[r][c] -= u_r conj(w_c) + w_r conj(u_c), local rows r, columns c > k
      const int cols = m;
      for (int i = tid; i < (nl - j1) * cols; i += kHhThreads) {
        const int jj = i / cols, c = k + 1 + (i - jj * cols);
        const int j = j1 + jj, r = g + j * G;
        const double2 a = cmulc(ub[r], wb[c]), b = cmulc(wb[r], ub[c]);
        double2 &e = R[(size_t)j * n + c];
        e = make_double2(e.x - a.x - b.x, e.y - a.y - b.y);
      }
      __syncthreads();
    }
  }
  // the last remote store preceded the last cluster barrier; d and |e| go to
  // the first row of the matrix's storage (no CTA reads the matrix any more)
  if (g == 0) {
    double *out = reinterpret_cast<double *>(A);
    for (int i = tid; i < n; i += kHhThreads) {
      out[i] = dd[i];
      out[n + i] = i < n - 1 ? ee[i] : 0.0;
    }
  }
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x: the
// negative pivots of the LDL^T factorisation of T - x I, a pivot of modulus
// below pivmin replaced by -pivmin.
__device__ __forceinline__ int sturm_count(const double *d, const double *e, int n, double x, double pivmin) {
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int cnt = q < 0.0;
  for (int i = 1; i < n; ++i) {
    const double ei = e[i - 1];
    q = (d[i] - x) - (ei * ei) / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

// Warp gw = b * n + j finds the j-th largest eigenvalue of matrix b.  The
// Sturm counts are bound by the FP64 pipe (a division per pivot), so each
// block is one warp: the warps spread over all SMs.
__global__ void __launch_bounds__(32) k_tridiag_eigs(const double2 *mats, int n, int batch, double *eig) {
  const int lane = threadIdx.x & 31;
  const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (gw >= (long long)batch * n) return;  // whole warps
  const int b = (int)(gw / n), j = (int)(gw - (long long)b * n);
  const double *d = reinterpret_cast<const double *>(mats + (size_t)b * n * n), *e = d + n;
  // Gershgorin interval and the pivot floor
  double lo = INFINITY, hi = -INFINITY, emax2 = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i < n - 1) emax2 = fmax(emax2, e[i] * e[i]);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    emax2 = fmax(emax2, __shfl_xor_sync(0xffffffffu, emax2, o));
  }
  const double pivmin = 2.2250738585072014e-308 * fmax(1.0, emax2);
  const double eps = 2.220446049250313e-16;
  const double tnorm = fmax(fabs(lo), fabs(hi));
  lo -= 2.0 * eps * tnorm * n + 2.0 * pivmin;
  hi += 2.0 * eps * tnorm * n + 2.0 * pivmin;
  const int i = n - 1 - j;  // ascending index: count(lo) <= i < count(hi)
  for (int it = 0; it < kBisectRounds; ++it) {
    if (!(hi - lo > 2.0 * eps * fmax(fabs(lo), fabs(hi)) + pivmin)) break;  // uniform over the warp
    const double x = lo + (hi - lo) * ((lane + 1) / 33.0);
    const unsigned below = __ballot_sync(0xffffffffu, sturm_count(d, e, n, x, pivmin) <= i);
    const int t = __popc(below);  // the lanes whose point lies at or below the eigenvalue
    const double xl = __shfl_sync(0xffffffffu, x, t > 0 ? t - 1 : 0);
    const double xh = __shfl_sync(0xffffffffu, x, t < 32 ? t : 31);
    if (t > 0) lo = xl;
    if (t < 32) hi = xh;
  }
  if (lane == 0) eig[(size_t)b * n + j] = 0.5 * (lo + hi);
}

size_t hh_smem(int n) {
  const size_t nlmax = (size_t)(n + kHhCluster - 1) / kHhCluster;
  return sizeof(double2) * (nlmax * n + 4 * (size_t)n) + sizeof(double) * (2 * (size_t)n + kHhCluster + 32);
}

}  // namespace

int herm_eig_tridiag_max_n() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  int n = 0;
  while (n < 4096 && hh_smem(n + 1) <= (size_t)optin) ++n;
  return n;
}

cudaError_t launch_herm_eigvals(double2 *mats, int n, int batch, double *eig, cudaStream_t s) {
  if (n < 1 || n > 4096 || batch < 1) return cudaErrorInvalidValue;
  // larger matrices, or a device that cannot hold a cluster of 8 such CTAs:
  // the cyclic Jacobi solver on the matrix in global memory
  if (n > herm_eig_tridiag_max_n()) return launch_jacobi_herm(mats, n, batch, eig, s);
  const size_t smem = hh_smem(n);
  cudaError_t e = cudaFuncSetAttribute(k_hh_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kHhCluster);
  cfg.blockDim = dim3(kHhThreads);
  cfg.dynamicSmemBytes = smem;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_hh_tridiag, &cfg) != cudaSuccess || clusters < 1) {
    (void)cudaGetLastError();
    return launch_jacobi_herm(mats, n, batch, eig, s);
  }
  k_hh_tridiag<<<batch * kHhCluster, kHhThreads, smem, s>>>(mats, n);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long warps = (long long)batch * n;
  k_tridiag_eigs<<<(unsigned)warps, 32, 0, s>>>(mats, n, batch, eig);
  return cudaGetLastError();
}

}  // namespace w2
