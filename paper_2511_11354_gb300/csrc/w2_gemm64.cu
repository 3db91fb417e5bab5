// Batched FP64 matrix products on the FP64 pipe (DFMA), the contractions of
// the spectral-element operators (Sec. 3.2): per phase-space point X the
// one-body tables act along one momentum axis, and the two-body term runs a
// chain of products through the y grid.
//
// Tile 64 x 64 x 16, 256 threads, a 4 x 4 register block per thread on a
// stride-16 lattice (rows ty + 16 i, columns tx + 16 j) so that the shared
// memory reads are broadcasts or consecutive; the next K tile is loaded into
// registers while the current one is used; every global access is predicated,
// so M, N and K are arbitrary.
#include "w2_sem.cuh"

namespace w2sem {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <int A_COL, int B_COL>
__global__ void __launch_bounds__(NT) k_gemm64(Gemm64 g) {
  __shared__ double As[2][BK][BM + 1];
  __shared__ double Bs[2][BK][BN + 1];
  const int b = blockIdx.x;
  const int n0 = blockIdx.y * BN, m0 = blockIdx.z * BM;
  const long long b1 = b / g.bdiv, b2 = b % g.bdiv;
  const double *A = g.A + b1 * g.sA1 + b2 * g.sA2;
  const double *B = g.B + b1 * g.sB1 + b2 * g.sB2;
  double *C = g.C + b1 * g.sC1 + b2 * g.sC2;
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;

  double ra[4], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = t + NT * r;
      int m, k;
      if (A_COL) { m = e & 63; k = e >> 6; } else { m = e >> 4; k = e & 15; }
      const int gm = m0 + m, gk = k0 + k;
      ra[r] = (gm < g.M && gk < g.K) ? (A_COL ? A[gm + gk * g.lda] : A[gm * g.lda + gk]) : 0.0;
      int n;
      if (B_COL) { n = e >> 4; k = e & 15; } else { n = e & 63; k = e >> 6; }
      const int gn = n0 + n;
      const int gk2 = k0 + k;
      rb[r] = (gn < g.N && gk2 < g.K) ? (B_COL ? B[gk2 + gn * g.ldb] : B[gk2 * g.ldb + gn]) : 0.0;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = t + NT * r;
      if (A_COL) As[buf][e >> 6][e & 63] = ra[r]; else As[buf][e & 15][e >> 4] = ra[r];
      if (B_COL) Bs[buf][e & 15][e >> 4] = rb[r]; else Bs[buf][e >> 6][e & 63] = rb[r];
    }
  };

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  const int ntile = (g.K + BK - 1) / BK;
  load(0);
  store(0);
  __syncthreads();
  for (int kt = 0; kt < ntile; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < ntile) load((kt + 1) * BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[cur][k][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[cur][k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    if (kt + 1 < ntile) store(cur ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      double *c = C + (long long)m * g.ldc + n;
      *c = (g.beta != 0.0) ? fma(g.alpha, acc[i][j], g.beta * *c) : g.alpha * acc[i][j];
    }
  }
}

}  // namespace

cudaError_t launch_gemm64(const Gemm64 &g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.nbatch <= 0) return cudaSuccess;
  const int tn = (g.N + BN - 1) / BN, tm = (g.M + BM - 1) / BM;
  if (tn > 65535 || tm > 65535 || g.bdiv <= 0) return cudaErrorInvalidValue;
  dim3 grid(g.nbatch, tn, tm);
  if (g.a_col) {
    if (g.b_col) k_gemm64<1, 1><<<grid, NT, 0, s>>>(g); else k_gemm64<1, 0><<<grid, NT, 0, s>>>(g);
  } else {
    if (g.b_col) k_gemm64<0, 1><<<grid, NT, 0, s>>>(g); else k_gemm64<0, 0><<<grid, NT, 0, s>>>(g);
  }
  return cudaGetLastError();
}

}  // namespace w2sem
