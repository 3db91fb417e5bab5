// Learned form: a multilayer perceptron that stands in for the two-body term
// Theta_{V12} of the pseudo-difference operator, with its own training
// kernels.  For a spatial point X = (x1, x2) the input is
//   [ s_f f(X, p1, p2) (nk^2),  s_f1 f1(x1, .), s_f1 f1(x2, .) (2 nk),
//     sin(2 pi m r / L), cos(2 pi m r / L) for m = 1..8 (r = x1 - x2),  zero padding ]
// (f1 = sum_{x2,p2} f dx dp is the reduced one-body Wigner function), and the
// output is s_y Theta_{V12}[f](X, ., .) (nk^2).  Layers: D_in -> H -> H -> H
// -> nk^2 with SiLU between them; weights kept in FP32 for the optimiser and
// in BF16 for the tensor-core products (FP32 accumulation).
//
//  k_gemm     : C = op(A) op(B) + epilogue on mma.sync m16n8k16 bf16; A and B
//               staged through shared memory with arbitrary element strides,
//               so the same kernel computes X W, dZ W^T and A^T dZ.
//  k_f1, k_features : the input rows, in BF16.
//  k_colsum, k_adam, k_f2bf, k_sqdiff : bias gradients, optimiser, casts and
//               the judge's squared-difference reduction.
#include <math.h>
#include <stdint.h>

#include "w2_internal.cuh"

namespace w2 {

__device__ __forceinline__ uint16_t f2bf(float x) {  // round to nearest even
  const uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);  // inf / nan
  const uint32_t r = u + 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(r >> 16);
}

__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float(((uint32_t)h) << 16); }

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }

__device__ __forceinline__ float dsilu(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

// D(16x8) += A(16x16) B(16x8), bf16 in, f32 accumulate.  Fragments (PTX ISA,
// mma.m16n8k16 .bf16): a = {A[g][2t..2t+1], A[g+8][2t..], A[g][2t+8..], A[g+8][2t+8..]},
// b = {B[2t..2t+1][g], B[2t+8..2t+9][g]}, d = {D[g][2t], D[g][2t+1], D[g+8][2t], D[g+8][2t+1]}.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

// C[m][n] = sum_k A(m, k) B(k, n); A(m, k) = A[m*sam + k*sak], B(k, n) = B[k*sbk + n*sbn].
// 128 threads: 2 x 2 warps, each 32 x 32 of C.  Edges are guarded (any M, N; K % 2 == 0).
__global__ void __launch_bounds__(128) k_gemm(GemmArgs a) {
  __shared__ __align__(16) uint16_t As[GBM][GBK + GPAD];
  __shared__ __align__(16) uint16_t Bs[GBN][GBK + GPAD];  // Bs[n][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int g = lane >> 2, t4 = lane & 3;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const uint16_t *A = (const uint16_t *)a.A, *B = (const uint16_t *)a.B;
  float acc[2][4][4] = {};
  for (int k0 = 0; k0 < a.K; k0 += GBK) {
    // consecutive threads walk the operand's unit-stride direction (coalesced reads)
    for (int e = tid; e < GBM * GBK; e += 128) {
      const int r = a.sak == 1 ? e / GBK : e % GBM, c = a.sak == 1 ? e % GBK : e / GBM;
      const int m = m0 + r, k = k0 + c;
      As[r][c] = (m < a.M && k < a.K) ? A[(size_t)m * a.sam + (size_t)k * a.sak] : (uint16_t)0;
    }
    for (int e = tid; e < GBN * GBK; e += 128) {
      const int r = a.sbk == 1 ? e / GBK : e % GBN, c = a.sbk == 1 ? e % GBK : e / GBN;  // r: n, c: k
      const int n = n0 + r, k = k0 + c;
      Bs[r][c] = (n < a.N && k < a.K) ? B[(size_t)k * a.sbk + (size_t)n * a.sbn] : (uint16_t)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm * 32 + i * 16 + g;
        af[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * t4]);
        af[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * t4]);
        af[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * t4 + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * t4 + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn * 32 + j * 8 + g;
        bfr[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + 2 * t4]);
        bfr[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + 2 * t4 + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm * 32 + i * 16 + g + (q >> 1) * 8;
        const int n = n0 + wn * 32 + j * 8 + 2 * t4 + (q & 1);
        if (m >= a.M || n >= a.N) continue;
        const size_t o = (size_t)m * a.N + n;
        float v = acc[i][j][q];
        switch (a.epi) {
          case GEMM_STORE:  // raw product (weight gradients)
            a.out_f32[o] = v;
            break;
          case GEMM_BIAS_SILU: {  // hidden layer: Z = C + b, A = silu(Z)
            v += a.bias[n];
            a.out_f32[o] = v;
            a.out_bf16[o] = f2bf(silu(v));
            break;
          }
          case GEMM_BIAS_SCALE:  // output layer: Y = (C + b) * scale
            a.out_f32[o] = (v + a.bias[n]) * a.scale;
            break;
          case GEMM_DSILU: {  // back through a hidden layer: dZ = C * silu'(Z)
            v *= dsilu(a.aux[o]);
            a.out_f32[o] = v;
            a.out_bf16[o] = f2bf(v);
            break;
          }
        }
      }
}

// ---------------------------------------------------------------------------
// Inference GEMM: C = A B + epilogue with A [M][K] (K contiguous) and B [K][N]
// (N contiguous), BF16 in, FP32 accumulation on mma.sync m16n8k16.  64 x 128
// tiles, 32-wide K steps, 4 warps (2 x 2, 32 x 64 each), three cp.async stages
// of 16-byte copies, fragments by ldmatrix (.trans for B); bias + SiLU (BF16
// out, optional FP32 pre-activation) or bias + scale (FP32 out) fused.
// ---------------------------------------------------------------------------
constexpr int FBM = 64, FBN = 128, FBK = 32, FSTAGES = 3;
constexpr int FAS = FBK + 8, FBS = FBN + 8;  // padded row strides (BF16): conflict-free ldmatrix

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void ldsm4(uint32_t (&r)[4], const uint16_t *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldsm4t(uint32_t (&r)[4], const uint16_t *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__global__ void __launch_bounds__(128) k_gemm_fwd(GemmArgs a) {
  __shared__ __align__(16) uint16_t As[FSTAGES][FBM][FAS];
  __shared__ __align__(16) uint16_t Bs[FSTAGES][FBK][FBS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1, g = lane >> 2, t4 = lane & 3;
  const int m0 = blockIdx.y * FBM, n0 = blockIdx.x * FBN;
  const uint16_t *A = (const uint16_t *)a.A, *B = (const uint16_t *)a.B;
  const int nkt = (a.K + FBK - 1) / FBK;

  auto load = [&](int kt, int st) {
    const int k0 = kt * FBK;
#pragma unroll
    for (int q = 0; q < 2; ++q) {  // A: 64 rows x 4 chunks
      const int c = tid + q * 128, r = c >> 2, ch = c & 3;
      const int row = m0 + r, k = k0 + ch * 8;
      const bool in = row < a.M && k < a.K;
      cp_async16(&As[st][r][ch * 8], in ? A + (size_t)row * a.K + k : A, in ? 16 : 0);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {  // B: 32 rows x 16 chunks
      const int c = tid + q * 128, r = c >> 4, ch = c & 15;
      const int k = k0 + r, n = n0 + ch * 8;
      const bool in = k < a.K && n < a.N;
      cp_async16(&Bs[st][r][ch * 8], in ? B + (size_t)k * a.N + n : B, in ? 16 : 0);
    }
  };

  float acc[2][8][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

#pragma unroll
  for (int st = 0; st < FSTAGES - 1; ++st) {
    if (st < nkt) load(st, st);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  for (int kt = 0; kt < nkt; ++kt) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(FSTAGES - 2) : "memory");
    __syncthreads();  // tile kt landed for everyone; tile kt - 1's buffer is free
    if (kt + FSTAGES - 1 < nkt) load(kt + FSTAGES - 1, (kt + FSTAGES - 1) % FSTAGES);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    const int st = kt % FSTAGES;
#pragma unroll
    for (int kk = 0; kk < FBK; kk += 16) {
      uint32_t af[2][4], bf[8][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) ldsm4(af[i], &As[st][wm * 32 + i * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        uint32_t r[4];
        ldsm4t(r, &Bs[st][kk + (lane & 15)][wn * 64 + j * 8 + (lane >> 4) * 8]);
        bf[j][0] = r[0];
        bf[j][1] = r[1];
        bf[j + 1][0] = r[2];
        bf[j + 1][1] = r[3];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");

#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + wm * 32 + i * 16 + g + 8 * h, n = n0 + wn * 64 + j * 8 + 2 * t4;
        if (m >= a.M || n >= a.N) continue;
        const size_t o = (size_t)m * a.N + n;
        const float v0 = acc[i][j][2 * h] + a.bias[n], v1 = acc[i][j][2 * h + 1] + a.bias[n + 1];
        if (a.epi == GEMM_BIAS_SILU) {
          if (a.out_f32) *reinterpret_cast<float2 *>(a.out_f32 + o) = make_float2(v0, v1);
          *reinterpret_cast<uint32_t *>(a.out_bf16 + o) = (uint32_t)f2bf(silu(v0)) | ((uint32_t)f2bf(silu(v1)) << 16);
        } else {
          *reinterpret_cast<float2 *>(a.out_f32 + o) = make_float2(v0 * a.scale, v1 * a.scale);
        }
      }
}

// The inference GEMM for unit-stride rows (A K-contiguous, B N-contiguous,
// K and N multiples of 8, 16-byte aligned rows).
cudaError_t launch_gemm_fwd(const GemmArgs &a, cudaStream_t s) {
  if (a.sak != 1 || a.sbn != 1 || a.sam != a.K || a.sbk != a.N || (a.K & 7) || (a.N & 7) ||
      (((uintptr_t)a.A | (uintptr_t)a.B) & 15) || (a.epi != GEMM_BIAS_SILU && a.epi != GEMM_BIAS_SCALE))
    return cudaErrorInvalidValue;
  dim3 grid((a.N + FBN - 1) / FBN, (a.M + FBM - 1) / FBM);
  k_gemm_fwd<<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gemm(const GemmArgs &a, cudaStream_t s) {
  dim3 grid((a.N + GBN - 1) / GBN, (a.M + GBM - 1) / GBM);
  k_gemm<<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

// f1[i][n] = dx dp sum_{i2, n2} f[i][i2][n][n2]  (T = double or float state).
// One warp per (i, n): lanes stride along n2 (coalesced rows), then a fixed
// shuffle tree; 8 warps per block, grid nx * ceil(nk / 8).
template <typename T>
__global__ void __launch_bounds__(256) k_f1(const T *f, float *f1, int nx, int nk, double w) {
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
  if (lane == 0) f1[(size_t)i * nk + n] = (float)(s * w);
}

// One input row per listed spatial point (xs[r] = i1 * nx + i2, or r itself when xs == null).
template <typename T>
__global__ void k_features(FeatArgs a, const T *f) {
  const int r = blockIdx.x;
  const int X = a.xs ? a.xs[r] : r;
  const int nx = a.nx, nk = a.nk, P = nk * nk;
  const int i1 = X / nx, i2 = X % nx;
  uint16_t *row = a.x + (size_t)r * a.din;
  const T *blk = f + (size_t)X * P;
  for (int e = threadIdx.x; e < a.din; e += blockDim.x) {
    float v = 0.f;
    if (e < P)
      v = a.s_f * (float)blk[e];
    else if (e < P + nk)
      v = a.s_f1 * a.f1[(size_t)i1 * nk + (e - P)];
    else if (e < P + 2 * nk)
      v = a.s_f1 * a.f1[(size_t)i2 * nk + (e - P - nk)];
    else if (e < P + 2 * nk + 2 * kMlpHarmonics) {  // sin, cos (2 pi m r / L), m = 1..kMlpHarmonics
      const int q = e - P - 2 * nk, m = q / 2 + 1;
      const float u = 2.f * (float)(m * (i1 - i2)) / (float)nx;
      v = (q & 1) ? cospif(u) : sinpif(u);
    }
    row[e] = f2bf(v);
  }
}

cudaError_t launch_features(const FeatArgs &a, const void *f, int f64, int rows, cudaStream_t s) {
  if (a.f1_src_rows > 0) {  // refresh f1 from the same state first
    const double w = a.dx * a.dp;
    if (f64)
      k_f1<double><<<a.nx * ((a.nk + 7) / 8), 256, 0, s>>>((const double *)f, a.f1, a.nx, a.nk, w);
    else
      k_f1<float><<<a.nx * ((a.nk + 7) / 8), 256, 0, s>>>((const float *)f, a.f1, a.nx, a.nk, w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (f64)
    k_features<double><<<rows, 256, 0, s>>>(a, (const double *)f);
  else
    k_features<float><<<rows, 256, 0, s>>>(a, (const float *)f);
  return cudaGetLastError();
}

// out[n] = sum_m in[m][n]  (bias gradients; fixed order)
__global__ void k_colsum(const float *in, float *out, int M, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += in[(size_t)m * N + n];
  out[n] = s;
}

cudaError_t launch_colsum(const float *in, float *out, int M, int N, cudaStream_t s) {
  k_colsum<<<(N + 127) / 128, 128, 0, s>>>(in, out, M, N);
  return cudaGetLastError();
}

// Adam with bias correction; refreshes the BF16 copy of the parameters.
__global__ void k_adam(float *p, const float *g, float *m, float *v, uint16_t *pb, size_t n, float lr, float b1,
                       float b2, float c1, float c2, float eps) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  if (pb) pb[i] = f2bf(pi);
}

cudaError_t launch_adam(float *p, const float *g, float *m, float *v, uint16_t *pb, size_t n, float lr, float b1,
                        float b2, int t, float eps, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, g, m, v, pb, n, lr, b1, b2, c1, c2, eps);
  return cudaGetLastError();
}

__global__ void k_f2bf(const float *in, uint16_t *out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = f2bf(in[i]);
}

cudaError_t launch_f2bf(const float *in, uint16_t *out, size_t n, cudaStream_t s) {
  k_f2bf<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

// dY = (Y - T) * 2/(M N); loss partials sum (Y - T)^2 per block (fixed order).
__global__ void k_mse(const float *Y, const float *T, float *dY, double *part, size_t n, float gscale) {
  __shared__ double red[256];
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = d * gscale;
    s += (double)d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

cudaError_t launch_mse(const float *Y, const float *T, float *dY, double *part, size_t n, float gscale,
                       cudaStream_t s) {
  k_mse<<<256, 256, 0, s>>>(Y, T, dY, part, n, gscale);
  return cudaGetLastError();
}

// part[b] = (sum (a - b)^2, sum b^2) over a grid-stride slice (fixed order).
template <typename TA, typename T>
__global__ void k_sqdiff(const TA *a, const T *b, double *part, size_t n, double bscale) {
  __shared__ double r0[256], r1[256];
  double s0 = 0.0, s1 = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double bv = (double)b[i] * bscale;
    const double d = (double)a[i] - bv;
    s0 += d * d;
    s1 += bv * bv;
  }
  r0[threadIdx.x] = s0;
  r1[threadIdx.x] = s1;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      r0[threadIdx.x] += r0[threadIdx.x + h];
      r1[threadIdx.x] += r1[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = r0[0];
    part[2 * blockIdx.x + 1] = r1[0];
  }
}

cudaError_t launch_sqdiff(const float *a, const void *b, int b_f64, double *part, size_t n, double bscale,
                          cudaStream_t s) {
  if (b_f64)
    k_sqdiff<float, double><<<128, 256, 0, s>>>(a, (const double *)b, part, n, bscale);
  else
    k_sqdiff<float, float><<<128, 256, 0, s>>>(a, (const float *)b, part, n, bscale);
  return cudaGetLastError();
}

cudaError_t launch_sqdiff64(const double *a, const double *b, double *part, size_t n, cudaStream_t s) {
  k_sqdiff<double, double><<<128, 256, 0, s>>>(a, b, part, n, 1.0);
  return cudaGetLastError();
}

}  // namespace w2
