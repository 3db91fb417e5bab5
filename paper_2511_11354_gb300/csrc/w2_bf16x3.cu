// Precision form, BF16 variant (W2_F32_BF16X3): the X-local pseudo-difference
// sweep of the FP32 state (the operator of Eqs. 33-35 as Toeplitz products,
// the pair term in sheared coordinates, as in w2_f32.cu) on mma.sync
// m16n8k16 with BF16 operands and FP32 accumulation.
//
// Splitting.  An FP32 value x is exactly h + m + l with h = bf16(x),
// m = bf16(x - h), l = x - h - m: each step removes the leading 8 bits of a
// 24-bit significand and the remainders are exact.  A kernel-table value
// (FP64) takes four parts, K = k1 + k2 + k3 + k4 to about 2^-32.  Seven
// products per tile keep every term down to 2^-16 and the fixed table's
// 2^-24 term:
//   k1 f1 (leading);  k1 f2, k2 f1 (2^-8);  k1 f3, k2 f2, k3 f1 (2^-16);
//   k4 f1 (2^-24: the table is the same every step, so its representation
//   error would act as a fixed perturbation of the potential).
// The dropped k2 f3, k3 f2 (2^-24) and below involve the state's low parts,
// which change from step to step.  Each product of two 8-bit significands is
// exact; the leading product gets a fresh accumulator for each 16-wide
// k-step, added to the running sum by an ordinary (round-to-nearest) FP32
// add, because the tensor core's accumulation truncates; the small products
// share one tensor-core accumulator.  Against the TF32 variant (two state
// parts, three table parts, four m16n8k8 products per 8-wide k-step, i.e.
// eight per 16 columns) this is seven m16n8k16 products per 16 columns.
//
// Layout per CTA (one X): the three BF16 planes of the block (row stride
// nk + 8 elements: conflict-free ldmatrix), pair tables P[j] = (part K(j),
// part K(j + 1)) of the three kernel rows in four parts each (one 32-bit
// load per fragment register), and the two-body term in FP32.  Warp w owns
// rows [16 (w >> 1), +16) and columns [(w & 1) nk / 2, +nk / 2).
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include "w2_blocks.cuh"
#include "w2_internal.cuh"

namespace w2 {
namespace {

template <int NK>
struct B3Layout {
  static constexpr int RT = NK / 16;       // 16-row tiles
  static constexpr int WARPS = 2 * RT;     // (row tile, column half)
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int NCT = NK / 16;      // 8-wide column tiles per warp
  static constexpr int SP = NK + 8;        // plane row stride (BF16 elements)
  static constexpr int PW = 2 * NK;        // words per pair table
  static constexpr size_t off_planes = (size_t)NK * NK * 4;  // after the FP32 two-body block
  static constexpr size_t off_pk = off_planes + (size_t)3 * NK * SP * 2;
  static constexpr size_t off_red = off_pk + (size_t)3 * 4 * PW * 4;
  static constexpr size_t bytes = off_red + 64 * sizeof(int) + 32 * sizeof(long long);
};

// products kept per state part s: table parts t < kParts[s]
__host__ __device__ constexpr int b3_parts(int s) { return s == 0 ? 4 : (s == 1 ? 2 : 1); }

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float bf16_value(uint16_t u) { return __uint_as_float((uint32_t)u << 16); }

// x = h + m + l exactly (FP32 x in the normal range).
__device__ __forceinline__ void split3_bf16(float x, uint16_t &h, uint16_t &m, uint16_t &l) {
  h = bf16_bits(x);
  const float r1 = x - bf16_value(h);
  m = bf16_bits(r1);
  l = bf16_bits(r1 - bf16_value(m));
}

// Four BF16 parts of an FP64 value (each residual is exact in FP64).
__device__ __forceinline__ void split4_bf16(double x, uint16_t (&p)[4]) {
  double r = x;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    p[t] = bf16_bits((float)r);
    r -= (double)bf16_value(p[t]);
  }
}

// D(16x8) += A(16x16) B(16x8), BF16 in, FP32 accumulate (PTX ISA fragment
// layout of mma.m16n8k16: a = {A[g][2t..], A[g+8][2t..], A[g][2t+8..], A[g+8][2t+8..]},
// b = {B[2t..2t+1][g], B[2t+8..2t+9][g]}, d = {D[g][2t], D[g][2t+1], D[g+8][2t], D[g+8][2t+1]}).
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void ldsm_a(uint32_t (&r)[4], const uint16_t *p) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}

__device__ __forceinline__ void ldsm_b(uint32_t (&r)[2], const uint16_t *p) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(s));
}

// Rows k, k + 1 of the sheared plane G(k, c) = P(k, c - k) (zero outside the
// window) packed as a B-fragment register.
template <int NK>
__device__ __forceinline__ uint32_t sheared_b(const uint16_t *P, int k, int c) {
  constexpr int SP = B3Layout<NK>::SP;
  const int m0 = c - k, m1 = c - k - 1;
  const uint32_t lo = (unsigned)m0 < (unsigned)NK ? P[k * SP + m0] : 0u;
  const uint32_t hi = (unsigned)m1 < (unsigned)NK ? P[(k + 1) * SP + m1] : 0u;
  return lo | (hi << 16);
}

// Two-body term of the sheared tiles c in [cg, cg + NT) (sheared columns
// s = n1 + n2) of rows [r0, r0 + 16), into A12[n1][n2].
template <int NK, int NT>
__device__ __forceinline__ void pair_tiles_b3(const uint16_t *planes, const uint32_t *pk, float *A12, int r0, int cg) {
  using Lay = B3Layout<NK>;
  constexpr int SP = Lay::SP, PW = Lay::PW;
  const int lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
  const int na = r0 + g, nb = na + 8;
  float acc[NT][4], sml[NT][4];
#pragma unroll
  for (int q = 0; q < NT; ++q)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[q][e] = sml[q][e] = 0.f;
  const int klo = max(0, 8 * cg - NK + 1) & ~15, khi = min(NK - 1, 8 * (cg + NT - 1) + 7);
  for (int kk = klo; kk <= khi; kk += 16) {
    const int ja = kk + 2 * t4 - na + NK - 1;  // A[n1][n1'] = K12(n1' - n1)
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const uint16_t *P = planes + s * NK * SP;
      uint32_t b[NT][2];
#pragma unroll
      for (int q = 0; q < NT; ++q) {
        const int c = 8 * (cg + q) + g;
        b[q][0] = sheared_b<NK>(P, kk + 2 * t4, c);
        b[q][1] = sheared_b<NK>(P, kk + 2 * t4 + 8, c);
      }
#pragma unroll
      for (int t = 0; t < b3_parts(s); ++t) {
        const uint32_t *K = pk + (2 * 4 + t) * PW;
        const uint32_t ka[4] = {K[ja], K[ja - 8], K[ja + 8], K[ja]};
#pragma unroll
        for (int q = 0; q < NT; ++q) {
          if (s == 0 && t == 0) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            mma_bf16(d, ka, b[q]);
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[q][e] += d[e];  // round-to-nearest on the CUDA cores
          } else {
            mma_bf16(sml[q], ka, b[q]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NT; ++q)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int n1 = e < 2 ? na : nb;
      const int n2 = 8 * (cg + q) + 2 * t4 + (e & 1) - n1;
      if ((unsigned)n2 < (unsigned)NK) A12[n1 * NK + n2] = acc[q][e] + sml[q][e];
    }
}

// One CTA per X.  MODE 0: out = Theta[in].  MODE 1: out = base + (h +
// half_tau Theta[in]), and with xsum given the exact per-X sum of out (the
// rule and bits of xsum_block).
template <int NK, int MODE>
__global__ void __launch_bounds__(B3Layout<NK>::THREADS, 1) k_theta_b3(Theta32Args a) {
  using Lay = B3Layout<NK>;
  constexpr int SP = Lay::SP, PW = Lay::PW, NCT = Lay::NCT, THREADS = Lay::THREADS, W = 2 * NK - 1;
  extern __shared__ __align__(16) unsigned char smb[];
  float *A12 = reinterpret_cast<float *>(smb);
  uint16_t *planes = reinterpret_cast<uint16_t *>(smb + Lay::off_planes);
  uint32_t *pk = reinterpret_cast<uint32_t *>(smb + Lay::off_pk);
  int *red = reinterpret_cast<int *>(smb + Lay::off_red);
  long long *lred = reinterpret_cast<long long *>(red + 64);

  const int X = blockIdx.x, nx = a.nx;
  const int i1 = X / nx, i2 = X - i1 * nx;
  int dd = i1 - i2;
  dd += (dd < 0) ? nx : 0;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  const size_t base = (size_t)X * NK * NK;

  // The block's three BF16 planes, straight from global memory.
  {
    constexpr int PER = NK * NK / 4 / THREADS;
    static_assert(PER * 4 * THREADS == NK * NK, "whole float4 per thread");
    const float4 *src = reinterpret_cast<const float4 *>(a.in + base);
    float4 v[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) v[i] = src[tid + i * THREADS];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = 4 * (tid + i * THREADS), r = e / NK, c = e - r * NK;
      uint16_t h[4], m[4], l[4];
      split3_bf16(v[i].x, h[0], m[0], l[0]);
      split3_bf16(v[i].y, h[1], m[1], l[1]);
      split3_bf16(v[i].z, h[2], m[2], l[2]);
      split3_bf16(v[i].w, h[3], m[3], l[3]);
      uint16_t *row = planes + r * SP + c;
      *reinterpret_cast<uint2 *>(row) = make_uint2(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16));
      *reinterpret_cast<uint2 *>(row + NK * SP) =
          make_uint2(m[0] | ((uint32_t)m[1] << 16), m[2] | ((uint32_t)m[3] << 16));
      *reinterpret_cast<uint2 *>(row + 2 * NK * SP) =
          make_uint2(l[0] | ((uint32_t)l[1] << 16), l[2] | ((uint32_t)l[3] << 16));
    }
  }
  // Pair tables: word j of table (family, t) = (part_t K(j), part_t K(j + 1)),
  // family 0: K1 row i1, 1: K2 row i2, 2: K12 row dd.
  {
    uint16_t *pkh = reinterpret_cast<uint16_t *>(pk);
    for (int e = tid; e < 3 * W; e += THREADS) {
      const int fam = e / W, j = e - fam * W;
      const double kv = fam == 0 ? a.K1[(size_t)i1 * W + j] : fam == 1 ? a.K2[(size_t)i2 * W + j]
                                                                        : a.K12[(size_t)dd * W + j];
      uint16_t p[4];
      split4_bf16(kv, p);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        uint16_t *T = pkh + (size_t)(fam * 4 + t) * PW * 2;
        T[2 * j] = p[t];
        if (j > 0) T[2 * j - 1] = p[t];
        if (j == W - 1) {  // K(W) = 0, and the table's last word
          T[2 * j + 1] = 0;
          T[2 * j + 2] = 0;
          T[2 * j + 3] = 0;
        }
      }
    }
  }
  __syncthreads();

  const int r0 = 16 * (w >> 1), c0 = (w & 1) * (NK / 2);
  const int na = r0 + g, nb = na + 8;

  // Two-body term: the sheared tiles of this row block, split between its two warps.
  {
    const int cfirst = r0 >> 3, clast = min((r0 + 15 + NK - 1) >> 3, (2 * NK - 2) >> 3);
    const int ntile = clast - cfirst + 1, half = (ntile + 1) >> 1;
    int c = (w & 1) ? cfirst + half : cfirst;
    const int cend = (w & 1) ? clast + 1 : cfirst + half;
    for (; c + 3 <= cend; c += 3) pair_tiles_b3<NK, 3>(planes, pk, A12, r0, c);
    if (cend - c == 2) pair_tiles_b3<NK, 2>(planes, pk, A12, r0, c);
    if (cend - c == 1) pair_tiles_b3<NK, 1>(planes, pk, A12, r0, c);
  }
  __syncthreads();

  // One-body terms T1 = A1(x1) F and T2 = F A2(x2)^T, on top of the two-body term.
  float acc[NCT][4], sml[NCT][4];
#pragma unroll
  for (int q = 0; q < NCT; ++q) {
    const int n2 = c0 + 8 * q + 2 * t4;
    acc[q][0] = A12[na * NK + n2];
    acc[q][1] = A12[na * NK + n2 + 1];
    acc[q][2] = A12[nb * NK + n2];
    acc[q][3] = A12[nb * NK + n2 + 1];
#pragma unroll
    for (int e = 0; e < 4; ++e) sml[q][e] = 0.f;
  }
  for (int kk = 0; kk < NK; kk += 16) {
    const int ja = kk + 2 * t4 - na + NK - 1;       // A1[n1][n1'] = K1(n1' - n1)
    const int jb = kk + 2 * t4 - c0 - g + NK - 1;   // B2[n2'][n2] = K2(n2' - n2), tile q at jb - 8q
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      const uint16_t *P = planes + s * NK * SP;
      uint32_t fa[4];
      ldsm_a(fa, P + (r0 + (lane & 15)) * SP + kk + (lane >> 4) * 8);  // F rows (A of T2)
      uint32_t ka[b3_parts(0)][4];
#pragma unroll
      for (int t = 0; t < b3_parts(s); ++t) {
        const uint32_t *K1t = pk + (0 * 4 + t) * PW;
        ka[t][0] = K1t[ja];
        ka[t][1] = K1t[ja - 8];
        ka[t][2] = K1t[ja + 8];
        ka[t][3] = K1t[ja];
      }
#pragma unroll
      for (int q = 0; q < NCT; ++q) {
        uint32_t fb[2];
        ldsm_b(fb, P + (kk + (lane & 15)) * SP + c0 + 8 * q);           // F columns (B of T1)
#pragma unroll
        for (int t = 0; t < b3_parts(s); ++t) {
          const uint32_t *K2t = pk + (1 * 4 + t) * PW;
          const uint32_t kb[2] = {K2t[jb - 8 * q], K2t[jb - 8 * q + 8]};
          if (s == 0 && t == 0) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            mma_bf16(d, ka[0], fb);
            mma_bf16(d, fa, kb);
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[q][e] += d[e];  // round-to-nearest on the CUDA cores
          } else {
            mma_bf16(sml[q], ka[t], fb);
            mma_bf16(sml[q], fa, kb);
          }
        }
      }
    }
  }

  // Epilogue; in the corrector with xsum given the outputs also wait in the
  // thread's own slots of A12 for the exact per-X sum.
  const bool sums = MODE == 1 && a.xsum;
  int em_loc = 0;
#pragma unroll
  for (int q = 0; q < NCT; ++q) {
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int n1 = hr ? nb : na, n2 = c0 + 8 * q + 2 * t4;
      const size_t o = base + (size_t)n1 * NK + n2;
      const float t0 = acc[q][2 * hr] + sml[q][2 * hr], t1 = acc[q][2 * hr + 1] + sml[q][2 * hr + 1];
      float2 v;
      if (MODE == 0) {
        v.x = t0;
        v.y = t1;
      } else {
        const float2 hv = *reinterpret_cast<const float2 *>(a.h + o);
        const float2 fv = *reinterpret_cast<const float2 *>(a.base + o);
        v.x = fv.x + fmaf(a.half_tau, t0, hv.x);
        v.y = fv.y + fmaf(a.half_tau, t1, hv.y);
      }
      if (sums) {
        em_loc = max(em_loc, max(expo_of(v.x), expo_of(v.y)));
        A12[n1 * NK + n2] = v.x;
        A12[n1 * NK + n2 + 1] = v.y;
      }
      *reinterpret_cast<float2 *>(a.out + o) = v;
    }
  }
  if (sums) {
    int em = __reduce_max_sync(0xffffffffu, em_loc);
    if (lane == 0) red[w] = em;
    __syncthreads();
    em = 0;
#pragma unroll
    for (int q = 0; q < Lay::WARPS; ++q) em = max(em, red[q]);
    em = max(em, 1);
    long long s = 0;
#pragma unroll
    for (int q = 0; q < NCT; ++q)
#pragma unroll
      for (int hr = 0; hr < 2; ++hr) {
        const int n1 = hr ? nb : na, n2 = c0 + 8 * q + 2 * t4;
        s += fixed_image(A12[n1 * NK + n2], em) + fixed_image(A12[n1 * NK + n2 + 1], em);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) lred[w] = s;
    __syncthreads();
    if (tid == 0) {
      long long tot = 0;
      for (int q = 0; q < Lay::WARPS; ++q) tot += lred[q];
      a.xsum[X] = em == 255 ? __longlong_as_double(0x7ff8000000000000ll) : ll_to_double_scaled(tot, em - 174);
    }
  }
}

template <int NK>
cudaError_t prep_b3() {
  cudaError_t e = cudaFuncSetAttribute(k_theta_b3<NK, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)B3Layout<NK>::bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_theta_b3<NK, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)B3Layout<NK>::bytes);
  return e;
}

template <int NK>
cudaError_t run_b3(int mode, const Theta32Args &a, cudaStream_t s) {
  using Lay = B3Layout<NK>;
  const int grid = a.nx * a.nx;
  if (mode == 0)
    k_theta_b3<NK, 0><<<grid, Lay::THREADS, Lay::bytes, s>>>(a);
  else
    k_theta_b3<NK, 1><<<grid, Lay::THREADS, Lay::bytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

#define W2_B3_SWITCH(nk, EXPR)                 \
  switch (nk) {                                \
    case 16: return EXPR(16);                  \
    case 32: return EXPR(32);                  \
    case 48: return EXPR(48);                  \
    case 64: return EXPR(64);                  \
    case 80: return EXPR(80);                  \
    case 96: return EXPR(96);                  \
    case 112: return EXPR(112);                \
    case 128: return EXPR(128);                \
    default: return cudaErrorInvalidValue;     \
  }

cudaError_t prepare_kernels_b3(int nk) {
#define W2_P(N) prep_b3<N>()
  W2_B3_SWITCH(nk, W2_P)
#undef W2_P
}

cudaError_t launch_theta_b3(int nk, int mode, const Theta32Args &a, cudaStream_t s) {
#define W2_T(N) run_b3<N>(mode, a, s)
  W2_B3_SWITCH(nk, W2_T)
#undef W2_T
}

}  // namespace w2
