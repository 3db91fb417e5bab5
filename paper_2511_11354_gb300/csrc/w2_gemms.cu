// FP64-accurate batched matrix products on the BF16 tensor cores by exact
// integer slices (the splitting scheme of Ozaki, Ogita, Oishi and Rump,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 59, 2012,
// with fixed-point digits and integer recombination), for the spectral-element
// operators of the non-periodic path (Sec. 3.2).
//
// Slicing.  Each line of an operand (a row of A, a column of B: the values
// along the contraction index k) is scaled by 2^-E, 2^E > every |v| of the
// line, rounded to 47-bit fixed point N = round(|v| 2^(47 - E)) and written as
// six balanced base-256 digits N = sum_s d_s 256^(5 - s) with d_0 in [0, 128]
// and d_1..d_5 in [-128, 127], each carrying v's sign and exact in BF16.
//
// Products.  sum_k a_k b_k = 2^(Ea + Eb - 94) sum_{s,t} 256^(10 - s - t) sum_k da_s db_t;
// the 21 digit pairs with s + t <= 5 are kept.  Pairs of one diagonal
// g = s + t share an FP32 accumulator (six of them).  Every digit product is
// at most 2^14 and a call contracts at most 256 terms, so the partial sums of
// the diagonals 0..3 (at most four pairs) stay within 2^24 and are exact
// integers whatever the order and truncation of the tensor core's additions;
// the diagonals 4 and 5 may round, near 2^-56 of the line scales.  The six
// accumulators are recombined in int64 (units of diagonal 5) and turned into
// FP64 by integer operations; an output either replaces C or is added to it.
// A line holding Inf or NaN marks its exponent, and the outputs that touch
// it are NaN.
//
// Tiles.  A CTA of 4 warps computes a 64 x 32 output tile (warp tile 32 x 16:
// two m16 by two n8 mma.m16n8k16 tiles), K in stages of 32 staged by cp.async
// into shared memory, two stages in flight.  Each 64-byte row of a digit
// plane keeps its four 16-byte chunks in the order c ^ ((row >> 1) & 3), so
// that the eight rows an ldmatrix reads fall in distinct banks without
// padding (74 KB per CTA: three CTAs per SM).  The output tiles of one
// batch entry are consecutive CTAs, so its operand slices are re-read from L2.
#include <math.h>
#include <stdint.h>

#include "w2_df.cuh"
#include "w2_sem.cuh"

namespace w2sem {
namespace {

constexpr int kDig = 6;
constexpr int kBadExp = 4096;  // exponent of a line holding Inf or NaN

__device__ __forceinline__ int expo(double v) {
  return (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff);
}

// Six balanced base-256 digits of |v| 2^(47 - E), with v's sign.
__device__ __forceinline__ void digits6(double v, int E, int (&d)[kDig]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = (b & 0xfffffffffffffull) | (e ? (1ull << 52) : 0ull);
  const int sh = 1028 + E - (e ? e : 1);  // >= 6 for |v| < 2^E
  long long n = (sh < 64 && sh > 0) ? (long long)((m + (1ull << (sh - 1))) >> sh) : 0;
#pragma unroll
  for (int s = kDig - 1; s >= 1; --s) {
    const int lo = (int)(n & 255);
    const int ds = lo - ((lo & 128) << 1);
    d[s] = ds;
    n = (n - ds) >> 8;
  }
  d[0] = (int)n;
  if (b >> 63) {
#pragma unroll
    for (int s = 0; s < kDig; ++s) d[s] = -d[s];
  }
}

// BF16 bits of a small integer (|d| <= 256): exact through the FP32 magic-number sum.
__device__ __forceinline__ uint16_t bf16_int(int d) {
  return (uint16_t)(__float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16);
}

// Line exponent E from the largest biased exponent of the line.
__device__ __forceinline__ int line_exp(int emax) { return emax == 0x7ff ? kBadExp : emax - 1022; }

// Row slicer: one warp per line of K contiguous values (K <= 512).
template <int MODE>
__global__ void __launch_bounds__(256) k_slice_rows(SliceArgs a) {
  const int warp = threadIdx.x >> 5, ln = threadIdx.x & 31;
  const int l = blockIdx.x * 8 + warp;
  const int b = blockIdx.y;
  if (l >= a.L) return;
  const long long b1 = b / a.bdiv, b2 = b % a.bdiv;
  const double *in = a.in + b1 * a.sIn1 + b2 * a.sIn2 + (long long)l * a.ls;
  double v[16];
  int emax = 0;
  const double *drow = nullptr;
  int Nyh = 0, dstride = 0;
  if (MODE == 1) {  // D_V weighting of the two-body chain: line l = y2 index, k = [re|im] x y1 index
    const int X = a.x0 + b;
    const int rho = X / a.nx - X % a.nx;
    Nyh = a.h + 1;
    dstride = (2 * a.nx - 1) * (4 * a.h + 1);
    drow = a.dtab + (long long)(rho + a.nx - 1) * (4 * a.h + 1) + 2 * a.h - (l - a.h);  // + r gives u = r - (l - h)
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int k = ln + 32 * i;
    double x = 0.0;
    if (k < a.K) {
      x = in[k];
      if (MODE == 1) {
        const int r = k % Nyh;
        x *= drow[(r ? dstride : 0) + r];
      }
    }
    v[i] = x;
    const int e = expo(x);
    emax = e > emax ? e : emax;
  }
  emax = __reduce_max_sync(0xffffffffu, emax);
  const int E = line_exp(emax);
  if (ln == 0) a.ex[b * a.sE + l] = E;
  uint16_t *P = a.planes + b * a.sP + (long long)l * a.Kp;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int k = ln + 32 * i;
    if (k >= a.Kp) break;
    int d[kDig];
    if (k < a.K && E != kBadExp) {
      digits6(v[i], E, d);
    } else {
#pragma unroll
      for (int s = 0; s < kDig; ++s) d[s] = 0;
    }
#pragma unroll
    for (int s = 0; s < kDig; ++s) P[(long long)s * a.pP + k] = bf16_int(d[s]);
  }
}

// Column slicer: lines are the columns of a row-major K x N matrix (row
// stride ks); the planes keep the row-major layout [K_p][ldp] so that the
// product reads them as B[k][n].  One CTA per 32 columns.
__global__ void __launch_bounds__(256) k_slice_cols(SliceArgs a) {
  __shared__ int red[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + tx;
  const int b = blockIdx.y;
  const long long b1 = b / a.bdiv, b2 = b % a.bdiv;
  const double *in = a.in + b1 * a.sIn1 + b2 * a.sIn2;
  int emax = 0;
  if (col < a.L)
    for (int k = ty; k < a.K; k += 8) {
      const int e = expo(in[(long long)k * a.ks + col]);
      emax = e > emax ? e : emax;
    }
  red[ty][tx] = emax;
  __syncthreads();
  if (ty == 0) {
    for (int i = 1; i < 8; ++i) emax = red[i][tx] > emax ? red[i][tx] : emax;
    red[0][tx] = emax;
  }
  __syncthreads();
  const int E = line_exp(red[0][tx]);
  if (ty == 0 && col < a.L) a.ex[b * a.sE + col] = E;
  uint16_t *P = a.planes + b * a.sP;
  if (col >= a.ldp) return;
  for (int k = ty; k < a.Kp; k += 8) {
    int d[kDig];
    if (col < a.L && k < a.K && E != kBadExp) {
      digits6(in[(long long)k * a.ks + col], E, d);
    } else {
#pragma unroll
      for (int s = 0; s < kDig; ++s) d[s] = 0;
    }
#pragma unroll
    for (int s = 0; s < kDig; ++s) P[(long long)s * a.pP + (long long)k * a.ldp + col] = bf16_int(d[s]);
  }
}

// Column slices of the D_V-weighted second transform for S'^T = E B: line
// y1 (a column of the planes) runs over k = [re | im] x y2, k < 2 Ny, with
// B(k, y1) = w(y1) D(rho; y1, y2) A^T[y2][part Nyh + y1] (part = k / Ny,
// y2 = k % Ny - h), A^T [Ny][2 Nyh] per X; planes [6][Kp][ldp] row-major.
__global__ void __launch_bounds__(256) k_slice_dstack(SliceArgs a) {
  __shared__ int red[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int y1 = blockIdx.x * 32 + tx;
  const int b = blockIdx.y;
  const int Nyh = a.h + 1, Ny = 2 * a.h + 1, K = 2 * Ny;
  const double *in = a.in + (long long)b * a.sIn1;  // A^T of this X, row stride ls = 2 Nyh
  const int X = a.x0 + b, rho = X / a.nx - X % a.nx;
  const double *drow = a.dtab + (y1 > 0 ? (long long)(2 * a.nx - 1) * (4 * a.h + 1) : 0) +
                       (long long)(rho + a.nx - 1) * (4 * a.h + 1) + 2 * a.h + y1 + a.h;  // + (-c) gives u = y1 - (c - h)
  auto val = [&](int k) -> double {
    const int part = k >= Ny, c = k - part * Ny;
    return in[(long long)c * a.ls + part * Nyh + y1] * drow[-c];
  };
  int emax = 0;
  if (y1 < Nyh)
    for (int k = ty; k < K; k += 8) {
      const int e = expo(val(k));
      emax = e > emax ? e : emax;
    }
  red[ty][tx] = emax;
  __syncthreads();
  if (ty == 0) {
    for (int i = 1; i < 8; ++i) emax = red[i][tx] > emax ? red[i][tx] : emax;
    red[0][tx] = emax;
  }
  __syncthreads();
  const int E = line_exp(red[0][tx]);
  if (ty == 0 && y1 < Nyh) a.ex[b * a.sE + y1] = E;
  uint16_t *P = a.planes + b * a.sP;
  if (y1 >= a.ldp) return;
  for (int k = ty; k < a.Kp; k += 8) {
    int d[kDig];
    if (y1 < Nyh && k < K && E != kBadExp) {
      digits6(val(k), E, d);
    } else {
#pragma unroll
      for (int s = 0; s < kDig; ++s) d[s] = 0;
    }
#pragma unroll
    for (int s = 0; s < kDig; ++s) P[(long long)s * a.pP + (long long)k * a.ldp + y1] = bf16_int(d[s]);
  }
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const uint16_t *p) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const uint16_t *p) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool full) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  const int n = full ? 16 : 0;  // 0: fill the 16 bytes with zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

constexpr int GM = 64, GN = 32, GK = 32, GT = 128;

// BF16 offset of chunk c (8 elements) of row r in a swizzled 32-element row.
__device__ __forceinline__ int swz(int r, int c) { return r * 32 + ((c ^ ((r >> 1) & 3)) << 3); }

template <int B_KN>
struct GLayout {
  static constexpr int a_stage = kDig * GM * GK;                           // BF16 elements
  static constexpr int b_stage = kDig * GN * GK;                           // [n][k] or [k][n], 32 x 32
  static constexpr size_t bytes = 2 * (size_t)(a_stage + b_stage) * 2;
};

template <int B_KN>
__global__ void __launch_bounds__(GT, 3) k_gemms(GemmSArgs g) {
  extern __shared__ __align__(16) uint16_t sm[];
  using Ly = GLayout<B_KN>;
  uint16_t *As = sm, *Bs = sm + 2 * Ly::a_stage;
  const int tn = (g.N + GN - 1) / GN;
  const int b = blockIdx.y, n0 = (blockIdx.x % tn) * GN, m0 = (blockIdx.x / tn) * GM;
  const long long b1 = b / g.bdiv, b2 = b % g.bdiv;
  const uint16_t *A = g.A + b1 * g.sA1 + b2 * g.sA2;
  const uint16_t *B = g.B + b1 * g.sB1 + b2 * g.sB2;
  const int t = threadIdx.x, warp = t >> 5, ln = t & 31;
  const int wm = warp & 1, wn = warp >> 1;

  // Per-thread copy plan: chunk t + 128 i of a stage is (digit, row, 16-byte
  // column q = t & 3); A rows t/4 and t/4 + 32, B row (or k row) t/4.
  const int q4 = t & 3, r4 = t >> 2;
  const bool okA0 = m0 + r4 < g.M, okA1 = m0 + r4 + 32 < g.M;
  const uint16_t *a0 = A + (long long)(okA0 ? m0 + r4 : 0) * g.lda + 8 * q4;
  const uint16_t *a1 = A + (long long)(okA1 ? m0 + r4 + 32 : 0) * g.lda + 8 * q4;
  const bool okB = B_KN ? (n0 + 8 * q4 < g.ldb) : (n0 + r4 < g.N);
  const uint16_t *b0 = B_KN ? B + (long long)r4 * g.ldb + (okB ? n0 + 8 * q4 : 0)
                            : B + (long long)(okB ? n0 + r4 : 0) * g.ldb + 8 * q4;
  const int dA0 = swz(r4, q4), dA1 = swz(r4 + 32, q4), dB = swz(r4, q4);
  auto load_stage = [&](int buf, int k0) {
    uint16_t *as = As + buf * Ly::a_stage;
    uint16_t *bs = Bs + buf * Ly::b_stage;
    const long long kb = B_KN ? (long long)k0 * g.ldb : k0;
#pragma unroll
    for (int s = 0; s < kDig; ++s) {
      cp_async16(as + s * GM * GK + dA0, a0 + s * g.pA + k0, okA0);
      cp_async16(as + s * GM * GK + dA1, a1 + s * g.pA + k0, okA1);
      cp_async16(bs + s * GN * GK + dB, b0 + s * g.pB + kb, okB);
    }
    cp_async_commit();
  };

  float acc[kDig][2][2][4];
#pragma unroll
  for (int d = 0; d < kDig; ++d)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[d][i][j][e] = 0.f;

  const int nst = (g.K + GK - 1) / GK;
  load_stage(0, g.k0);
  for (int st = 0; st < nst; ++st) {
    const int cur = st & 1;
    if (st + 1 < nst) {
      load_stage(cur ^ 1, g.k0 + (st + 1) * GK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const uint16_t *as = As + cur * Ly::a_stage;
    const uint16_t *bs = Bs + cur * Ly::b_stage;
#pragma unroll
    for (int kk = 0; kk < GK; kk += 16) {
      uint32_t bf[kDig][4];  // per digit: n-tile 0 (2 regs), n-tile 1 (2 regs)
      const int q = ln >> 3, r = ln & 7;
#pragma unroll
      for (int s = 0; s < kDig; ++s) {
        if (!B_KN) {
          ldsm_x4(bf[s], bs + swz(s * GN + wn * 16 + (q >> 1) * 8 + r, (kk >> 3) + (q & 1)));
        } else {
          ldsm_x4_t(bf[s], bs + swz(s * GK + kk + (q & 1) * 8 + r, 2 * wn + (q >> 1)));
        }
      }
#pragma unroll
      for (int s = 0; s < kDig; ++s) {
        uint32_t af[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          ldsm_x4(af[mt], as + swz(s * GM + wm * 32 + mt * 16 + (q & 1) * 8 + r, (kk >> 3) + (q >> 1)));
        }
#pragma unroll
        for (int tt = 0; tt < kDig - s; ++tt) {
          const int gd = s + tt;
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            mma16816(acc[gd][mt][0], af[mt], bf[tt][0], bf[tt][1]);
            mma16816(acc[gd][mt][1], af[mt], bf[tt][2], bf[tt][3]);
          }
        }
      }
    }
    __syncthreads();
  }

  double *C = g.C + b1 * g.sC1 + b2 * g.sC2;
  const int *Ae = g.Ae + b1 * g.sAe1 + b2 * g.sAe2;
  const int *Be = g.Be + b1 * g.sBe1 + b2 * g.sBe2;
  // Outputs of this thread: rows m0 + wm 32 + mt 16 + ln/4 (+ 8), columns
  // n0 + wn 16 + nt 8 + 2 (ln & 3) (+ 1).  With beta the old values are all
  // requested before any is used, so their latencies overlap.
  double old[2][4][2];
  if (g.beta) {
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int row = m0 + wm * 32 + mt * 16 + (ln >> 2) + (e >= 2 ? 8 : 0);
          const int col = n0 + wn * 16 + nt * 8 + 2 * (ln & 3) + (e & 1);
          old[mt][e][nt] = (row < g.M && col < g.N) ? C[(long long)row * g.ldc + col] : 0.0;
        }
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int row = m0 + wm * 32 + mt * 16 + (ln >> 2) + (e >= 2 ? 8 : 0);
      if (row >= g.M) continue;
      const int ea = Ae[row];
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int col = n0 + wn * 16 + nt * 8 + 2 * (ln & 3) + (e & 1);
        if (col >= g.N) continue;
        const int eb = Be[col];
        const long long I = (long long)__float2int_rn(acc[0][mt][nt][e]) * (1ll << 40) +
                            (long long)__float2int_rn(acc[1][mt][nt][e]) * (1ll << 32) +
                            (long long)__float2int_rn(acc[2][mt][nt][e]) * (1ll << 24) +
                            (long long)__float2int_rn(acc[3][mt][nt][e]) * (1ll << 16) +
                            __float2ll_rn(acc[4][mt][nt][e]) * (1ll << 8) + __float2ll_rn(acc[5][mt][nt][e]);
        double v = (ea == kBadExp || eb == kBadExp) ? __longlong_as_double(0x7ff8000000000000ll)
                                                    : w2::ll_to_double_scaled(I, ea + eb - 54);
        C[(long long)row * g.ldc + col] = g.beta ? old[mt][e][nt] + v : v;
      }
    }
}

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

}  // namespace

int slice_kp(int K) { return round_up(K, GK); }

cudaError_t launch_slice(int cols, int mode, const SliceArgs &a, cudaStream_t s) {
  if (a.nbatch <= 0 || a.L <= 0) return cudaSuccess;
  if (a.nbatch > 65535 || a.bdiv <= 0) return cudaErrorInvalidValue;
  if (!cols) {
    if (a.K > 512 || a.Kp < a.K || a.Kp > 512) return cudaErrorInvalidValue;
    dim3 grid((a.L + 7) / 8, a.nbatch);
    if (mode == 1) k_slice_rows<1><<<grid, 256, 0, s>>>(a); else k_slice_rows<0><<<grid, 256, 0, s>>>(a);
  } else {
    if (a.ldp < a.L || a.ldp % 8 || a.Kp < a.K) return cudaErrorInvalidValue;
    dim3 grid((a.ldp + 31) / 32, a.nbatch);
    k_slice_cols<<<grid, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_slice_dstack(const SliceArgs &a, cudaStream_t s) {
  if (a.nbatch <= 0) return cudaSuccess;
  if (a.nbatch > 65535 || a.ldp % 8 || a.ldp < a.h + 1 || a.Kp < 2 * (2 * a.h + 1)) return cudaErrorInvalidValue;
  dim3 grid((a.ldp + 31) / 32, a.nbatch);
  k_slice_dstack<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gemms(int b_kn, const GemmSArgs &g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.nbatch <= 0) return cudaSuccess;
  if (g.K > 256 || g.K <= 0 || g.bdiv <= 0 || g.lda % 8 || g.ldb % 8 || g.k0 % GK) return cudaErrorInvalidValue;
  const long long tiles = (long long)((g.N + GN - 1) / GN) * ((g.M + GM - 1) / GM);
  if (tiles > 0x7fffffffLL || g.nbatch > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)tiles, g.nbatch);
  cudaError_t e;
  if (b_kn) {
    e = cudaFuncSetAttribute(k_gemms<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GLayout<1>::bytes);
    if (e != cudaSuccess) return e;
    k_gemms<1><<<grid, GT, GLayout<1>::bytes, s>>>(g);
  } else {
    e = cudaFuncSetAttribute(k_gemms<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GLayout<0>::bytes);
    if (e != cudaSuccess) return e;
    k_gemms<0><<<grid, GT, GLayout<0>::bytes, s>>>(g);
  }
  return cudaGetLastError();
}

}  // namespace w2sem
