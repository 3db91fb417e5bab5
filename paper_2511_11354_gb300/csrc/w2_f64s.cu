// FP64-accurate pseudo-difference sweep on the BF16 tensor cores, by exact
// integer slices (the splitting scheme of Ozaki, Ogita, Oishi and Rump,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 59, 2012,
// here with fixed-point digits and integer recombination).
//
// For one spatial point X = (x1, x2) the state block F = f(X, ., .) and the
// three kernel rows K1(x1, .), K2(x2, .), K12(x1 - x2, .) of Eq. Hartree_FSM
// and Eq. two_body_FSM are scaled by powers of two, 2^EF >= |F| for the block
// and 2^EK >= |K| for the three rows together, rounded to 48-bit fixed point
// N = round(|v| 2^(48 - E)) and written as six balanced base-256 digits
//     N = sum_{s=0..5} d_s 256^(5-s),   d_0 in [0, 256],  d_1..d_5 in [-128, 127],
// each carrying the sign of v and each exact in BF16 (8 significant bits).
// The operator's three Toeplitz contractions (K1 along p1, K2 along p2, K12
// along the anti-diagonal, as in k_theta of w2_f64.cu) become sums over digit
// pairs (s, t) of integer products; the 21 pairs with s + t <= 5 are kept, the
// rest lie below 2^-48 of the block scale.
//
// Exactness.  Pairs of one diagonal d = s + t share an FP32 accumulator.  A
// product of two digits is at most 2^16 (d_0 d_0), 2^15 (d_0 d_t) or 2^14, a
// contraction has at most 64 terms and the one-body sweep adds two of them, so
// every partial sum of diagonals 0..3 stays below 2^24 and is an exact integer
// whatever the order and rounding of the tensor core's additions.  Diagonals
// 4 and 5 share the last accumulator (the d = 5 products take a 2^-8 factor in
// their K digit); its rounding lies below 2^-50 of the block scale.  The
// diagonals are recombined in 64-bit integers (the two-body part through
// shared memory, unsheared) and turned into FP64 with integer operations; the
// FP64 pipe does one fused multiply-add per output, the corrector combination.
// A block holding Inf or NaN gives NaN outputs.
//
// Layout per CTA (one X): digit planes D_s[n1][n2] in BF16 (row stride nk + 8,
// conflict-free ldmatrix), pair tables P[j] = (d(K(j)), d(K(j + 1))) of the
// three kernel rows (and their 2^-8 copies) so that an A/B fragment register
// is one 32-bit load, and the two-body term as int64.  Warp w owns rows
// [16 (w >> 1), +16) and columns [(w & 1) nk / 2, +nk / 2).
#include <math.h>
#include <stdint.h>

#include "w2_blocks.cuh"
#include "w2_df.cuh"
#include "w2_internal.cuh"
#include "w2_slice.cuh"

namespace w2 {
namespace {

using slice::kDig;
using slice::expo;
using slice::digits6;
using slice::bf16_int;

template <int NK>
struct SlicedLayout {
  static constexpr int RT = NK / 16;        // 16-row tiles
  static constexpr int WARPS = 2 * RT;      // (row tile, column half)
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int NCT = NK / 16;       // 8-wide column tiles per warp in the one-body sweep
  static constexpr int SP = NK + 8;         // digit-plane row stride (BF16 elements)
  static constexpr int PW = 2 * NK;         // words per pair table
  static constexpr size_t off_planes = (size_t)NK * NK * 8;  // after the int64 two-body block
  static constexpr size_t off_pk = off_planes + (size_t)kDig * NK * SP * 2;
  static constexpr size_t off_red = off_pk + (size_t)3 * 2 * kDig * PW * 4;
  static constexpr size_t bytes = off_red + 2 * 32 * sizeof(int);
};

// The five diagonal accumulators of one output as an int64 in units of
// 2^-4 of a diagonal-4 unit.
__device__ __forceinline__ long long combine5(float a0, float a1, float a2, float a3, float a4) {
  return (long long)__float2int_rn(a0) * (1ll << 36) + (long long)__float2int_rn(a1) * (1ll << 28) +
         (long long)__float2int_rn(a2) * (1ll << 20) + (long long)__float2int_rn(a3) * (1ll << 12) +
         (long long)__float2int_rn(a4 * 16.f);
}

// D(16x8) += A(16x16) B(16x8), BF16 in, FP32 accumulate (PTX ISA fragment
// layout of mma.m16n8k16: a = {A[g][2t..], A[g+8][2t..], A[g][2t+8..], A[g+8][2t+8..]},
// b = {B[2t..2t+1][g], B[2t+8..2t+9][g]}, d = {D[g][2t], D[g][2t+1], D[g+8][2t], D[g+8][2t+1]}).
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
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

__device__ __forceinline__ void ldsm_x2_t(uint32_t (&r)[2], const uint16_t *p) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(s));
}

// Two consecutive rows k, k+1 of the sheared block G(k, c) = D(k, c - k) (zero
// outside the window) packed as a B-fragment register.
template <int NK>
__device__ __forceinline__ uint32_t sheared_pair(const uint16_t *P, int k, int c) {
  constexpr int SP = SlicedLayout<NK>::SP;
  const int m0 = c - k, m1 = c - k - 1;
  const uint32_t lo = (unsigned)m0 < (unsigned)NK ? P[k * SP + m0] : 0u;
  const uint32_t hi = (unsigned)m1 < (unsigned)NK ? P[(k + 1) * SP + m1] : 0u;
  return lo | (hi << 16);
}

// Two-body term of the tiles c in [cg, cg + NT) (sheared columns s = n1 + n2)
// of rows [r0, r0 + 16): the 21 digit products, recombined into I12[n1][n2].
template <int NK, int NT>
__device__ __forceinline__ void pair_tiles(const uint16_t *planes, const uint32_t *pk, long long *I12, int r0,
                                           int cg) {
  using Lay = SlicedLayout<NK>;
  constexpr int SP = Lay::SP, PW = Lay::PW;
  const int lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
  const int na = r0 + g, nb = na + 8;
  float acc[5][NT][4];
#pragma unroll
  for (int d = 0; d < 5; ++d)
#pragma unroll
    for (int q = 0; q < NT; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[d][q][e] = 0.f;
  const int klo = max(0, 8 * cg - NK + 1) & ~15, khi = min(NK - 1, 8 * (cg + NT - 1) + 7);
  for (int kk = klo; kk <= khi; kk += 16) {
    const int ja = kk + 2 * t4 - na + NK - 1;  // A[n1][n1'] = K12(n1' - n1)
#pragma unroll
    for (int s = 0; s < kDig; ++s) {
      const uint16_t *P = planes + s * NK * SP;
      uint32_t b[NT][2];
#pragma unroll
      for (int q = 0; q < NT; ++q) {
        const int c = 8 * (cg + q) + g;
        b[q][0] = sheared_pair<NK>(P, kk + 2 * t4, c);
        b[q][1] = sheared_pair<NK>(P, kk + 2 * t4 + 8, c);
      }
#pragma unroll
      for (int t = 0; s + t < kDig; ++t) {
        const int d = s + t;
        const uint32_t *K = pk + ((4 + (d == 5)) * kDig + t) * PW;
        const uint32_t ka[4] = {K[ja], K[ja - 8], K[ja + 8], K[ja]};
#pragma unroll
        for (int q = 0; q < NT; ++q) mma16816(acc[d < 4 ? d : 4][q], ka, b[q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NT; ++q)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int n1 = e < 2 ? na : nb;
      const int n2 = 8 * (cg + q) + 2 * t4 + (e & 1) - n1;
      if ((unsigned)n2 < (unsigned)NK)
        I12[n1 * NK + n2] = combine5(acc[0][q][e], acc[1][q][e], acc[2][q][e], acc[3][q][e], acc[4][q][e]);
    }
}

// The exact per-X sum of the block's outputs (the rule and bits of
// xsum_block), second pass: each thread's outputs wait in its own slots of
// I12 (as FP64 bit patterns, at [n1][n2] for the outputs (n1, n2) the
// epilogue of k_theta_s gives it), em_loc is the largest exponent among them.
// Every thread of the CTA calls this; red: 64 ints of shared memory.  Thread
// 0 writes *out.
template <int NK, int NCT>
__device__ __forceinline__ void slot_exact_sum(const long long *I12, int em_loc, double *out, int *red) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5, g = lane >> 2, t4 = lane & 3;
  const int r0 = 16 * (w >> 1), c0 = (w & 1) * (NK / 2);
  long long *lred = reinterpret_cast<long long *>(red + 32);
  int em = __reduce_max_sync(0xffffffffu, em_loc);
  if (lane == 0) red[w] = em;
  __syncthreads();
  em = 0;
  for (int q = 0; q < nw; ++q) em = max(em, red[q]);
  em = max(em, 1);
  long long acc = 0;
#pragma unroll
  for (int q = 0; q < NCT; ++q)
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int n1 = r0 + g + 8 * hr, n2 = c0 + 8 * q + 2 * t4;
      acc += fixed_image(__longlong_as_double(I12[n1 * NK + n2]), em);
      acc += fixed_image(__longlong_as_double(I12[n1 * NK + n2 + 1]), em);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) lred[w] = acc;
  __syncthreads();
  if (tid == 0) {
    long long tot = 0;
    for (int q = 0; q < nw; ++q) tot += lred[q];
    *out = em == 2047 ? __longlong_as_double(0x7ff8000000000000ll) : ll_to_double_scaled(tot, em - 1071);
  }
  __syncthreads();
}

// One CTA per spatial point X (with a.sym: per X with i1 <= i2, the mirror
// block written as well).  MODE 0: out = Theta[in].  MODE 1: out = h + half_tau Theta[in].
template <int NK, int MODE>
__global__ void __launch_bounds__(SlicedLayout<NK>::THREADS, 512 / SlicedLayout<NK>::THREADS)
    k_theta_s(ThetaArgs a) {
  using Lay = SlicedLayout<NK>;
  constexpr int SP = Lay::SP, PW = Lay::PW, NCT = Lay::NCT, W = 2 * NK - 1, THREADS = Lay::THREADS;
  extern __shared__ __align__(16) unsigned char smraw[];
  long long *I12 = reinterpret_cast<long long *>(smraw);
  uint16_t *planes = reinterpret_cast<uint16_t *>(smraw + Lay::off_planes);
  uint32_t *pk = reinterpret_cast<uint32_t *>(smraw + Lay::off_pk);
  int *red = reinterpret_cast<int *>(smraw + Lay::off_red);

  const int nx = a.nx;
  int i1, i2;
  if (a.sym) {  // block b of the upper triangle, row by row: i1 <= i2
    int b = blockIdx.x;
    i1 = 0;
    while (b >= nx - i1) {
      b -= nx - i1;
      ++i1;
    }
    i2 = i1 + b;
  } else {
    i1 = blockIdx.x / nx;
    i2 = blockIdx.x - i1 * nx;
  }
  const int X = i1 * nx + i2;
  int dd = i1 - i2;
  dd += (dd < 0) ? nx : 0;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  const size_t base = (size_t)X * NK * NK;
  const bool two_body = a.pair == nullptr;
  const int nfam = two_body ? 3 : 2;
  const double *k1row = a.K1 + (size_t)i1 * W, *k2row = a.K2 + (size_t)i2 * W, *k12row = a.K12 + (size_t)dd * W;

  // Block exponents (largest biased exponent of the state block / the kernel rows).
  constexpr int PER = NK / 8;  // element pairs per thread
  double2 fv[PER];
  int ef = 0, ek = 0;
  {
    const double2 *src = reinterpret_cast<const double2 *>(a.in + base);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      fv[i] = src[tid + i * THREADS];
      ef = max(ef, max(expo(fv[i].x), expo(fv[i].y)));
    }
    for (int e = tid; e < nfam * W; e += THREADS) {
      const int fam = e / W, j = e - fam * W;
      ek = max(ek, expo((fam == 0 ? k1row : fam == 1 ? k2row : k12row)[j]));
    }
    ef = __reduce_max_sync(0xffffffffu, ef);
    ek = __reduce_max_sync(0xffffffffu, ek);
    if (lane == 0) {
      red[w] = ef;
      red[32 + w] = ek;
    }
    __syncthreads();
    ef = ek = 0;
#pragma unroll
    for (int q = 0; q < Lay::WARPS; ++q) {
      ef = max(ef, red[q]);
      ek = max(ek, red[32 + q]);
    }
  }
  const bool bad = ef == 2047 || ek == 2047;
  const int emax = max(ef, 1), kmax = max(ek, 1);

  // Digit planes of the block.
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int p = tid + i * THREADS;
    const int r = (2 * p) / NK, c = 2 * p - r * NK;
    int dx[kDig], dy[kDig];
    digits6(fv[i].x, emax, dx);
    digits6(fv[i].y, emax, dy);
#pragma unroll
    for (int s = 0; s < kDig; ++s)
      *reinterpret_cast<uint32_t *>(planes + s * NK * SP + r * SP + c) = bf16_int(dx[s]) | (bf16_int(dy[s]) << 16);
  }
  // Pair tables: word j of table (family, scaled, t) = (digit_t K(j), digit_t K(j + 1)).
  {
    uint16_t *pkh = reinterpret_cast<uint16_t *>(pk);
    for (int e = tid; e < nfam * W; e += THREADS) {
      const int fam = e / W, j = e - fam * W;
      int dk[kDig];
      digits6((fam == 0 ? k1row : fam == 1 ? k2row : k12row)[j], kmax, dk);
#pragma unroll
      for (int t = 0; t < kDig; ++t) {
        const uint16_t u = (uint16_t)bf16_int(dk[t]);
        const uint16_t us = dk[t] ? (uint16_t)(u - 0x0400) : (uint16_t)0;  // times 2^-8
        uint16_t *T0 = pkh + (size_t)((fam * 2 + 0) * kDig + t) * PW * 2;
        uint16_t *T1 = pkh + (size_t)((fam * 2 + 1) * kDig + t) * PW * 2;
        T0[2 * j] = u;
        T1[2 * j] = us;
        if (j > 0) {
          T0[2 * j - 1] = u;
          T1[2 * j - 1] = us;
        }
      }
    }
  }
  __syncthreads();

  const int r0 = 16 * (w >> 1), c0 = (w & 1) * (NK / 2);
  const int na = r0 + g, nb = na + 8;

  // Two-body term: the sheared tiles of this row block, split between the two warps.
  if (two_body) {
    const int cfirst = r0 >> 3, clast = min((r0 + 15 + NK - 1) >> 3, (2 * NK - 2) >> 3);
    const int ntile = clast - cfirst + 1, half = (ntile + 1) >> 1;
    int c = (w & 1) ? cfirst + half : cfirst;
    const int cend = (w & 1) ? clast + 1 : cfirst + half;
    for (; c + 3 <= cend; c += 3) pair_tiles<NK, 3>(planes, pk, I12, r0, c);
    if (cend - c == 2) pair_tiles<NK, 2>(planes, pk, I12, r0, c);
    if (cend - c == 1) pair_tiles<NK, 1>(planes, pk, I12, r0, c);
  }

  // One-body terms T1 = A1(x1) F and T2 = F A2(x2)^T on the digit planes.
  float acc[5][NCT][4];
#pragma unroll
  for (int d = 0; d < 5; ++d)
#pragma unroll
    for (int q = 0; q < NCT; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[d][q][e] = 0.f;
  for (int kk = 0; kk < NK; kk += 16) {
    const int ja = kk + 2 * t4 - na + NK - 1;       // A1[n1][n1'] = K1(n1' - n1)
    const int jb = kk + 2 * t4 - c0 - g + NK - 1;   // B2[n2'][n2] = K2(n2' - n2), tile q at jb - 8q
#pragma unroll
    for (int s = 0; s < kDig; ++s) {
      const uint16_t *P = planes + s * NK * SP;
      uint32_t fa[4], fb[NCT][2];
      ldsm_x4(fa, P + (r0 + (lane & 15)) * SP + kk + (lane >> 4) * 8);  // F rows (A of T2)
#pragma unroll
      for (int q = 0; q < NCT; q += 2) {                                 // F columns (B of T1)
        if (q + 1 < NCT) {
          uint32_t r[4];
          ldsm_x4_t(r, P + (kk + (lane & 15)) * SP + c0 + 8 * q + (lane >> 4) * 8);
          fb[q][0] = r[0];
          fb[q][1] = r[1];
          fb[q + 1][0] = r[2];
          fb[q + 1][1] = r[3];
        } else {
          uint32_t r[2];
          ldsm_x2_t(r, P + (kk + (lane & 15)) * SP + c0 + 8 * q);
          fb[q][0] = r[0];
          fb[q][1] = r[1];
        }
      }
#pragma unroll
      for (int t = 0; s + t < kDig; ++t) {
        const int d = s + t;
        const uint32_t *K1t = pk + ((0 + (d == 5)) * kDig + t) * PW;
        const uint32_t *K2t = pk + ((2 + (d == 5)) * kDig + t) * PW;
        const uint32_t ka[4] = {K1t[ja], K1t[ja - 8], K1t[ja + 8], K1t[ja]};
        uint32_t kprev = K2t[jb + 8];
#pragma unroll
        for (int q = 0; q < NCT; ++q) {
          mma16816(acc[d < 4 ? d : 4][q], ka, fb[q]);
          const uint32_t bq[2] = {K2t[jb - 8 * q], kprev};
          kprev = bq[0];
          mma16816(acc[d < 4 ? d : 4][q], fa, bq);
        }
      }
    }
  }

  // The one-body products above read only the digit planes and the pair
  // tables, so each warp went on to them as soon as its sheared tiles were
  // done; the epilogue reads the other warps' two-body results (and the
  // mirror staging overwrites the digit planes).
  const bool mirror = a.sym && i1 != i2;
  if (two_body || mirror) __syncthreads();

  // Epilogue: recombine, add the two-body term, scale, combine with h; in the
  // corrector (with xsum given) also the exact per-X sum of the outputs, whose
  // values wait in the thread's own slots of I12 for the second pass.
  const int xs = emax + kmax - 2096;  // one unit of the recombined integer is 2^xs
  const bool sums = MODE == 1 && a.xsum;
  double *C = reinterpret_cast<double *>(planes);  // Theta at X for the mirror block, row stride NK + 1
  int em_loc = 0;
#pragma unroll
  for (int q = 0; q < NCT; ++q) {
#pragma unroll
    for (int hr = 0; hr < 2; ++hr) {
      const int n1 = hr ? nb : na, n2 = c0 + 8 * q + 2 * t4;
      long long v0 = combine5(acc[0][q][2 * hr], acc[1][q][2 * hr], acc[2][q][2 * hr], acc[3][q][2 * hr],
                              acc[4][q][2 * hr]);
      long long v1 = combine5(acc[0][q][2 * hr + 1], acc[1][q][2 * hr + 1], acc[2][q][2 * hr + 1],
                              acc[3][q][2 * hr + 1], acc[4][q][2 * hr + 1]);
      const size_t o = base + (size_t)n1 * NK + n2;
      double t0, t1;
      if (two_body) {
        v0 += I12[n1 * NK + n2];
        v1 += I12[n1 * NK + n2 + 1];
        t0 = ll_to_double_scaled(v0, xs);
        t1 = ll_to_double_scaled(v1, xs);
      } else {
        t0 = ll_to_double_scaled(v0, xs) + (double)a.pair[o];
        t1 = ll_to_double_scaled(v1, xs) + (double)a.pair[o + 1];
      }
      if (bad) t0 = t1 = __longlong_as_double(0x7ff8000000000000ll);
      if (mirror) {
        C[n1 * (NK + 1) + n2] = t0;
        C[n1 * (NK + 1) + n2 + 1] = t1;
      }
      double2 v;
      if (MODE == 0) {
        v.x = t0;
        v.y = t1;
      } else {
        const double2 hv = *reinterpret_cast<const double2 *>(a.h + o);
        v.x = fma(a.half_tau, t0, hv.x);
        v.y = fma(a.half_tau, t1, hv.y);
      }
      if (sums) {
        em_loc = max(em_loc, max(expo(v.x), expo(v.y)));
        I12[n1 * NK + n2] = __double_as_longlong(v.x);
        I12[n1 * NK + n2 + 1] = __double_as_longlong(v.y);
      }
      *reinterpret_cast<double2 *>(a.out + o) = v;
    }
  }
  if (sums) slot_exact_sum<NK, NCT>(I12, em_loc, a.xsum + X, red);
  if (mirror) {
    __syncthreads();  // C complete
    slice::mirror_block<NK, THREADS, MODE>(a, C, i2 * nx + i1, red);
  }
}

template <int NK>
cudaError_t prep_s() {
  cudaError_t e = cudaFuncSetAttribute(k_theta_s<NK, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)SlicedLayout<NK>::bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_theta_s<NK, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SlicedLayout<NK>::bytes);
}

template <int NK>
cudaError_t run_s(int mode, const ThetaArgs &a, cudaStream_t s) {
  using Lay = SlicedLayout<NK>;
  const int grid = a.sym ? a.nx * (a.nx + 1) / 2 : a.nx * a.nx;
  if (mode == 0)
    k_theta_s<NK, 0><<<grid, Lay::THREADS, Lay::bytes, s>>>(a);
  else
    k_theta_s<NK, 1><<<grid, Lay::THREADS, Lay::bytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool nk_supported_f64s(int nk) { return nk == 16 || nk == 32 || nk == 48 || nk == 64; }

cudaError_t prepare_kernels_f64s(int nk) {
  switch (nk) {
    case 16: return prep_s<16>();
    case 32: return prep_s<32>();
    case 48: return prep_s<48>();
    case 64: return prep_s<64>();
    default: return cudaErrorInvalidValue;
  }
}

// Sliced sweep (mode 0 / 1 as launch_theta_f64, per-X sums of the corrector's output included).
cudaError_t launch_theta_f64s(int nk, int mode, const ThetaArgs &a, cudaStream_t s) {
  switch (nk) {
    case 16: return run_s<16>(mode, a, s);
    case 32: return run_s<32>(mode, a, s);
    case 48: return run_s<48>(mode, a, s);
    case 64: return run_s<64>(mode, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace w2
