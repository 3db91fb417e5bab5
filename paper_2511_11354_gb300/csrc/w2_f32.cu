// Precision form: FP32 state, split-precision tensor-core contractions.
//
//  k_theta32 : the X-local pseudo-difference sweep of w2_f64.cu on
//              mma.sync m16n8k8 tf32 with FP32 accumulation.  The state block
//              is split into two TF32 parts (hi = tf32(x), lo = tf32(x - hi))
//              and the kernel table into three; four partial products per
//              tile (see mma5_a3).  The operator's output enters
//              the time step scaled by tau*|Theta| (a few 1e-2), so its error
//              stays below the FP32 rounding of the state.
//  k_adv32   : periodic cubic-spline shift along x2 (DIR 0) and x1 (DIR 1).
//              The shift of the state is computed as an increment
//              delta = (S - I) f from taps that merge the B-spline evaluation
//              weights with the (1,4,1)/6 interpolation condition, so its FP32
//              error is proportional to the (sub-cell) shift, not to |f|; the
//              state itself is rounded once per step, in the corrector.  The
//              spline coefficients are solved in double-float pairs (about
//              2^-47 per operation) and kept as (hi, lo) FP32 pairs in shared
//              memory; the evaluation reads both parts.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "w2_blocks.cuh"
#include "w2_df.cuh"
#include "w2_internal.cuh"

namespace w2 {

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}

// Three TF32 parts of an FP64 kernel value: x = hi + mid + lo to ~2^-33.
__device__ __forceinline__ void split3_tf32_d(double x, uint32_t &hi, uint32_t &mid, uint32_t &lo) {
  hi = tf32_rna((float)x);
  const double r1 = x - (double)__uint_as_float(hi);
  mid = tf32_rna((float)r1);
  lo = tf32_rna((float)(r1 - (double)__uint_as_float(mid)));
}

// D(16x8) += A(16x8) B(8x8), TF32 in, FP32 accumulate.  Fragments (PTX ISA,
// mma.m16n8k8 .tf32): a = A[g][t], A[g+8][t], A[g][t+4], A[g+8][t+4];
// b = B[t][g], B[t+4][g]; d = D[g][2t], D[g][2t+1], D[g+8][2t], D[g+8][2t+1]
// with g = lane>>2, t = lane&3.
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Products of a three-part operand K = kh + km + kl (the kernel table) with a
// two-part operand F = fh + fl: kh fh, the 2^-11 terms km fh and kh fl, and
// kl fh (2^-22, kept because the table is the same every step).  The dropped
// km fl (2^-22) involves the low part of the state, which changes from step
// to step, so its omission does not accumulate coherently.  The leading
// product goes to the accumulator `big`, the small ones to `small`.  The
// tensor core's FP32 accumulation drops the bits of the smaller addend below
// the larger one's last place (no rounding to nearest), which biases long
// running sums; so the callers give `big` a fresh zero accumulator for each
// 8-wide k-step and add it to the running sum with an ordinary FP32 add.
// The kernel table is the same in every step, so a representation error in
// it would act like a fixed perturbation of the potential and accumulate
// coherently; three parts remove it.
__device__ __forceinline__ void mma5_a3(float (&big)[4], float (&small)[4], const uint32_t (&kh)[4],
                                        const uint32_t (&km)[4], const uint32_t (&kl)[4], const uint32_t (&fh)[2],
                                        const uint32_t (&fl)[2]) {
  mma_tf32(small, kl, fh);
  mma_tf32(small, km, fh);
  mma_tf32(small, kh, fl);
  mma_tf32(big, kh, fh);
}

// Same with the kernel table as the B operand and F as the A operand.
__device__ __forceinline__ void mma5_b3(float (&big)[4], float (&small)[4], const uint32_t (&fh)[4],
                                        const uint32_t (&fl)[4], const uint32_t (&kh)[2], const uint32_t (&km)[2],
                                        const uint32_t (&kl)[2]) {
  mma_tf32(small, fh, kl);
  mma_tf32(small, fh, km);
  mma_tf32(small, fl, kh);
  mma_tf32(big, fh, kh);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

template <int NK>
struct Theta32Smem {
  static constexpr int S = NK + 8;  // padded row stride (floats): conflict-free B fragments
  static constexpr size_t words = 3 * (size_t)NK * S + 9 * 2 * NK + 64;  // + the per-X sum's scratch
  static constexpr size_t bytes = 4 * words;
};

// Warps per 16-row block of the X block: the two warps of a row block share
// its A fragments and split its 8-wide column tiles (and its sheared
// two-body tiles) in halves, so a CTA of 4 NK threads keeps twice the warps of
// one warp per row block with half the accumulators per thread.  Every output
// tile goes through the same sequence of products either way.
constexpr int kTh32Split = 2;

// One CTA per X; the SPLIT warps SPLIT r .. SPLIT r + SPLIT - 1 own momentum
// rows [16r, 16r + 16) and split its column tiles; warps beyond SPLIT nk / 16
// only take part in the loads and barriers (the persistent batch step runs
// every item with the same block).  The split does not change the bits.
// MODE 0: out = Theta[in].  MODE 1: out = base + (h + half_tau Theta[in]).
template <int NK, int MODE, int SPLIT = kTh32Split>
// compiled once (not inlined) so the single-problem and batched kernels
// run the same machine code and give identical bits
__device__ __noinline__ void theta32_block(const Theta32Args &a, const int X, uint32_t *smu) {
  using L = Theta32Smem<NK>;
  constexpr int S = L::S, NT = NK / 8, W = 2 * NK - 1;
  uint32_t *Fh = smu, *Fl = smu + NK * S;
  float *Acc = reinterpret_cast<float *>(smu + 2 * NK * S);
  uint32_t *kt = smu + 3 * NK * S;  // hi, mid, lo parts of K1, K2, K12, 2NK words each
  uint32_t *k1h = kt, *k1m = kt + 2 * NK, *k1l = kt + 4 * NK;
  uint32_t *k2h = kt + 6 * NK, *k2m = kt + 8 * NK, *k2l = kt + 10 * NK;
  uint32_t *k12h = kt + 12 * NK, *k12m = kt + 14 * NK, *k12l = kt + 16 * NK;

  const int nx = a.nx;
  const int i1 = X / nx, i2 = X - i1 * nx;
  int dd = i1 - i2;
  dd += (dd < 0) ? nx : 0;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  const int part = w % SPLIT;                 // this warp's part of the column tiles
  constexpr int NTH = NT / SPLIT;
  static_assert(NT % SPLIT == 0, "the warps of a row block split its column tiles evenly");
  const bool active = w < SPLIT * (NK / 16);
  const int bfirst = part * NTH;
  const size_t base = (size_t)X * NK * NK;
  {
    // the raw block goes to the Fl buffer by 16-byte asynchronous copies (all
    // in flight together, overlapping the kernel-table loads); each thread
    // then splits the values it copied into their TF32 parts in place
    const float4 *src = reinterpret_cast<const float4 *>(a.in + base);
    for (int e = tid; e < NK * NK / 4; e += blockDim.x) {
      const int r = (4 * e) / NK, c = 4 * e - r * NK;
      cp_async16(Fl + r * S + c, src + e);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int j = tid; j < W; j += blockDim.x) {
      split3_tf32_d(a.K1[(size_t)i1 * W + j], k1h[j], k1m[j], k1l[j]);
      split3_tf32_d(a.K2[(size_t)i2 * W + j], k2h[j], k2m[j], k2l[j]);
      split3_tf32_d(a.K12[(size_t)dd * W + j], k12h[j], k12m[j], k12l[j]);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    for (int e = tid; e < NK * NK / 4; e += blockDim.x) {
      const int r = (4 * e) / NK, c = 4 * e - r * NK;
      const float4 v = *reinterpret_cast<const float4 *>(Fl + r * S + c);
      uint4 h, l;
      split_tf32(v.x, h.x, l.x);
      split_tf32(v.y, h.y, l.y);
      split_tf32(v.z, h.z, l.z);
      split_tf32(v.w, h.w, l.w);
      *reinterpret_cast<uint4 *>(Fh + r * S + c) = h;
      *reinterpret_cast<uint4 *>(Fl + r * S + c) = l;
    }
  }
  __syncthreads();

  const int r0 = 16 * (w / SPLIT);
  const int na = r0 + g, nb = r0 + g + 8;  // the two A/D rows of this lane

  // Two-body term in sheared coordinates (see k_theta in w2_f64.cu); the
  // sheared tiles of the row block are split between its warps.
  if (active) {
    const int cfirst = r0 >> 3, cmax = min((r0 + 15 + NK - 1) >> 3, (2 * NK - 2) >> 3);
    const int ntile = cmax - cfirst + 1;
    const int cbeg = cfirst + (part * ntile + SPLIT - 1) / SPLIT;
    const int cend = cfirst + ((part + 1) * ntile + SPLIT - 1) / SPLIT - 1;
    for (int c = cbeg; c <= cend; ++c) {
      float d[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f};
      const int nlo = max(0, 8 * c - NK + 1), nhi = min(NK - 1, 8 * c + 7);
      const int s = 8 * c + g;
      for (int kk = nlo & ~7; kk <= nhi; kk += 8) {
        uint32_t ah[4], am[4], al[4], bh[2], bl[2];
        const int c0 = kk + t4, c1 = kk + t4 + 4;
        const int j0 = c0 - na + NK - 1, j1 = c0 - nb + NK - 1, j2 = c1 - na + NK - 1, j3 = c1 - nb + NK - 1;
        ah[0] = k12h[j0]; am[0] = k12m[j0]; al[0] = k12l[j0];
        ah[1] = k12h[j1]; am[1] = k12m[j1]; al[1] = k12l[j1];
        ah[2] = k12h[j2]; am[2] = k12m[j2]; al[2] = k12l[j2];
        ah[3] = k12h[j3]; am[3] = k12m[j3]; al[3] = k12l[j3];
        const int m0 = s - c0, m1 = s - c1;
        const bool v0 = (m0 >= 0 && m0 < NK), v1 = (m1 >= 0 && m1 < NK);
        bh[0] = v0 ? Fh[c0 * S + m0] : 0u; bl[0] = v0 ? Fl[c0 * S + m0] : 0u;
        bh[1] = v1 ? Fh[c1 * S + m1] : 0u; bl[1] = v1 ? Fl[c1 * S + m1] : 0u;
        float t[4] = {0.f, 0.f, 0.f, 0.f};
        mma5_a3(t, e, ah, am, al, bh, bl);
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] += t[q];  // round-to-nearest on the CUDA cores
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) d[q] += e[q];
      const int sa = 8 * c + 2 * t4;
      int n2;
      n2 = sa - na;     if (n2 >= 0 && n2 < NK) Acc[na * S + n2] = d[0];
      n2 = sa + 1 - na; if (n2 >= 0 && n2 < NK) Acc[na * S + n2] = d[1];
      n2 = sa - nb;     if (n2 >= 0 && n2 < NK) Acc[nb * S + n2] = d[2];
      n2 = sa + 1 - nb; if (n2 >= 0 && n2 < NK) Acc[nb * S + n2] = d[3];
    }
  }
  __syncthreads();  // the row block's Acc rows come from all of its warps
  const bool sums = MODE == 1 && a.xsum;
  int em_loc = 0;  // largest exponent of this thread's outputs (for the per-X sum)
  if (active) {
  float acc[NTH][4], sml[NTH][4];
#pragma unroll
  for (int bb = 0; bb < NTH; ++bb) {
    const int b = bfirst + bb;
    acc[bb][0] = Acc[na * S + 8 * b + 2 * t4];
    acc[bb][1] = Acc[na * S + 8 * b + 2 * t4 + 1];
    acc[bb][2] = Acc[nb * S + 8 * b + 2 * t4];
    acc[bb][3] = Acc[nb * S + 8 * b + 2 * t4 + 1];
#pragma unroll
    for (int q = 0; q < 4; ++q) sml[bb][q] = 0.f;
  }
  for (int kk = 0; kk < NK; kk += 8) {
    const int c0 = kk + t4, c1 = kk + t4 + 4;
    uint32_t a1h[4], a1m[4], a1l[4], a2h[4], a2l[4];
    {  // A1[n1][n1'] = K1(n1' - n1)
      const int j0 = c0 - na + NK - 1, j1 = c0 - nb + NK - 1, j2 = c1 - na + NK - 1, j3 = c1 - nb + NK - 1;
      a1h[0] = k1h[j0]; a1m[0] = k1m[j0]; a1l[0] = k1l[j0];
      a1h[1] = k1h[j1]; a1m[1] = k1m[j1]; a1l[1] = k1l[j1];
      a1h[2] = k1h[j2]; a1m[2] = k1m[j2]; a1l[2] = k1l[j2];
      a1h[3] = k1h[j3]; a1m[3] = k1m[j3]; a1l[3] = k1l[j3];
    }
    a2h[0] = Fh[na * S + c0]; a2l[0] = Fl[na * S + c0];               // F[n1][n2']
    a2h[1] = Fh[nb * S + c0]; a2l[1] = Fl[nb * S + c0];
    a2h[2] = Fh[na * S + c1]; a2l[2] = Fl[na * S + c1];
    a2h[3] = Fh[nb * S + c1]; a2l[3] = Fl[nb * S + c1];
#pragma unroll
    for (int bb = 0; bb < NTH; ++bb) {
      const int n2 = 8 * (bfirst + bb) + g;
      uint32_t bh[2], bm[2], bl[2];
      bh[0] = Fh[c0 * S + n2]; bl[0] = Fl[c0 * S + n2];               // F[n1'][n2]
      bh[1] = Fh[c1 * S + n2]; bl[1] = Fl[c1 * S + n2];
      float t[4] = {0.f, 0.f, 0.f, 0.f};
      mma5_a3(t, sml[bb], a1h, a1m, a1l, bh, bl);
      const int j0 = c0 - n2 + NK - 1, j1 = c1 - n2 + NK - 1;         // K2(n2' - n2)
      bh[0] = k2h[j0]; bm[0] = k2m[j0]; bl[0] = k2l[j0];
      bh[1] = k2h[j1]; bm[1] = k2m[j1]; bl[1] = k2l[j1];
      mma5_b3(t, sml[bb], a2h, a2l, bh, bm, bl);
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[bb][q] += t[q];  // round-to-nearest on the CUDA cores
    }
  }
#pragma unroll
  for (int bb = 0; bb < NTH; ++bb)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[bb][q] += sml[bb][q];

#pragma unroll
  for (int bb = 0; bb < NTH; ++bb) {
    const int b = bfirst + bb;
#pragma unroll
    for (int hrow = 0; hrow < 2; ++hrow) {
      const int n1 = hrow ? nb : na;
      const size_t o = base + (size_t)n1 * NK + 8 * b + 2 * t4;
      float2 v;
      if (MODE == 0) {
        v.x = acc[bb][2 * hrow];
        v.y = acc[bb][2 * hrow + 1];
      } else {
        const float2 hv = *reinterpret_cast<const float2 *>(a.h + o);
        const float2 fv = *reinterpret_cast<const float2 *>(a.base + o);
        v.x = fv.x + fmaf(a.half_tau, acc[bb][2 * hrow], hv.x);
        v.y = fv.y + fmaf(a.half_tau, acc[bb][2 * hrow + 1], hv.y);
      }
      if (sums) {  // the outputs wait in this thread's own Acc slots for the sum's second pass
        em_loc = max(em_loc, max(expo_of(v.x), expo_of(v.y)));
        Acc[n1 * S + 8 * b + 2 * t4] = v.x;
        Acc[n1 * S + 8 * b + 2 * t4 + 1] = v.y;
      }
      *reinterpret_cast<float2 *>(a.out + o) = v;
    }
  }
  }  // active
  if (sums) {
    // exact per-X sum of the outputs, the rule and bits of xsum_block
    int *red = reinterpret_cast<int *>(smu + L::words - 64);
    long long *lred = reinterpret_cast<long long *>(red + 32);
    const int nw = blockDim.x >> 5;
    int em = __reduce_max_sync(0xffffffffu, em_loc);
    if (lane == 0) red[w] = em;
    __syncthreads();
    em = 0;
    for (int q = 0; q < nw; ++q) em = max(em, red[q]);
    em = max(em, 1);
    long long acc2 = 0;
    if (active) {
#pragma unroll
      for (int bb = 0; bb < NTH; ++bb)
#pragma unroll
        for (int hrow = 0; hrow < 2; ++hrow) {
          const int n1 = hrow ? nb : na, c = 8 * (bfirst + bb) + 2 * t4;
          acc2 += fixed_image(Acc[n1 * S + c], em) + fixed_image(Acc[n1 * S + c + 1], em);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc2 += __shfl_xor_sync(0xffffffffu, acc2, o);
    if (lane == 0) lred[w] = acc2;
    __syncthreads();
    if (tid == 0) {
      long long tot = 0;
      for (int q = 0; q < nw; ++q) tot += lred[q];
      a.xsum[X] = em == 255 ? __longlong_as_double(0x7ff8000000000000ll) : ll_to_double_scaled(tot, em - 174);
    }
    __syncthreads();
  }
}

template <int NK, int MODE>
__global__ void __launch_bounds__(NK * 2 * kTh32Split, 1) k_theta32(Theta32Args a) {
  extern __shared__ __align__(16) uint32_t smu[];
  theta32_block<NK, MODE>(a, blockIdx.x, smu);
}

// ---------------------------------------------------------------------------
// Spline shift, FP32
// ---------------------------------------------------------------------------

__device__ __forceinline__ void spline_coeffs32(float *col, int stride, int n, float z, float zscale, int nterm) {
  float c0 = 0.f, zk = 1.f;
  for (int k = 0; k < nterm; ++k) {
    c0 = fmaf(zk, col[((n - k) % n) * stride], c0);
    zk *= z;
  }
  float prev = c0 * zscale;
  col[0] = prev;
  for (int i = 1; i < n; ++i) {
    prev = fmaf(z, prev, col[i * stride]);
    col[i * stride] = prev;
  }
  float dN = 0.f;
  zk = 1.f;
  for (int k = 0; k < nterm; ++k) {
    dN = fmaf(zk, col[((n - 1 + k) % n) * stride], dN);
    zk *= z;
  }
  prev = dN * zscale;
  col[(n - 1) * stride] = prev;
  for (int i = n - 2; i >= 0; --i) {
    prev = fmaf(z, prev, col[i * stride]);
    col[i * stride] = prev;
  }
}

// The same solve on one or two strided columns (c1 may be null) by several
// threads per column: each runs both recursions over its rows [lo, hi) (empty
// for a thread without a piece), started from its own start sums (the same
// periodic sums as above, at the piece's first / last row; with nterm < n
// they drop |z|^nterm < 2^-24 of the tail).  Every thread of the CTA calls
// this: it holds the CTA barriers between the phases.
__device__ __forceinline__ void spline_coeffs32_chunked(float *c0, float *c1, int stride, int n, float z, float zscale,
                                                        int nterm, int lo, int hi) {
  const int nt = hi > lo ? nterm : 0;  // an empty piece reads nothing
  float s0 = 0.f, s1 = 0.f, zk = 1.f;
  for (int k = 0; k < nt; ++k) {
    int idx = lo - k;
    idx += (idx < 0) ? n : 0;
    s0 = fmaf(zk, c0[idx * stride], s0);
    if (c1) s1 = fmaf(zk, c1[idx * stride], s1);
    zk *= z;
  }
  __syncthreads();  // every start sum has read the input line
  if (hi > lo) {
    float p0 = s0 * zscale, p1 = s1 * zscale;
    c0[lo * stride] = p0;
    if (c1) c1[lo * stride] = p1;
    for (int i = lo + 1; i < hi; ++i) {
      p0 = fmaf(z, p0, c0[i * stride]);
      c0[i * stride] = p0;
      if (c1) {
        p1 = fmaf(z, p1, c1[i * stride]);
        c1[i * stride] = p1;
      }
    }
  }
  __syncthreads();
  const int e = hi - 1;
  s0 = s1 = 0.f;
  zk = 1.f;
  for (int k = 0; k < nt; ++k) {
    int idx = e + k;
    idx -= (idx >= n) ? n : 0;
    s0 = fmaf(zk, c0[idx * stride], s0);
    if (c1) s1 = fmaf(zk, c1[idx * stride], s1);
    zk *= z;
  }
  __syncthreads();  // every start sum has read the causal pass
  if (hi > lo) {
    float p0 = s0 * zscale, p1 = s1 * zscale;
    c0[e * stride] = p0;
    if (c1) c1[e * stride] = p1;
    for (int i = e - 1; i >= lo; --i) {
      p0 = fmaf(z, p0, c0[i * stride]);
      c0[i * stride] = p0;
      if (c1) {
        p1 = fmaf(z, p1, c1[i * stride]);
        c1[i * stride] = p1;
      }
    }
  }
  __syncthreads();
}

// (oh, ol) = z (h, l) + (xh, xl) in double-float arithmetic, renormalised by
// Fast2Sum (where the sum cancels, |t| may exceed |s|; the pair then still
// holds s + t to within 2^-48 of the larger input, which is the accuracy the
// line needs).
__device__ __forceinline__ void df_madd(float2 z, float h, float l, float xh, float xl, float &oh, float &ol) {
  float ph, pe, s, t;
  df_mul(z.x, z.y, h, l, ph, pe);
  two_sum(ph, xh, s, t);
  t = __fadd_rn(t, __fadd_rn(pe, xl));
  fast_two_sum(s, t, oh, ol);
}

// Start sum sum_{k < nt} z^k (h, l)[row(k)] of one column, times the periodic
// scale, normalised: double-float products for the terms above 2^-26 of the
// sum's scale (k < 14, |z|^14 < 2^-26), FP32 for the rest (their rounding is
// below 2^-50 of the scale).
template <typename Row>
__device__ __forceinline__ void df_start(const float *ch, const float *cl, int stride, const Adv32Args &a, int nt,
                                         Row row, float &oh, float &ol) {
  float sh = 0.f, se = 0.f, tail = 0.f;
  const int kdf = nt < 14 ? nt : 14;
  for (int k = 0; k < kdf; ++k) {
    const int idx = row(k);
    const float2 zk = __ldg(a.zpow + k);
    float ph, pe;
    df_mul(zk.x, zk.y, ch[idx * stride], cl[idx * stride], ph, pe);
    df_acc(sh, se, ph, pe);
  }
  for (int k = kdf; k < nt; ++k) tail = __fmaf_rn(__ldg(a.zpow + k).x, ch[row(k) * stride], tail);
  two_sum(sh, __fadd_rn(se, tail), sh, se);
  float ph, pe;
  df_mul(a.zscale_df.x, a.zscale_df.y, sh, se, ph, pe);
  two_sum(ph, pe, oh, ol);
}

// The threads that work on one shift slab: the whole CTA (bar < 0:
// __syncthreads), or one group of whole warps of a batch CTA synchronised by
// its own named barrier (several slabs in flight per CTA).
struct SlabGroup {
  int tid, nthr, bar;
  __device__ __forceinline__ void sync() const {
    if (bar < 0)
      __syncthreads();
    else
      asm volatile("bar.sync %0, %1;\n" ::"r"(bar), "r"(nthr) : "memory");
  }
};

// The coefficient solve of spline_coeffs32_chunked in double-float pairs: on
// entry (h0, l0) and (h1, l1) (h1 may be null) hold each line's values as
// (hi, lo) pairs, on return the coefficients d of the causal and anti-causal
// recursions with pole z, started from periodic sums over nterm_df terms
// (exact up to |z|^28 < 2^-53 when nterm_df < n).  Every thread of the CTA
// calls this: it holds the CTA barriers between the phases.
__device__ __forceinline__ void spline_coeffs_df_chunked(float *h0, float *l0, float *h1, float *l1, int stride, int n,
                                                         const Adv32Args &a, int lo, int hi,
                                                         const SlabGroup &gp) {
  const int nt = hi > lo ? a.nterm_df : 0;  // an empty piece reads nothing
  float p0h = 0.f, p0l = 0.f, p1h = 0.f, p1l = 0.f;
  auto back = [lo, n](int k) {
    int idx = lo - k;
    return idx + ((idx < 0) ? n : 0);
  };
  df_start(h0, l0, stride, a, nt, back, p0h, p0l);
  if (h1) df_start(h1, l1, stride, a, nt, back, p1h, p1l);
  gp.sync();  // every start sum has read the input line
  if (hi > lo) {
    h0[lo * stride] = p0h;
    l0[lo * stride] = p0l;
    if (h1) {
      h1[lo * stride] = p1h;
      l1[lo * stride] = p1l;
    }
    for (int i = lo + 1; i < hi; ++i) {
      df_madd(a.zdf, p0h, p0l, h0[i * stride], l0[i * stride], p0h, p0l);
      h0[i * stride] = p0h;
      l0[i * stride] = p0l;
      if (h1) {
        df_madd(a.zdf, p1h, p1l, h1[i * stride], l1[i * stride], p1h, p1l);
        h1[i * stride] = p1h;
        l1[i * stride] = p1l;
      }
    }
  }
  gp.sync();
  const int e = hi - 1;
  auto fwd = [e, n](int k) {
    int idx = e + k;
    return idx - ((idx >= n) ? n : 0);
  };
  df_start(h0, l0, stride, a, nt, fwd, p0h, p0l);
  if (h1) df_start(h1, l1, stride, a, nt, fwd, p1h, p1l);
  gp.sync();  // every start sum has read the causal pass
  if (hi > lo) {
    h0[e * stride] = p0h;
    l0[e * stride] = p0l;
    if (h1) {
      h1[e * stride] = p1h;
      l1[e * stride] = p1l;
    }
    for (int i = e - 1; i >= lo; --i) {
      df_madd(a.zdf, p0h, p0l, h0[i * stride], l0[i * stride], p0h, p0l);
      h0[i * stride] = p0h;
      l0[i * stride] = p0l;
      if (h1) {
        df_madd(a.zdf, p1h, p1l, h1[i * stride], l1[i * stride], p1h, p1l);
        h1[i * stride] = p1h;
        l1[i * stride] = p1l;
      }
    }
  }
  gp.sync();
}

__device__ __forceinline__ int wrap(int j, int n) {
  j %= n;
  return j < 0 ? j + n : j;
}

// Columns in shared memory carry kGhost copies of the periodic neighbours at
// each end (row r holds element r - kGhost), so stencils within kGhost of a
// point read straight rows without wrapping the index.
constexpr int kGhost = 4;

__device__ __forceinline__ void fill_ghosts(float *col, int stride, int n) {
#pragma unroll
  for (int k = 0; k < kGhost; ++k) {
    col[(kGhost + n + k) * stride] = col[(kGhost + k) * stride];
    col[(kGhost - 1 - k) * stride] = col[(kGhost + n - 1 - k) * stride];
  }
}

// S f at i: sum_{a=-1..2} w_a d_{i + k0 + a}; col points at row 0 (ghosts included)
__device__ __forceinline__ float eval32(const float *col, int stride, int n, int i, int k0, const float *w) {
  float v = 0.f;
  if (k0 >= -3 && k0 <= 2) {
    const float *c = col + (kGhost + i + k0 - 1) * stride;
#pragma unroll
    for (int q = 0; q < 4; ++q) v = fmaf(w[q], c[q * stride], v);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) v = fmaf(w[q], col[(kGhost + wrap(i + k0 - 1 + q, n)) * stride], v);
  }
  return v;
}

// (S - I) f at i.  ct[0..6]: merged taps at offsets -3..3, ct[7] = 1 when they
// apply (|k0| small); otherwise the evaluation and the interpolation condition
// are summed separately.
__device__ __forceinline__ float incr32(const float *col, int stride, int n, int i, int k0, const float *w,
                                        const float *ct, float z) {
  const float *c = col + (kGhost + i) * stride;
  if (ct[7] != 0.f) {
    float v = 0.f;
#pragma unroll
    for (int o = -3; o <= 3; ++o) v = fmaf(ct[o + 3], c[o * stride], v);
    return v;
  }
  const float sv = eval32(col, stride, n, i, k0, w);
  const float fi = -z * (c[-stride] + 4.f * c[0] + c[stride]);
  return sv - fi;
}

// DIR 0 (lines along x2 at fixed (i1 = blockIdx.y, n1 = blockIdx.x); the line
// of column n2 is shifted by tau p_{n2}/m):
//   d2 = (S2 - I) f,  g2 = S2 g (when g is given).
// DIR 1 (lines along x1 at fixed (i2 = blockIdx.y, n1 = blockIdx.x); shift
// tau p_{n1}/m), u = f + d2:
//   two arrays: d1 = (S1 - I) u, b = S1 g2, ft = u + d1 + tau b,
//               dh = d2 + d1 + tau/2 b   (dh may overwrite d2 in place)
//   one array : ft = u + d1  (= S1 S2 f)
// Columns (momentum values n2) handled by one CTA of the shift: at most 64, so
// that a slab of a few arrays leaves room for two or three CTAs per SM.
template <int NK>
struct AdvCols {
  static constexpr int C = NK >= 64 ? 64 : NK;
  static constexpr int blocks = NK / C;
};

// Stage rows i = 0..nx-1 of C contiguous floats (global stride lineStride)
// into rows kGhost + i of a shared slab of stride C, 16 bytes per copy, all
// copies of the CTA in flight together.
template <int C>
__device__ __forceinline__ void stage_slab(float *slab, const float *src, size_t lineStride, int nx,
                                           const SlabGroup &gp) {
  constexpr int Q = C / 4;
  for (int e = gp.tid; e < nx * Q; e += gp.nthr) {
    const int i = e / Q, c = 4 * (e - i * Q);
    cp_async16(slab + (kGhost + i) * C + c, src + i * lineStride + c);
  }
}

// DIR 0 (lines along x2 at fixed (i1, n1); the line of column n2 is shifted by
// tau p_{n2}/m):  d2 = (S2 - I) f,  g2 = S2 g (when g is given).
// DIR 1 (lines along x1 at fixed (i2, n1); shift tau p_{n1}/m), u = f + d2:
//   two arrays: d1 = (S1 - I) u, b = S1 g2, ft = u + d1 + tau b,
//               dh = d2 + d1 + tau/2 b   (dh may overwrite d2 in place)
//   one array : ft = u + d1  (= S1 S2 f)
// A group of threads (the CTA, or a group of whole warps of a batch CTA)
// owns columns [cb*C, cb*C + C) of the slab with adv32_pieces(nx) threads per
// column: its thread t takes column t % C and the rows of piece t / C
// (staging, the spline solve in pieces, the evaluation).  Shared memory: the
// staged slabs (FP32) and the lo parts of the two solved arrays (FP32),
// rows nx + 2 kGhost each: 4 slabs for DIR 0, 5 for DIR 1.
template <int DIR>
__host__ __device__ constexpr int adv32_slabs() { return DIR == 0 ? 4 : 5; }

template <int NK, int DIR, int C>
// compiled once (not inlined) so the single-problem and batched kernels
// run the same machine code and give identical bits
__device__ __noinline__ void adv32_block(const Adv32Args &a, const int n1, const int cb, const int fixed,
                                         float *sm32, const SlabGroup &gp) {
  const int nx = a.nx;
  // the pieces depend on nx only, so that every launch shape gives the same bits;
  // threads beyond them idle (a batch launch is sized for its longest lines)
  const int t = gp.tid % C, q = gp.tid / C, P = adv32_pieces(nx);
  const int col = cb * C + t;
  const int rows = nx + 2 * kGhost;
  const int lo = q < P ? (q * nx) / P : 0, hi = q < P ? ((q + 1) * nx) / P : 0;
  const size_t lineStride = (DIR == 0) ? (size_t)NK * NK : (size_t)nx * NK * NK;
  const size_t base = ((DIR == 0) ? ((size_t)fixed * nx * NK + n1) * NK : ((size_t)fixed * NK + n1) * NK) + cb * C;
  const int sidx = (DIR == 0) ? col : n1;
  const int k0 = a.k0tab[sidx];
  float w[4], ct[8];
#pragma unroll
  for (int r = 0; r < 4; ++r) w[r] = a.wtab[4 * sidx + r];
#pragma unroll
  for (int r = 0; r < 8; ++r) ct[r] = a.ctab[8 * sidx + r];
  const size_t slab = (size_t)rows * C;
  float *SA = sm32, *SB = sm32 + slab;
  float *SC = sm32 + 2 * slab;                                // DIR 1 only
  float *LA = sm32 + (DIR == 0 ? 2 : 3) * slab, *L1 = LA + slab;  // lo parts of A and of B (DIR 0) / C (DIR 1)
  float *A = SA + t, *B = SB + t, *Cc = SC + t, *la = LA + t, *l1 = L1 + t;  // this thread's column
  if (DIR == 0) {
    const bool two = a.g != nullptr;
    stage_slab<C>(SA, a.f + base, lineStride, nx, gp);
    if (two) stage_slab<C>(SB, a.g + base, lineStride, nx, gp);
    for (int i = lo; i < hi; ++i) {
      la[(kGhost + i) * C] = 0.f;
      l1[(kGhost + i) * C] = 0.f;
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    gp.sync();
    spline_coeffs_df_chunked(A + kGhost * C, la + kGhost * C, two ? B + kGhost * C : nullptr,
                             two ? l1 + kGhost * C : nullptr, C, nx, a, lo, hi, gp);
    if (gp.tid < C) {
      fill_ghosts(A, C, nx);
      fill_ghosts(la, C, nx);
      if (two) {
        fill_ghosts(B, C, nx);
        fill_ghosts(l1, C, nx);
      }
    }
    gp.sync();
    for (int i = lo; i < hi; ++i) {
      const size_t o = base + i * lineStride + t;
      a.d2[o] = incr32(A, C, nx, i, k0, w, ct, a.z) + incr32(la, C, nx, i, k0, w, ct, a.z);
      if (two) a.g2[o] = eval32(B, C, nx, i, k0, w) + eval32(l1, C, nx, i, k0, w);
    }
  } else {
    const bool two = a.g2in != nullptr;
    stage_slab<C>(SA, a.f + base, lineStride, nx, gp);
    stage_slab<C>(SB, a.d2in + base, lineStride, nx, gp);
    if (two) stage_slab<C>(SC, a.g2in + base, lineStride, nx, gp);
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    gp.sync();
    for (int i = lo; i < hi; ++i) {  // u = f + d2 as an exact pair
      float uh, ul;
      two_sum(A[(kGhost + i) * C], B[(kGhost + i) * C], uh, ul);
      A[(kGhost + i) * C] = uh;
      la[(kGhost + i) * C] = ul;
      l1[(kGhost + i) * C] = 0.f;
    }
    gp.sync();
    spline_coeffs_df_chunked(A + kGhost * C, la + kGhost * C, two ? Cc + kGhost * C : nullptr,
                             two ? l1 + kGhost * C : nullptr, C, nx, a, lo, hi, gp);
    if (gp.tid < C) {
      fill_ghosts(A, C, nx);
      fill_ghosts(la, C, nx);
      if (two) {
        fill_ghosts(Cc, C, nx);
        fill_ghosts(l1, C, nx);
      }
    }
    gp.sync();
    for (int i = lo; i < hi; ++i) {
      const size_t o = base + i * lineStride + t;
      const float d1 = incr32(A, C, nx, i, k0, w, ct, a.z) + incr32(la, C, nx, i, k0, w, ct, a.z);
      // u_i recovered from its spline coefficients: u = (1,4,1)/6 eta = -z (d_{i-1} + 4 d_i + d_{i+1})
      const float *ca = A + (kGhost + i) * C, *cl = la + (kGhost + i) * C;
      const float u = -a.z * (ca[-C] + 4.f * ca[0] + ca[C]) - a.z * (cl[-C] + 4.f * cl[0] + cl[C]);
      if (two) {
        const float b = eval32(Cc, C, nx, i, k0, w) + eval32(l1, C, nx, i, k0, w);
        const float da = B[(kGhost + i) * C] + d1;
        a.ft[o] = u + fmaf(a.tau, b, d1);
        a.dh[o] = fmaf(0.5f * a.tau, b, da);
      } else {
        a.ft[o] = u + d1;
      }
    }
  }
}

// Columns per CTA of the single-problem shift from 128 points per line on: 32
// (16 when nk is an odd multiple of 16), so that five slabs of nx + 2 kGhost
// rows fit and, at 128 points, two or three CTAs share an SM (with 64 columns
// one CTA of 8 warps per SM left the serial recursions latency bound).
template <int NK>
struct AdvColsWide {
  static constexpr int C = NK % 32 == 0 ? 32 : 16;
  static constexpr int blocks = NK / C;
};

// From 256 points per line: 16 columns per CTA (with 16 pieces per line, 256
// threads), so that two CTAs of five 264-row slabs share an SM.
struct AdvColsLong {
  static constexpr int C = 16;
};

template <int NK, int DIR, int C>
__global__ void __launch_bounds__(256) k_adv32(Adv32Args a) {
  extern __shared__ __align__(16) float sm32[];
  constexpr int NB = NK / C;
  adv32_block<NK, DIR, C>(a, blockIdx.x / NB, blockIdx.x % NB, blockIdx.y, sm32,
                          SlabGroup{(int)threadIdx.x, (int)blockDim.x, -1});
}


// ---------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------

bool nk_supported_f32(int nk) { return nk >= 16 && nk <= 128 && nk % 16 == 0; }

template <int NK>
static cudaError_t prep32() {
  cudaError_t e = cudaFuncSetAttribute(k_theta32<NK, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Theta32Smem<NK>::bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_theta32<NK, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Theta32Smem<NK>::bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adv32<NK, 0, AdvCols<NK>::C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adv32<NK, 1, AdvCols<NK>::C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adv32<NK, 0, AdvColsWide<NK>::C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             220 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adv32<NK, 1, AdvColsWide<NK>::C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             220 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adv32<NK, 0, AdvColsLong::C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adv32<NK, 1, AdvColsLong::C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  return e;
}

template <int NK>
static cudaError_t run_theta32(int mode, const Theta32Args &a, cudaStream_t s) {
  dim3 grid(a.nx * a.nx), block(NK * 2 * kTh32Split);
  if (mode == 0)
    k_theta32<NK, 0><<<grid, block, Theta32Smem<NK>::bytes, s>>>(a);
  else
    k_theta32<NK, 1><<<grid, block, Theta32Smem<NK>::bytes, s>>>(a);
  return cudaGetLastError();
}

template <int NK, int C>
static cudaError_t run_adv32_c(int dir, const Adv32Args &a, cudaStream_t s) {
  dim3 grid(NK * (NK / C), a.nx), block(C * adv32_pieces(a.nx));
  const int slabs = dir == 0 ? adv32_slabs<0>() : adv32_slabs<1>();
  const size_t smem = sizeof(float) * (size_t)slabs * (a.nx + 2 * kGhost) * C;
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  if (dir == 0)
    k_adv32<NK, 0, C><<<grid, block, smem, s>>>(a);
  else
    k_adv32<NK, 1, C><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NK>
static cudaError_t run_adv32(int dir, const Adv32Args &a, cudaStream_t s) {
  if (a.nx < 128) return run_adv32_c<NK, AdvCols<NK>::C>(dir, a, s);
  if (a.nx < 256) return run_adv32_c<NK, AdvColsWide<NK>::C>(dir, a, s);
  return run_adv32_c<NK, AdvColsLong::C>(dir, a, s);
}

#define W2_NK32_SWITCH(nk, EXPR_TEMPLATE) \
  switch (nk) {                          \
    case 16: return EXPR_TEMPLATE(16);   \
    case 32: return EXPR_TEMPLATE(32);   \
    case 48: return EXPR_TEMPLATE(48);   \
    case 64: return EXPR_TEMPLATE(64);   \
    case 80: return EXPR_TEMPLATE(80);   \
    case 96: return EXPR_TEMPLATE(96);   \
    case 112: return EXPR_TEMPLATE(112); \
    case 128: return EXPR_TEMPLATE(128); \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t prepare_kernels_f32(int nk) {
#define W2_P(N) prep32<N>()
  W2_NK32_SWITCH(nk, W2_P)
#undef W2_P
}

cudaError_t launch_theta_f32(int nk, int mode, const Theta32Args &a, cudaStream_t s) {
#define W2_T(N) run_theta32<N>(mode, a, s)
  W2_NK32_SWITCH(nk, W2_T)
#undef W2_T
}

cudaError_t launch_adv_f32(int nk, int dir, const Adv32Args &a, cudaStream_t s) {
#define W2_A(N) run_adv32<N>(dir, a, s)
  W2_NK32_SWITCH(nk, W2_A)
#undef W2_A
}


// ---------------------------------------------------------------------------
// Batch step: one persistent launch per Lawson step of every instance
// ---------------------------------------------------------------------------


int bstep_shift_items(int nk, int shift_cols) { return nk / bstep_cols(nk, shift_cols); }

// Largest k with off[k] <= item among off[0..n] (off ascending, off[0] = 0).
__device__ __forceinline__ int bsearch_inst(const int *off, int n, int item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Warps per 16-row block of a batch Theta item: with TS = 2, as many as the
// 8 warps of the CTA allow (NK / 16 row blocks; the count must divide the
// NK / 8 column tiles), so that NK = 32 keeps every warp busy (4 per row
// block) instead of half of them; TS = 1 keeps one.  The split does not
// change the bits.
__host__ __device__ constexpr int bstep_tsplit(int nk, int ts) {
  return ts == 1 ? 1 : (nk / 8) % (kBatchThreads / 32 / (nk / 16)) == 0 ? kBatchThreads / 32 / (nk / 16) : 2;
}

template <int NK, int TS>
__device__ __forceinline__ void bstep_theta(const BStepPlan &P, int p, int i, int j, unsigned char *sm) {
  constexpr int SPLIT = bstep_tsplit(NK, TS);
  if (p == 1) theta32_block<NK, 0, SPLIT>(P.th[2 * i], j, reinterpret_cast<uint32_t *>(sm));
  else theta32_block<NK, 1, SPLIT>(P.th[2 * i + 1], j, reinterpret_cast<uint32_t *>(sm));
}

// Shift units [u0, u1) of instance i (phase 2: x2 pass, 3: x1 pass).  The
// slab's adv32_pieces(nx) x C threads, rounded up to whole warps, form a
// group; as many groups as fit the CTA's threads and shared memory (at most
// eight) take the units in turn, each in its own part of shared memory and
// with its own named barrier, so small lines do not leave most of the CTA
// idle.  Threads outside the groups return at once.
template <int NK, int CS>
__device__ __forceinline__ void bstep_shift(const BStepPlan &P, int p, int i, int u0, int u1, unsigned char *sm) {
  constexpr int C = bstep_cols(NK, CS);
  constexpr int NB = NK / C;
  const int nx = P.nx[i];
  const int S = (C * adv32_pieces(nx) + 31) & ~31;
  if (S > (int)blockDim.x) {  // the host refuses such shapes; never wait on a barrier that cannot fill
    if (threadIdx.x == 0) atomicCAS(P.err, 0, (int)W2_ERR_UNSUPPORTED);
    return;
  }
  const size_t slab_bytes =
      ((size_t)(p == 2 ? adv32_slabs<0>() : adv32_slabs<1>()) * (nx + 2 * kGhost) * C * sizeof(float) + 15) & ~(size_t)15;
  const int G = max(1, min(min((int)blockDim.x / S, (int)(P.smem / slab_bytes)), 8));
  const int grp = threadIdx.x / S;
  if (grp >= G) return;
  const SlabGroup gp{(int)threadIdx.x - grp * S, S, 1 + grp};
  float *sm32 = reinterpret_cast<float *>(sm + grp * slab_bytes);
  for (int u = u0 + grp; u < u1; u += G) {
    if (p == 2)
      adv32_block<NK, 0, C>(P.adv[2 * i], (u / NB) % NK, u % NB, (u / NB) / NK, sm32, gp);
    else
      adv32_block<NK, 1, C>(P.adv[2 * i + 1], (u / NB) % NK, u % NB, (u / NB) / NK, sm32, gp);
    gp.sync();  // the group's slabs are free again
  }
}

template <int CS, int TS>
__global__ void __launch_bounds__(kBatchThreads, 2) k_bstep(BStepPlan P) {
  extern __shared__ __align__(16) unsigned char smb[];
  __shared__ int s_item, s_ok;
  const int total = P.phase_off[kBatchPhases];
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(P.next, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    int p = 0;
    while (item >= P.phase_off[p + 1]) ++p;
    const int *io = P.inst_off + p * (P.n + 1);
    const int local = item - P.phase_off[p];
    const int i = bsearch_inst(io, P.n, local);
    const int j = local - io[i];
    if (threadIdx.x == 0) {
      int ok = *(volatile int *)P.err == 0;
      if (ok && p > 0) {
        const int *po = P.inst_off + (p - 1) * (P.n + 1);
        const int target = po[i + 1] - po[i];
        const volatile int *d = P.done + (p - 1) * P.n + i;
        const long long t0 = clock64();
        while (*d < target) {
          if (*(volatile int *)P.err) {
            ok = 0;
            break;
          }
          if (clock64() - t0 > P.wait_cycles) {
            atomicCAS(P.err, 0, (int)W2_ERR_TIMEOUT);
            ok = 0;
            break;
          }
          __nanosleep(128);
        }
        __threadfence();  // the finished items' writes are seen before this item reads them
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    const int nk = P.nk[i], g = P.gsz[p];
    const int u0 = j * g, u1 = min((j + 1) * g, P.units[p * P.n + i]);
    if (p == 2 || p == 3) {
      switch (nk) {
        case 16: bstep_shift<16, CS>(P, p, i, u0, u1, smb); break;
        case 32: bstep_shift<32, CS>(P, p, i, u0, u1, smb); break;
        case 48: bstep_shift<48, CS>(P, p, i, u0, u1, smb); break;
        case 64: bstep_shift<64, CS>(P, p, i, u0, u1, smb); break;
        default: break;
      }
      __syncthreads();  // every group's writes are issued; shared memory is free again
    } else {
      for (int u = u0; u < u1; ++u) {
        if (p == 4) {
          const BXsum &a = P.xs_ft[i];
          xsum_block<float, 16>(a.f, a.xsum, a.nk, u, reinterpret_cast<double *>(smb));
        } else if (p == 0 || p == 5) {
          const int nx = P.nx[i];
          tables_block(P.tab[i], u % nx, u / nx, reinterpret_cast<double *>(smb));
        } else {
          switch (nk) {
            case 16: bstep_theta<16, TS>(P, p, i, u, smb); break;
            case 32: bstep_theta<32, TS>(P, p, i, u, smb); break;
            case 48: bstep_theta<48, TS>(P, p, i, u, smb); break;
            case 64: bstep_theta<64, TS>(P, p, i, u, smb); break;
            default: break;
          }
        }
        __syncthreads();  // every thread's writes of this unit are issued; shared memory is free again
      }
    }
    if (threadIdx.x == 0) {
      __threadfence();
      if (!(P.skip && *P.skip == 1 + p * P.n + i)) atomicAdd(P.done + p * P.n + i, 1);
    }
  }
  // the last CTA to leave resets the counters for the next launch
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(P.left, 1) == (int)gridDim.x - 1) {
      for (int k = 0; k < kBatchPhases * P.n; ++k) P.done[k] = 0;
      *P.next = 0;
      *P.left = 0;
      __threadfence();
    }
  }
}

template <int CS, int TS>
static cudaError_t prep_bstep_v() {
  return cudaFuncSetAttribute(k_bstep<CS, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
}

#define W2_BSTEP_SWITCH(sh, EXPR)                                       \
  if (sh.shift_cols == 64 && sh.theta_split == 2) return EXPR(64, 2);  \
  if (sh.shift_cols == 64 && sh.theta_split == 1) return EXPR(64, 1);  \
  if (sh.shift_cols == 32 && sh.theta_split == 2) return EXPR(32, 2);  \
  if (sh.shift_cols == 32 && sh.theta_split == 1) return EXPR(32, 1);  \
  return cudaErrorInvalidValue;

cudaError_t prepare_bstep(const BStepShape &sh) {
#define W2_PB(CS, TS) prep_bstep_v<CS, TS>()
  W2_BSTEP_SWITCH(sh, W2_PB)
#undef W2_PB
}

// Shared memory of the persistent step: the largest of its items' needs
// (shift: five slabs of nx + 2 kGhost rows; Theta: the split block; tables:
// densities and fine-point potentials; per-X sums: 256 doubles).
// Shared memory of a batch CTA: the largest single unit (a Theta block or a
// shift slab set), and at least 110 KB while two CTAs still fit an SM, so
// that several shift slabs of the smaller instances are in flight at once.
size_t bstep_smem(const BStepShape &sh, int nxmax, int nkmax) {
  size_t m = 256 * sizeof(double);
  m = std::max(m, sizeof(double) * (size_t)(nxmax + 2 * nkmax));
  for (int nk = 16; nk <= nkmax; nk += 16) {
    const size_t th = 4 * (3 * (size_t)nk * (nk + 8) + 9 * 2 * nk + 64);
    const size_t ad = sizeof(float) * 5 * (size_t)(nxmax + 2 * kGhost) * bstep_cols(nk, sh.shift_cols);
    m = std::max(m, std::max(th, ad));
  }
  return std::max(m, (size_t)110 * 1024);
}

int bstep_max_ctas_per_sm(const BStepShape &sh, size_t smem) {
  int n = 0;
#define W2_OC(CS, TS) \
  (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_bstep<CS, TS>, kBatchThreads, smem) == cudaSuccess ? n : 0)
  if (sh.shift_cols == 64 && sh.theta_split == 2) return W2_OC(64, 2);
  if (sh.shift_cols == 64 && sh.theta_split == 1) return W2_OC(64, 1);
  if (sh.shift_cols == 32 && sh.theta_split == 2) return W2_OC(32, 2);
  if (sh.shift_cols == 32 && sh.theta_split == 1) return W2_OC(32, 1);
#undef W2_OC
  return 0;
}

cudaError_t launch_bstep(const BStepShape &sh, const BStepPlan &p, int grid, size_t smem, cudaStream_t s) {
  if (smem > 220 * 1024 || grid < 1) return cudaErrorInvalidValue;
#define W2_LB(CS, TS) (k_bstep<CS, TS><<<grid, kBatchThreads, smem, s>>>(p), cudaGetLastError())
  W2_BSTEP_SWITCH(sh, W2_LB)
#undef W2_LB
}

}  // namespace w2
