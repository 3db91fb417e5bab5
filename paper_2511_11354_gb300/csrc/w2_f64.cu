// FP64 kernels of the periodic two-body Wigner 2-RDM step (sm_103a).
//
//  k_tables   : densities -> one-body potential on the fine points -> the real
//               shift kernels K(x, j) of the pseudo-difference operator
//               (Sec. 3.1, Eqs. Hartree_FSM and two_body_FSM).
//  k_theta    : X-local sweep.  Per phase-space point X = (x1, x2) the
//               operator is three Toeplitz contractions of the nk x nk block
//               F(p1, p2): K1(x1) along p1, K2(x2) along p2 and K12(x1 - x2)
//               along the anti-diagonal p1 + p2 = const (the two-body shift
//               (p1 + j dp, p2 - j dp)).  They run on the FP64 tensor path
//               (mma.sync m8n8k4 f64), the anti-diagonal one after shearing
//               the block in shared memory.  Fused epilogue: the Lawson
//               corrector combination and the per-X momentum sums.
//  k_adv      : P-local sweep.  Periodic cubic B-spline shift (Sec. 4.1) of
//               every x-line by tau p / m, one axis per launch; the spline
//               coefficients come from the causal/anti-causal factorisation
//               of the (1, 4, 1)/6 circulant with exact periodic start values.
#include <math.h>

#include "w2_blocks.cuh"
#include "w2_internal.cuh"

namespace w2 {

// ---------------------------------------------------------------------------
// Tables
// ---------------------------------------------------------------------------

__global__ void k_tables(TabArgs a) {
  extern __shared__ double sm[];
  tables_block(a, blockIdx.x, blockIdx.y, sm);
}

cudaError_t launch_tables(const TabArgs &a, cudaStream_t s) {
  dim3 grid(a.nx, a.pair_mode ? 1 : 2);
  size_t smem = sizeof(double) * (a.nx + a.M);
  k_tables<<<grid, 512, smem, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Theta sweep on the FP64 tensor path
// ---------------------------------------------------------------------------

// D(8x8) += A(8x4) B(4x8), FP64.  Fragments (PTX ISA, mma.m8n8k4 .f64):
// a = A[lane>>2][lane&3], b = B[lane&3][lane>>2],
// d0, d1 = D[lane>>2][2*(lane&3) + {0,1}].
__device__ __forceinline__ void dmma(double &d0, double &d1, double a, double b) {
  asm("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
      : "+d"(d0), "+d"(d1)
      : "d"(a), "d"(b));
}

template <int NK>
struct ThetaSmem {
  static constexpr int T = NK / 8;     // 8x8 tiles per momentum axis
  static constexpr int S = NK + 4;     // padded row stride (doubles): 2 wavefronts per fragment load
  static constexpr int doubles = 2 * NK * S + 3 * 2 * NK + 32;
  static constexpr size_t bytes = sizeof(double) * doubles;
};

// One CTA per spatial point X; warp w owns momentum rows n1 in [8w, 8w+8).
// mode 0: out = Theta[in].  mode 1: out = h + half_tau * Theta[in] and, when
// xsum is given, xsum[X] = sum_P out (the exact fixed-point sum of xsum_block).
template <int NK, int MODE>
__global__ void __launch_bounds__(NK * 4) k_theta(ThetaArgs a) {
  using L = ThetaSmem<NK>;
  constexpr int T = L::T, S = L::S;
  extern __shared__ __align__(16) double sm[];
  double *F = sm;               // [NK][S] input block
  double *Acc = F + NK * S;     // [NK][S] two-body term, unsheared
  double *k1 = Acc + NK * S;    // [2NK] K1(x1, j + NK - 1)
  double *k2 = k1 + 2 * NK;
  double *k12 = k2 + 2 * NK;
  double *red = k12 + 2 * NK;   // [32] (the per-X sum's scratch)

  const int nx = a.nx;
  const int X = blockIdx.x;
  const int i1 = X / nx, i2 = X - i1 * nx;
  int dd = i1 - i2;
  dd += (dd < 0) ? nx : 0;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int g = lane >> 2, t4 = lane & 3;

  const size_t base = (size_t)X * NK * NK;
  {
    const double2 *src = reinterpret_cast<const double2 *>(a.in + base);
    for (int e = tid; e < NK * NK / 2; e += blockDim.x) {
      double2 v = src[e];
      int r = (2 * e) / NK, c = (2 * e) - r * NK;
      F[r * S + c] = v.x;
      F[r * S + c + 1] = v.y;
    }
    const int W = 2 * NK - 1;
    for (int j = tid; j < W; j += blockDim.x) {
      k1[j] = a.K1[(size_t)i1 * W + j];
      k2[j] = a.K2[(size_t)i2 * W + j];
      k12[j] = a.K12[(size_t)dd * W + j];
    }
  }
  __syncthreads();

  const int n1 = 8 * w + g;  // A-fragment / D-fragment row of this lane

  // Two-body term in sheared coordinates: T12'(n1, s) = sum_{n1'} K12(n1' - n1)
  // G(n1', s), G(n1', s) = F(n1', s - n1') (zero outside the window).  Output
  // tiles s in [8c, 8c + 8) with c in [w, w + T] cover every valid n2 = s - n1.
  // A supplied two-body term (the learned form) replaces it.
  if (a.pair) {
    for (int e = lane; e < 8 * NK; e += 32) {
      const int r = 8 * w + e / NK, c = e % NK;
      Acc[r * S + c] = (double)a.pair[base + (size_t)r * NK + c];
    }
  }
  for (int c = w; c <= w + T && !a.pair; ++c) {
    double d0 = 0.0, d1 = 0.0;
    const int nlo = max(0, 8 * c - NK + 1), nhi = min(NK - 1, 8 * c + 7);
    const int s = 8 * c + g;  // B-fragment column
    for (int k = nlo >> 2; k <= (nhi >> 2); ++k) {
      const int n1p = 4 * k + t4;
      const double av = k12[n1p - n1 + NK - 1];
      const int n2 = s - n1p;
      const double bv = (n2 >= 0 && n2 < NK) ? F[n1p * S + n2] : 0.0;
      dmma(d0, d1, av, bv);
    }
    const int n2a = 8 * c + 2 * t4 - n1;
    if (n2a >= 0 && n2a < NK) Acc[n1 * S + n2a] = d0;
    if (n2a + 1 >= 0 && n2a + 1 < NK) Acc[n1 * S + n2a + 1] = d1;
  }
  __syncwarp();

  // One-body terms: T1 = A1(x1) F, T2 = F A2(x2)^T, accumulated on top of T12.
  double acc[T][2];
#pragma unroll
  for (int b = 0; b < T; ++b) {
    acc[b][0] = Acc[n1 * S + 8 * b + 2 * t4];
    acc[b][1] = Acc[n1 * S + 8 * b + 2 * t4 + 1];
  }
#pragma unroll 2
  for (int k = 0; k < NK / 4; ++k) {
    const int kk = 4 * k + t4;
    const double a1 = k1[kk - n1 + NK - 1];   // A1[n1][n1'] = K1(n1' - n1)
    const double a2 = F[n1 * S + kk];          // F[n1][n2']
#pragma unroll
    for (int b = 0; b < T; ++b) {
      const double b1 = F[kk * S + 8 * b + g];         // F[n1'][n2]
      dmma(acc[b][0], acc[b][1], a1, b1);
      const double b2 = k2[kk - (8 * b + g) + NK - 1]; // K2(n2' - n2)
      dmma(acc[b][0], acc[b][1], a2, b2);
    }
  }

  // Epilogue.
  double held[2 * T];
#pragma unroll
  for (int b = 0; b < T; ++b) {
    const size_t o = base + (size_t)n1 * NK + 8 * b + 2 * t4;
    double2 v;
    if (MODE == 0) {
      v.x = acc[b][0];
      v.y = acc[b][1];
    } else {
      const double2 hv = *reinterpret_cast<const double2 *>(a.h + o);
      v.x = hv.x + a.half_tau * acc[b][0];
      v.y = hv.y + a.half_tau * acc[b][1];
    }
    held[2 * b] = v.x;
    held[2 * b + 1] = v.y;
    *reinterpret_cast<double2 *>(a.out + o) = v;
  }
  if (MODE == 1 && a.xsum) block_exact_sum(held, a.xsum + X, reinterpret_cast<int *>(red));
}

template <int NK>
static cudaError_t prep_theta() {
  cudaError_t e = cudaFuncSetAttribute(k_theta<NK, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)ThetaSmem<NK>::bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_theta<NK, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)ThetaSmem<NK>::bytes);
}

template <int NK>
static cudaError_t run_theta(int mode, const ThetaArgs &a, cudaStream_t s) {
  dim3 grid(a.nx * a.nx), block(NK * 4);
  if (mode == 0)
    k_theta<NK, 0><<<grid, block, ThetaSmem<NK>::bytes, s>>>(a);
  else
    k_theta<NK, 1><<<grid, block, ThetaSmem<NK>::bytes, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Characteristic shift (periodic cubic B-spline), one axis per launch
// ---------------------------------------------------------------------------

// Spline-coefficient solve in place on a strided column (length n):
// (1, 4, 1)/6 eta = f  ==>  eta = -6 z d, with the causal pass
// c_i = f_i + z c_{i-1} and the anti-causal pass d_i = c_i + z d_{i+1}; both
// started from their exact periodic values (geometric sums over the period).
// The factor -6 z is folded into the evaluation weights.
__device__ __forceinline__ void spline_coeffs(double *col, int stride, int n, double z, double zscale,
                                              int nterm) {
  double c0 = 0.0, zk = 1.0;
  for (int k = 0; k < nterm; ++k) {
    int idx = (n - k) % n;
    c0 += zk * col[idx * stride];
    zk *= z;
  }
  double prev = c0 * zscale;
  col[0] = prev;
  for (int i = 1; i < n; ++i) {
    prev = fma(z, prev, col[i * stride]);
    col[i * stride] = prev;
  }
  double dN = 0.0;
  zk = 1.0;
  for (int k = 0; k < nterm; ++k) {
    int idx = (n - 1 + k) % n;
    dN += zk * col[idx * stride];
    zk *= z;
  }
  prev = dN * zscale;
  col[(n - 1) * stride] = prev;
  for (int i = n - 2; i >= 0; --i) {
    prev = fma(z, prev, col[i * stride]);
    col[i * stride] = prev;
  }
}

// Value of the spline at x_i - shift: sum_{a=-1..2} w_a d_{(i + k0 + a) mod n}.
__device__ __forceinline__ double spline_eval(const double *col, int stride, int n, int i, int k0,
                                              double w0, double w1, double w2, double w3) {
  int j = (i + k0 - 1) % n;
  j += (j < 0) ? n : 0;
  double v = w0 * col[j * stride];
  j = (j + 1 == n) ? 0 : j + 1;
  v = fma(w1, col[j * stride], v);
  j = (j + 1 == n) ? 0 : j + 1;
  v = fma(w2, col[j * stride], v);
  j = (j + 1 == n) ? 0 : j + 1;
  v = fma(w3, col[j * stride], v);
  return v;
}

// DIR 0: lines along x2 at fixed (i1 = blockIdx.y, n1 = blockIdx.x); the
//        shift of line n2 is tau p_{n2} / m.
// DIR 1: lines along x1 at fixed (i2 = blockIdx.y, n1 = blockIdx.x); the
//        shift of every line is tau p_{n1} / m.
// TWO: shift in0 and in1 together.  With DIR 1 and TWO the outputs are
//      out0 = a + tau b, out1 = a + tau/2 b (a = shifted in0, b = shifted in1).
// One thread per momentum column n2; the slab [x][n2] is staged in shared memory.
template <int NK, int DIR, int TWO>
__global__ void __launch_bounds__(NK) k_adv(AdvArgs a) {
  constexpr int S = NK + 1;
  extern __shared__ double sm[];
  const int nx = a.nx;
  double *A0 = sm, *A1 = sm + (size_t)nx * S;
  const int n1 = blockIdx.x, fixed = blockIdx.y, t = threadIdx.x;
  const size_t lineStride = (DIR == 0) ? (size_t)NK * NK : (size_t)nx * NK * NK;
  const size_t base = (DIR == 0) ? ((size_t)fixed * nx * NK + n1) * NK   // i1 fixed
                                 : ((size_t)fixed * NK + n1) * NK;       // i2 fixed
  for (int i = 0; i < nx; ++i) {
    A0[i * S + t] = a.in0[base + i * lineStride + t];
    if (TWO) A1[i * S + t] = a.in1[base + i * lineStride + t];
  }
  const int sidx = (DIR == 0) ? t : n1;
  const int k0 = a.k0tab[sidx];
  const double w0 = a.wtab[4 * sidx], w1 = a.wtab[4 * sidx + 1], w2 = a.wtab[4 * sidx + 2],
               w3 = a.wtab[4 * sidx + 3];
  spline_coeffs(A0 + t, S, nx, a.z, a.zscale, a.nterm);
  if (TWO) spline_coeffs(A1 + t, S, nx, a.z, a.zscale, a.nterm);
  for (int i = 0; i < nx; ++i) {
    const double va = spline_eval(A0 + t, S, nx, i, k0, w0, w1, w2, w3);
    const size_t o = base + i * lineStride + t;
    if (!TWO) {
      a.out0[o] = va;
    } else {
      const double vb = spline_eval(A1 + t, S, nx, i, k0, w0, w1, w2, w3);
      if (DIR == 0) {
        a.out0[o] = va;
        a.out1[o] = vb;
      } else {
        a.out0[o] = fma(a.tau, vb, va);
        a.out1[o] = fma(0.5 * a.tau, vb, va);
      }
    }
  }
}

template <int NK>
static cudaError_t prep_adv(int smem_max) {
  cudaError_t e = cudaSuccess;
#define W2_ADV_ATTR(D, T2)                                                                 \
  e = cudaFuncSetAttribute(k_adv<NK, D, T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           smem_max);                                                      \
  if (e != cudaSuccess) return e;
  W2_ADV_ATTR(0, 0) W2_ADV_ATTR(0, 1) W2_ADV_ATTR(1, 0) W2_ADV_ATTR(1, 1)
#undef W2_ADV_ATTR
  return e;
}

template <int NK>
static cudaError_t run_adv(int dir, int two, const AdvArgs &a, cudaStream_t s) {
  dim3 grid(NK, a.nx), block(NK);
  size_t smem = sizeof(double) * (size_t)(two ? 2 : 1) * a.nx * (NK + 1);
  if (dir == 0 && !two) k_adv<NK, 0, 0><<<grid, block, smem, s>>>(a);
  if (dir == 0 && two) k_adv<NK, 0, 1><<<grid, block, smem, s>>>(a);
  if (dir == 1 && !two) k_adv<NK, 1, 0><<<grid, block, smem, s>>>(a);
  if (dir == 1 && two) k_adv<NK, 1, 1><<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Dispatch on nk
// ---------------------------------------------------------------------------

bool nk_supported_f64(int nk) { return nk >= 8 && nk <= 64 && nk % 8 == 0; }

#define W2_NK_SWITCH(nk, CALL)       \
  switch (nk) {                      \
    case 8: return CALL<8>;          \
    case 16: return CALL<16>;        \
    case 24: return CALL<24>;        \
    case 32: return CALL<32>;        \
    case 40: return CALL<40>;        \
    case 48: return CALL<48>;        \
    case 56: return CALL<56>;        \
    case 64: return CALL<64>;        \
    default: return cudaErrorInvalidValue; \
  }

template <int NK>
static cudaError_t prep_all() {
  cudaError_t e = prep_theta<NK>();
  if (e != cudaSuccess) return e;
  return prep_adv<NK>(200 * 1024);
}

cudaError_t prepare_kernels_f64(int nk) {
#define W2_CALL_PREP(N) prep_all<N>()
  switch (nk) {
    case 8: return W2_CALL_PREP(8);
    case 16: return W2_CALL_PREP(16);
    case 24: return W2_CALL_PREP(24);
    case 32: return W2_CALL_PREP(32);
    case 40: return W2_CALL_PREP(40);
    case 48: return W2_CALL_PREP(48);
    case 56: return W2_CALL_PREP(56);
    case 64: return W2_CALL_PREP(64);
    default: return cudaErrorInvalidValue;
  }
#undef W2_CALL_PREP
}

cudaError_t launch_theta_f64(int nk, int mode, const ThetaArgs &a, cudaStream_t s) {
  switch (nk) {
    case 8: return run_theta<8>(mode, a, s);
    case 16: return run_theta<16>(mode, a, s);
    case 24: return run_theta<24>(mode, a, s);
    case 32: return run_theta<32>(mode, a, s);
    case 40: return run_theta<40>(mode, a, s);
    case 48: return run_theta<48>(mode, a, s);
    case 56: return run_theta<56>(mode, a, s);
    case 64: return run_theta<64>(mode, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_adv_f64(int nk, int dir, int two, const AdvArgs &a, cudaStream_t s) {
  switch (nk) {
    case 8: return run_adv<8>(dir, two, a, s);
    case 16: return run_adv<16>(dir, two, a, s);
    case 24: return run_adv<24>(dir, two, a, s);
    case 32: return run_adv<32>(dir, two, a, s);
    case 40: return run_adv<40>(dir, two, a, s);
    case 48: return run_adv<48>(dir, two, a, s);
    case 56: return run_adv<56>(dir, two, a, s);
    case 64: return run_adv<64>(dir, two, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace w2
