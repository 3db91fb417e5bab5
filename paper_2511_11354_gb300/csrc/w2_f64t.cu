// FP64-accurate pseudo-difference sweep on the 5th-generation tensor cores:
// the exact 8-bit slice scheme of k_theta_s (w2_f64s.cu; Ozaki, Ogita, Oishi
// and Rump, Numer. Algorithms 59, 2012, with fixed-point digits) with every
// digit product on tcgen05.mma (kind::f16, BF16 operands in shared memory,
// FP32 accumulators in tensor memory), for N_k = 64.  Persistent CTAs of 512
// threads, one per SM (215 KB of shared memory, all 512 TMEM columns), each
// taking a run of consecutive spatial points X.
//
// The three Toeplitz contractions of Eq. Hartree_FSM / Eq. two_body_FSM for
// the block F = f(X, ., .) and the kernel rows K1(x1), K2(x2), K12(x1 - x2):
//   T1[n1][n2]  = sum_k K1(k - n1) F[k][n2]            (A1 F)
//   T2[n1][n2]  = sum_m F[n1][m] K2(m - n2)            (F B2)
//   T12[n1][n2] = sum_k K12(k - n1) F[k][n1 + n2 - k]  (sheared)
// each a sum over digit pairs (s, t), s + t <= 5, of products of the state's
// digit plane F_s and the kernel's digit t.
//
// One-body terms, 128-row MMAs by stacking two digits along M:
//   T1: A = [A1_t ; A1_(t+1)] (two Toeplitz digit matrices), B = F_s;
//   T2: A = [F_s ; F_(s+1)] (two digit planes), B = B2_t;
// the top 64 rows give the pair of diagonal d = s + t, the bottom 64 rows the
// pair of diagonal d + 1, and every such "domino" has an even top diagonal
// (stacking starts at t or s = 0, 2, 4 for an even other digit and at -1, 1,
// 3 for an odd one, digit -1 being a zero matrix), so three accumulators
// Q0, Q2, Q4 of 128 lanes x 64 columns take all 21 pairs of both terms:
// lanes 0-63 of Q_e hold diagonal e, lanes 64-127 diagonal e + 1.
//
// Two-body term, transposed so that the sheared index c = n1 + n2 (0..126)
// runs along M:
//   T12^T[c][n1] = sum_k' G_s[c][k'] H_t[k'][n1],
//   G_s[c][k'] = F_s[63 - k'][c - 63 + k'] (zero outside the block),
//   H_t[k'][n1] = K12_t(63 - k' - n1),
// with k' = 63 - k.  H_t is a Hankel matrix: its 8 x 8 core matrices depend
// on the sum of their indices only, so 15 of them (1920 bytes) describe it
// with both descriptor strides 128 bytes.  G_s is built per digit into one of
// two buffers while the tensor core works on the other.  Accumulators: one per
// diagonal 0..3 and one for diagonals 4 and 5 together (the d = 5 products
// take a 2^-8 copy of the K12 digits, as in k_theta_s), 64 columns each.
//
// Exactness is that of k_theta_s: every accumulator half holds a subset of one
// diagonal's products, integers below 2^24, except the two-body d = 4 / 5
// accumulator whose rounding lies below 2^-50 of the block scale.  The
// diagonals are recombined in int64 in units of 2^-4 of a d = 4 unit (the
// d = 5 part rounded to that unit), the two-body part added through shared
// memory at (n1, c - n1), and converted to FP64 with integer operations.
//
// Every wait is bounded (about a second, or a.wait_limit clocks); on time-out
// the CTA stops issuing, waits for the products it did issue, marks its
// outputs NaN (this block and the rest of its run), sets a.err if given, and
// still releases its tensor memory.
#include <math.h>
#include <stdint.h>

#include "w2_slice.cuh"
#include "w2_umma.cuh"

namespace w2 {
namespace {

using slice::kDig;

constexpr int NK = 64, THREADS = 512, PER = NK * NK / THREADS;
constexpr int ISSUER = THREADS / 32 - 1, BUILDERS = THREADS - 32;  // the last warp issues the products
constexpr uint32_t MAT = NK * NK * 2;       // one 64 x 64 BF16 matrix, tiled
constexpr uint32_t HMAT = 15 * 128;         // one Hankel matrix (15 core matrices)
constexpr uint32_t GMAT = 2 * NK * NK * 2;  // one sheared plane, 128 x 64
// shared memory map (bytes)
constexpr uint32_t OFF_F = 0;                      // [zero, F_0 .. F_5]; in the epilogue the mirror staging after the zero
constexpr uint32_t OFF_T1 = OFF_F + 7 * MAT;       // [zero, A1_0 .. A1_5] (kept along a row of blocks)
constexpr uint32_t OFF_B2 = OFF_T1 + 7 * MAT;      // [B2_0 .. B2_5]; in the epilogue the int64 sums I12
constexpr uint32_t OFF_H = OFF_B2 + 6 * MAT;       // [H_0 .. H_5, H'_0 .. H'_5] (H' = 2^-8 H)
constexpr uint32_t OFF_G = OFF_H + 12 * HMAT;      // two sheared planes; the digit tables before
constexpr uint32_t OFF_MISC = OFF_G + 2 * GMAT;    // mbarriers, TMEM address, reduction scratch
constexpr uint32_t SMEM = OFF_MISC + 512;
static_assert(OFF_G % 16 == 0 && OFF_H % 16 == 0, "operands on 16-byte boundaries");
static_assert(SMEM <= 227 * 1024, "shared memory");
static_assert(NK * 65 * 8 <= 6 * MAT, "epilogue buffers fit (I12 in B2, the mirror staging in F_0 .. F_5)");
constexpr int IST = NK + 1;                        // row stride of I12 and of the mirror staging
// TMEM columns: Q0, Q2, Q4 (one-body), then the two-body diagonals 0..3 and 4/5
constexpr uint32_t COL_Q = 0, COL_P = 192;
constexpr long long WAIT_LIMIT = 2000000000ll;     // SM clocks, about a second

// Byte offset of element (r, c) of a tiled matrix with ncol columns.
__device__ __forceinline__ uint32_t toff(int r, int c, int ncol) { return umma::tile_off(r, c, ncol); }

// The eight 16-bit entries tab[i0 .. i0 + 7] of a table of 32-bit words (two
// entries each, entry 2j in the low half of word j) as four words.
__device__ __forceinline__ uint4 window8(const uint32_t *tab, int i0) {
  const int p = i0 >> 1;
  uint32_t w0 = tab[p], w1 = tab[p + 1], w2 = tab[p + 2], w3 = tab[p + 3];
  if (i0 & 1) {
    const uint32_t w4 = tab[p + 4];
    w0 = __funnelshift_r(w0, w1, 16);
    w1 = __funnelshift_r(w1, w2, 16);
    w2 = __funnelshift_r(w2, w3, 16);
    w3 = __funnelshift_r(w3, w4, 16);
  }
  return make_uint4(w0, w1, w2, w3);
}

// Entries [o, o + 8) of the 16 entries (lo, hi), o in [0, 8).
__device__ __forceinline__ uint4 shift8(uint4 lo, uint4 hi, int o) {
  const uint32_t W[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
  const int h = o >> 1;
  uint32_t a[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) a[i] = h == 0 ? W[i] : h == 1 ? W[i + 1] : h == 2 ? W[i + 2] : W[min(i + 3, 7)];
  if (o & 1) {
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = __funnelshift_r(a[i], a[i + 1], 16);
  }
  return make_uint4(a[0], a[1], a[2], a[3]);
}

// ---- tensor-core issue (one thread) -----------------------------------------

// One-body dominoes into Q0, Q2, Q4 (column 64 e for Q_2e).
//   T1: A = [A1_ts ; A1_(ts+1)] K-major (core strides: K 128, M 1024),
//       B = F_s MN-major (K 1024, N 128);
//   T2: A = [F_ss ; F_(ss+1)] K-major (K 128, M 1024), B = B2_t K-major (K 128, N 1024).
// Digit -1 is the zero matrix stored just before digit 0.  24 chains, 12 of
// T1 then 12 of T2; the first product into each accumulator (the s = 0
// dominoes of T1) overwrites it.
__device__ __forceinline__ void issue_one_body(uint32_t sb, uint32_t tmem) {
  const uint32_t id1 = umma::idesc_bf16(128, 64, false, true), id2 = umma::idesc_bf16(128, 64, false, false);
  for (int s = 0; s < kDig; ++s)
    for (int ts = (s & 1) ? -1 : 0; s + ts <= 4; ts += 2) {
      const uint32_t q = tmem + COL_Q + 32u * (uint32_t)(s + ts);
      for (int kc = 0; kc < 4; ++kc) {
        const uint64_t ad = umma::smem_desc(sb + OFF_T1 + (uint32_t)(ts + 1) * MAT + 256u * kc, 128, 1024);
        const uint64_t bd = umma::smem_desc(sb + OFF_F + (uint32_t)(s + 1) * MAT + 2048u * kc, 1024, 128);
        umma::mma_bf16(q, ad, bd, id1, (s == 0 && kc == 0) ? 0u : 1u);
      }
    }
  for (int t = 0; t < kDig; ++t)
    for (int ss = (t & 1) ? -1 : 0; ss + t <= 4; ss += 2) {
      const uint32_t q = tmem + COL_Q + 32u * (uint32_t)(ss + t);
      for (int kc = 0; kc < 4; ++kc) {
        const uint64_t ad = umma::smem_desc(sb + OFF_F + (uint32_t)(ss + 1) * MAT + 256u * kc, 128, 1024);
        const uint64_t bd = umma::smem_desc(sb + OFF_B2 + (uint32_t)t * MAT + 256u * kc, 128, 1024);
        umma::mma_bf16(q, ad, bd, id2, 1u);
      }
    }
}

// Two-body products of state digit s: A = G_s MN-major (K 2048, M 128), B =
// H_t (or H'_t for d = 5) with both core strides 128; accumulator of diagonal
// d = s + t (d = 4 and 5 share one).  The s = 0 products (t <= 4) open them.
__device__ __forceinline__ void issue_two_body(uint32_t sb, uint32_t tmem, int s) {
  const uint32_t id = umma::idesc_bf16(128, 64, true, false);
  const uint32_t g = sb + OFF_G + (uint32_t)(s & 1) * GMAT;
  for (int t = 0; s + t < kDig; ++t) {
    const int d = s + t;
    const uint32_t acc = tmem + COL_P + 64u * (uint32_t)(d < 4 ? d : 4);
    const uint32_t h = sb + OFF_H + (uint32_t)(d == 5 ? kDig + t : t) * HMAT;
    for (int kc = 0; kc < 4; ++kc) {
      const uint64_t ad = umma::smem_desc(g + 4096u * kc, 2048, 128);
      const uint64_t bd = umma::smem_desc(h + 256u * kc, 128, 128);
      umma::mma_bf16(acc, ad, bd, id, (s == 0 && t <= 4 && kc == 0) ? 0u : 1u);
    }
  }
}

// ---- operand builders (all threads) -------------------------------------------

// Hankel digit matrices of the pair kernel: core matrix q (0..14), row b,
// entry a holds K12(63 - 8 q - a - b), the eight table entries from
// 119 - 8 q - b in reverse order; H_t (family 2) then H'_t (family 3).
__device__ __forceinline__ void build_hankel(unsigned char *sm, const uint32_t *tabs) {
  for (int q = threadIdx.x; q < 2 * kDig * 120; q += THREADS) {
    const int m = q / 120, rem = q - m * 120, core = rem >> 3, b = rem & 7;
    const int sc = m >= kDig, t = m - sc * kDig;
    const uint4 u = window8(tabs + ((2 + sc) * kDig + t) * 64, 119 - 8 * core - b);
    const uint4 v = make_uint4(__byte_perm(u.w, 0, 0x1032), __byte_perm(u.z, 0, 0x1032), __byte_perm(u.y, 0, 0x1032),
                               __byte_perm(u.x, 0, 0x1032));
    *reinterpret_cast<uint4 *>(sm + OFF_H + (uint32_t)m * HMAT + core * 128 + b * 16) = v;
  }
}

// Sheared plane of digit s into buffer s & 1, by threads t0, t0 + nt, ...: G_s[c][k'] = F_s[63 - k'][c - 63 + k'],
// MN-major (core (k' / 8, c / 8), row k' % 8, entries c % 8 .. + 7).  The
// eight entries of a core row are a window of row 63 - k' of F_s starting at
// m0 = c - 63 + k' (zero outside the block), cut from two 16-byte chunks.
__device__ __forceinline__ void build_sheared(unsigned char *sm, int s, int t0, int nt) {
  const unsigned char *P = sm + OFF_F + (uint32_t)(s + 1) * MAT;
  unsigned char *G = sm + OFF_G + (uint32_t)(s & 1) * GMAT;
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  for (int q = t0; q < 1024; q += nt) {
    const int kp = ((q >> 7) << 3) + (q & 7), cg = (q >> 3) & 15;
    const int r = 63 - kp, m0 = 8 * cg - 63 + kp, o = m0 & 7, jc = (m0 - o) >> 3;
    const uint4 lo = (unsigned)jc < 8u ? *reinterpret_cast<const uint4 *>(P + toff(r, 8 * jc, NK)) : z;
    const uint4 hi = (unsigned)(jc + 1) < 8u ? *reinterpret_cast<const uint4 *>(P + toff(r, 8 * jc + 8, NK)) : z;
    *reinterpret_cast<uint4 *>(G + toff(kp, 8 * cg, 2 * NK)) = shift8(lo, hi, o);
  }
}

// ---- the sweep -------------------------------------------------------------------

__device__ __forceinline__ long long ll_of(uint32_t bits) { return (long long)__float2int_rn(__uint_as_float(bits)); }

// Block number b -> (i1, i2): row-major, or with a.sym the upper triangle row by row.
__device__ __forceinline__ void block_xy(const ThetaArgs &a, int b, int &i1, int &i2) {
  const int nx = a.nx;
  if (a.sym) {
    i1 = 0;
    while (b >= nx - i1) {
      b -= nx - i1;
      ++i1;
    }
    i2 = i1 + b;
  } else {
    i1 = b / nx;
    i2 = b - i1 * nx;
  }
}

// What a CTA reads from HBM for a block before its digits are cut, loaded one
// block ahead: the state block (core matrices 4 w .. 4 w + 3 of warp w, thread
// (row lane / 4, columns 2 (lane % 4), + 1), 64-byte row segments) and one
// value of the block's three kernel rows (entry tid of 3 x 127, or zero).
struct Ahead {
  double2 f[4];
  double k;
};

__device__ __forceinline__ void load_ahead(const ThetaArgs &a, int b, Ahead &p) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int i1, i2;
  block_xy(a, b, i1, i2);
  const size_t base = (size_t)(i1 * a.nx + i2) * NK * NK;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int cm = 4 * w + i, r = 8 * (cm >> 3) + (lane >> 2), c = 8 * (cm & 7) + 2 * (lane & 3);
    p.f[i] = *reinterpret_cast<const double2 *>(a.in + base + (size_t)r * NK + c);
  }
  constexpr int W = 2 * NK - 1;
  int dd = i1 - i2;
  dd += (dd < 0) ? a.nx : 0;
  if (tid < 3 * W) {
    const int fam = tid / W, j = tid - fam * W;
    const double *row = fam == 0 ? a.K1 + (size_t)i1 * W : fam == 1 ? a.K2 + (size_t)i2 * W : a.K12 + (size_t)dd * W;
    p.k = row[j];
  } else {
    p.k = 0.0;
  }
}

// Digit tables from the kernel values the threads hold (thread tid < 381:
// entry tid % 127 of family tid / 127): word w of table (fam, t) holds the
// BF16 digits t of K_fam(2 w) and K_fam(2 w + 1) (fam 0: K1(x1), 1: K2(x2),
// 2: K12(x1 - x2), 3: K12 times 2^-8; entry j is the kernel at offset j - 63;
// entry 127 is zero).
__device__ __forceinline__ void build_tables(uint32_t *tabs, double k, int kmax) {
  constexpr int W = 2 * NK - 1;
  uint16_t *t16 = reinterpret_cast<uint16_t *>(tabs);
  const int tid = threadIdx.x;
  if (tid < 4 * kDig) t16[tid * 128 + 127] = 0;
  if (tid < 3 * W) {
    const int fam = tid / W, j = tid - fam * W;
    int dk[kDig];
    slice::digits6(k, kmax, dk);
#pragma unroll
    for (int t = 0; t < kDig; ++t) {
      const uint16_t u = (uint16_t)slice::bf16_int(dk[t]);
      t16[(fam * kDig + t) * 128 + j] = u;
      if (fam == 2) t16[(3 * kDig + t) * 128 + j] = dk[t] ? (uint16_t)(u - 0x0400) : (uint16_t)0;
    }
  }
}

// Toeplitz digit matrices M[r][k] = K(k - r), tiled K-major, of family fam
// (0: A1_t of K1 after the zero matrix at OFF_T1; 1: B2_t of K2 at OFF_B2).
// Thread q writes the 16 bytes at chunk q of its matrix (row r, columns 8 kg .. + 7).
__device__ __forceinline__ void build_toeplitz(unsigned char *sm, const uint32_t *tabs, int fam) {
  for (int q = threadIdx.x; q < kDig * 512; q += THREADS) {
    const int t = q >> 9, ch = q & 511;
    const int r = ((ch >> 6) << 3) + (ch & 7), kg = (ch >> 3) & 7;
    const uint4 v = window8(tabs + (fam * kDig + t) * 64, 8 * kg - r + 63);
    unsigned char *dst = sm + (fam ? OFF_B2 + (uint32_t)t * MAT : OFF_T1 + (uint32_t)(t + 1) * MAT);
    *reinterpret_cast<uint4 *>(dst + toff(r, 8 * kg, NK)) = v;
  }
}

// Persistent CTAs, one per SM: CTA c takes the blocks b in [c P, (c + 1) P)
// (P = ceil(blocks / CTAs)) in order, so that consecutive blocks mostly share
// i1 and the A1 digit matrices are rebuilt only when i1 changes.  Per block:
// digits and operands, the products (two-body digit 0, its completion signal,
// the one-body chains, then digits 1..5 with the sheared planes rebuilt
// alternately), the next block's state and kernel values loaded while the
// last products run, the epilogue.  MODE 0: out = Theta[in].  MODE 1: out =
// h + half_tau Theta[in], with the exact per-X sums of out.  With a.sym the
// blocks are those with i1 <= i2 and each mirror block is written as well.
template <int MODE>
__global__ void __launch_bounds__(THREADS, 1) k_theta_t(ThetaArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  // mbar[0], mbar[1]: sheared buffer 0 / 1 consumed; mbar[2]: every product
  // issued has completed; mbar[3], mbar[4]: sheared buffer 0 / 1 built (one
  // arrival per builder warp)
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + OFF_MISC);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + OFF_MISC + 40);
  int *flag = reinterpret_cast<int *>(sm + OFF_MISC + 44);  // a wait timed out
  int *red = reinterpret_cast<int *>(sm + OFF_MISC + 64);   // 32 ints + 32 long longs
  uint32_t *tabs = reinterpret_cast<uint32_t *>(sm + OFF_G + GMAT);
  long long *I12 = reinterpret_cast<long long *>(sm + OFF_B2);        // epilogue: after the products
  double *C = reinterpret_cast<double *>(sm + OFF_F + MAT);            // mirror staging, after the zero plane
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t sb = umma::smem_u32(sm);
  const int nx = a.nx;
  const int nblocks = a.sym ? nx * (nx + 1) / 2 : nx * nx;
  const int per = (nblocks + (int)gridDim.x - 1) / (int)gridDim.x;
  const int b0 = (int)blockIdx.x * per, b1 = min(nblocks, b0 + per);
  if (b0 >= b1) return;
  const long long limit = a.wait_limit > 0 ? a.wait_limit : WAIT_LIMIT;

  if (w == 0) {
    umma::tmem_alloc(tslot, 512);
    umma::tmem_relinquish();
  }
  if (tid == 0) {
    umma::mbar_init(&mbar[0], 1);
    umma::mbar_init(&mbar[1], 1);
    umma::mbar_init(&mbar[2], 1);
    umma::mbar_init(&mbar[3], BUILDERS / 32);
    umma::mbar_init(&mbar[4], BUILDERS / 32);
    *flag = 0;
  }
  {
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < (int)(MAT / 16); i += THREADS) {
      reinterpret_cast<uint4 *>(sm + OFF_F)[i] = z;
      reinterpret_cast<uint4 *>(sm + OFF_T1)[i] = z;
    }
  }
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tslot;
  const int qd = w & 3, cg = w >> 2, L = 32 * qd + lane;  // epilogue: TMEM lane L, columns 16 cg .. + 15
  const uint32_t tl = tmem + ((uint32_t)(32 * qd) << 16);

  Ahead p;
  load_ahead(a, b0, p);
  int last_i1 = -1, last_kmax = -1;
  for (int b = b0, j = 0; b < b1; ++b, ++j) {
    int i1, i2;
    block_xy(a, b, i1, i2);
    const int X = i1 * nx + i2;
    const size_t base = (size_t)X * NK * NK;
    const bool mirror = a.sym && i1 != i2;
    __syncthreads();  // the previous block's epilogue is done with I12, C and red
    const bool skip = *flag != 0;

    int ef = 0, ek = slice::expo(p.k);
#pragma unroll
    for (int i = 0; i < 4; ++i) ef = max(ef, max(slice::expo(p.f[i].x), slice::expo(p.f[i].y)));
    ef = __reduce_max_sync(0xffffffffu, ef);
    ek = __reduce_max_sync(0xffffffffu, ek);
    if (lane == 0) {
      red[w] = ef;
      red[16 + w] = ek;
    }
    __syncthreads();
    ef = ek = 0;
#pragma unroll
    for (int q = 0; q < THREADS / 32; ++q) {
      ef = max(ef, red[q]);
      ek = max(ek, red[16 + q]);
    }
    const bool bad = ef == 2047 || ek == 2047;
    const int emax = max(ef, 1), kmax = max(ek, 1);

    if (!skip) {
      // digit planes F_s (one core matrix per warp and step) and the digit tables
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int cm = 4 * w + i, r = 8 * (cm >> 3) + (lane >> 2), c = 8 * (cm & 7) + 2 * (lane & 3);
        int dx[kDig], dy[kDig];
        slice::digits6(p.f[i].x, emax, dx);
        slice::digits6(p.f[i].y, emax, dy);
#pragma unroll
        for (int s = 0; s < kDig; ++s)
          *reinterpret_cast<uint32_t *>(sm + OFF_F + (uint32_t)(s + 1) * MAT + toff(r, c, NK)) =
              slice::bf16_int(dx[s]) | (slice::bf16_int(dy[s]) << 16);
      }
      build_tables(tabs, p.k, kmax);
      __syncthreads();
      // A1 depends on i1 and on the kernel rows' shared exponent: rebuilt when either differs
      if (i1 != last_i1 || kmax != last_kmax) build_toeplitz(sm, tabs, 0);
      build_toeplitz(sm, tabs, 1);
      build_hankel(sm, tabs);
      build_sheared(sm, 0, tid, THREADS);
      umma::fence_proxy_async();
      umma::fence_before();
      __syncthreads();
      umma::fence_after();
      if (w == ISSUER) {
        // the issuing warp: digit 0's two-body products, their signal, the
        // one-body chains, then digits 1..5 as their planes are reported built
        if (lane == 0) {
          issue_two_body(sb, tmem, 0);
          umma::mma_commit(&mbar[0]);
          issue_one_body(sb, tmem);
          for (int s = 1; s < kDig; ++s) {
            const int bb = s & 1;
            const uint32_t par = (uint32_t)(bb ? 3 * j + ((s - 1) >> 1) : 2 * j + (s >> 1) - 1) & 1u;
            if (!*flag && !umma::mbar_wait_bounded(&mbar[3 + bb], par, limit)) atomicOr(flag, 1);
            umma::fence_after();
            // a.stall (host-side fault injection): digit 1's products and their
            // completion signal are left out, so the builders' wait at digit 3 runs out
            if (!*flag && !(a.stall && s == 1)) {
              issue_two_body(sb, tmem, s);
              umma::mma_commit(&mbar[bb]);
            }
          }
          umma::mma_commit(&mbar[2]);
        }
        __syncwarp();
      } else {
        // the builder warps: plane s into buffer s & 1 once digit s - 2's
        // products have released it, then one arrival per warp
        for (int s = 1; s < kDig; ++s) {
          const int bb = s & 1;
          const uint32_t par = (uint32_t)(3 * j + ((s - 2) >> 1)) & 1u;
          if (s >= 2 && !*flag && !umma::mbar_wait_bounded(&mbar[bb], par, limit)) atomicOr(flag, 1);
          build_sheared(sm, s, tid, BUILDERS);
          umma::fence_proxy_async();
          __syncwarp();
          if (lane == 0) umma::mbar_arrive(&mbar[3 + bb]);
        }
      }
    }
    last_i1 = i1;
    last_kmax = kmax;

    // the corrector's base for this block and the next block's inputs, read
    // while the last products run
    double hv[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) hv[i] = MODE == 1 ? a.h[base + tid + i * THREADS] : 0.0;
    if (b + 1 < b1) load_ahead(a, b + 1, p);
    if (!skip && !umma::mbar_wait_bounded(&mbar[2], (uint32_t)j & 1u, limit)) atomicOr(flag, 1);
    umma::fence_after();
    __syncthreads();
    const bool tmo = *flag != 0;
    if (tmo && !skip && tid == 0 && a.err) atomicOr(a.err, 1);

    // Epilogue.  Warp w reads TMEM lanes 32 (w % 4) .. + 31, columns 16 (w / 4)
    // .. + 15 of each accumulator.  The integers, in units of 2^4 diagonal-5
    // units (2^-4 of a diagonal-4 unit, as in k_theta_s), go to I12[n1][n2]
    // (int64, row stride 65): the one-body top half (diagonals 0, 2, 4)
    // written, the bottom half (1, 3, 5) added, then the two-body part of lane
    // c added at (n1, c - n1).
    if (!tmo) {
      {
        long long acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = 0;
        const bool top = qd < 2;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          uint32_t r[16];
          umma::tmem_ld16(tl + COL_Q + 64u * e + 16u * cg, r);
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const long long v = ll_of(r[q]);
            if (top)
              acc[q] += v * (1ll << (8 * (4 - 2 * e) + 4));
            else if (e < 2)
              acc[q] += v * (1ll << (8 * (3 - 2 * e) + 4));
            else
              acc[q] += (v + 8) >> 4;  // diagonal 5, rounded to the unit
          }
        }
        const int n1 = L & 63;
        if (top) {
#pragma unroll
          for (int q = 0; q < 16; ++q) I12[n1 * IST + 16 * cg + q] = acc[q];
        }
        __syncthreads();
        if (!top) {
#pragma unroll
          for (int q = 0; q < 16; ++q) I12[n1 * IST + 16 * cg + q] += acc[q];
        }
        __syncthreads();
      }
      {
        long long acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = 0;
#pragma unroll
        for (int d = 0; d < 5; ++d) {
          uint32_t r[16];
          umma::tmem_ld16(tl + COL_P + 64u * d + 16u * cg, r);
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            if (d < 4)
              acc[q] += ll_of(r[q]) * (1ll << (8 * (4 - d) + 4));
            else
              acc[q] += __float2ll_rn(__uint_as_float(r[q]) * 16.f);
          }
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int n1 = 16 * cg + q, n2 = L - n1;
          if ((unsigned)n2 < (unsigned)NK) I12[n1 * IST + n2] += acc[q];
        }
      }
      umma::fence_before();
      __syncthreads();
    }

    // FP64 outputs (row-major, coalesced), the corrector combination, the
    // exact per-X sum and the mirror block.
    const int xs = emax + kmax - 2096;  // one unit of I12 is 2^xs
    const bool nan_out = bad || tmo;
    double v[PER];
    int em = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int e = tid + i * THREADS, n1 = e >> 6, n2 = e & 63;
      const double t =
          nan_out ? __longlong_as_double(0x7ff8000000000000ll) : ll_to_double_scaled(I12[n1 * IST + n2], xs);
      if (mirror) C[n1 * IST + n2] = t;
      v[i] = MODE == 0 ? t : fma(a.half_tau, t, hv[i]);
      a.out[base + e] = v[i];
      em = max(em, slice::expo(v[i]));
    }
    if (MODE == 1 && a.xsum) slice::held_exact_sum<PER>(v, em, a.xsum + X, red);
    if (mirror) {
      __syncthreads();
      slice::mirror_block<NK, THREADS, MODE>(a, C, i2 * nx + i1, red);
    }
  }
  umma::fence_before();
  __syncthreads();
  if (w == 0) umma::tmem_dealloc(tmem, 512);
}

}  // namespace

bool theta_t_supported(int nk, const ThetaArgs &a) { return nk == NK && a.pair == nullptr; }

cudaError_t prepare_kernels_f64t() {
  cudaError_t e = cudaFuncSetAttribute(k_theta_t<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_theta_t<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
}

// The tcgen05 sweep (mode 0 / 1 as launch_theta_f64s) for N_k = 64 without a
// learned pair term.
cudaError_t launch_theta_f64t(int mode, const ThetaArgs &a, cudaStream_t s) {
  const int nblocks = a.sym ? a.nx * (a.nx + 1) / 2 : a.nx * a.nx;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int grid = nblocks < nsm ? nblocks : nsm;
  if (mode == 0)
    k_theta_t<0><<<grid, THREADS, SMEM, s>>>(a);
  else
    k_theta_t<1><<<grid, THREADS, SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace w2
