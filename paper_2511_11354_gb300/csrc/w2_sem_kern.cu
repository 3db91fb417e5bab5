// Kernels of the non-periodic path: static tables of the spectral-element
// operators (Sec. 3.2), densities and potentials, the D_V weighting of the
// two-body chain (Sec. 3.2.2), the natural-boundary spline shift (Sec. 4.1),
// the Lawson combinations and the observables.
#include <math.h>

#include "w2_df.cuh"
#include "w2_internal.cuh"
#include "w2_sem.cuh"

namespace w2sem {
namespace {

constexpr double kPi = 3.14159265358979323846;

// int_{-1}^{1} T_k T_l for k + l even (0 otherwise).
__device__ __forceinline__ double cheb_gram(int k, int l) {
  const double a = (double)(k + l), b = (double)(k - l);
  return 1.0 / (1.0 - a * a) + 1.0 / (1.0 - b * b);
}

// O_l(z) = int_{-1}^{1} e^{i z eta} T_l(eta) deta for l < Q at z = width d dx / hbar,
// d = 0 .. nx-1, by the Jacobi-Anger expansion
//   e^{i z eta} = J_0(z) + 2 sum_{k>=1} i^k J_k(z) T_k(eta)
// with the Bessel values J_k(z) from Miller's backward recurrence
// J_{k-1} = (2k/z) J_k - J_{k+1}, normalised by J_0 + 2 sum J_{2k} = 1.  The
// sums over k are accumulated during the recurrence (unnormalised) and
// divided by the normalisation at the end.  O_l is real for even l and
// imaginary for odd l.
__global__ void k_sem_osc(SemTabArgs a) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= a.nx) return;
  const int Q = a.Q;
  double S[32];
#pragma unroll
  for (int l = 0; l < 32; ++l) S[l] = 0.0;
  double norm = 1.0;
  const double z = a.width * (double)d * a.dx / a.hbar;
  if (d == 0) {
    for (int l = 0; l < Q; l += 2) S[l] = cheb_gram(0, l);  // J_k(0) = [k == 0]
  } else {
    int kst = (int)(z + 20.0 * cbrt(z + 1.0) + 40.0);
    kst += kst & 1;
    double jp1 = 0.0, jk = 1e-280;  // j_{k+1}, j_k at k = kst
    norm = 0.0;
    for (int k = kst; k >= 0; --k) {
      // fold j_k into the sums
      const double ck = (k == 0) ? 1.0 : 2.0;
      if ((k & 1) == 0) {
        norm += ck * jk;
        const double sg = ((k >> 1) & 1) ? -1.0 : 1.0;
        for (int l = 0; l < Q; l += 2) S[l] = fma(ck * sg * cheb_gram(k, l), jk, S[l]);
      } else {
        const double sg = (((k - 1) >> 1) & 1) ? -1.0 : 1.0;
        for (int l = 1; l < Q; l += 2) S[l] = fma(2.0 * sg * cheb_gram(k, l), jk, S[l]);
      }
      if (k == 0) break;
      const double jm1 = (2.0 * k / z) * jk - jp1;
      jp1 = jk;
      jk = jm1;
      if (fabs(jk) > 1e250) {  // rescale everything accumulated so far
        jk *= 1e-250; jp1 *= 1e-250; norm *= 1e-250;
        for (int l = 0; l < Q; ++l) S[l] *= 1e-250;
      }
    }
  }
  for (int l = 0; l < Q; ++l) {
    const double v = S[l] / norm;
    a.osc[(d * Q + l) * 2 + 0] = (l % 2 == 0) ? v : 0.0;
    a.osc[(d * Q + l) * 2 + 1] = (l % 2 == 0) ? 0.0 : v;
  }
}

// O_l(width y / hbar) for y = d dx with d of either sign (O_l(-z) = conj O_l(z)).
__device__ __forceinline__ double2 osc_at(const double *osc, int Q, int d, int l) {
  const int ad = d < 0 ? -d : d;
  double2 o = make_double2(osc[(ad * Q + l) * 2], osc[(ad * Q + l) * 2 + 1]);
  if (d < 0) o.y = -o.y;
  return o;
}

// One-body table: psi[d + nx - 1][i][j] = (dx / (pi hbar^2)) width
//   sum_l C[l][q] Im[e^{-2i (p_i - c_s) y_d / hbar} O_l(width y_d / hbar)],
// j = s Q + q, y_d = d dx, so that the operator's matrix at x_m is
// G(x_m) = sum_n U(x_n) psi[n - m].
__global__ void k_sem_psi(SemTabArgs a) {
  const long long np = a.np, total = (long long)(2 * a.nx - 1) * np * np;
  const double pref = a.dx * a.width / (kPi * a.hbar * a.hbar);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e % np), i = (int)((e / np) % np), dd = (int)(e / (np * np));
    const int d = dd - (a.nx - 1), s = j / a.Q, q = j % a.Q;
    const double y = (double)d * a.dx;
    double sn, cs;
    sincos(-2.0 * (a.p[i] - a.centre[s]) * y / a.hbar, &sn, &cs);
    double acc = 0.0;
    for (int l = 0; l < a.Q; ++l) {
      const double2 o = osc_at(a.osc, a.Q, d, l);
      acc = fma(a.cheb[l * a.Q + q], cs * o.y + sn * o.x, acc);  // Im[(cs + i sn)(o.x + i o.y)]
    }
    a.psi[e] = pref * acc;
  }
}

// Two-body transform rows Phi_j(y_n) = sum_l C[l][q] (width/2) e^{2i c_s y_n / hbar}
// O_l(width y_n / hbar), n = -h .. h (the exact transform of a nodal vector's
// cell expansions at frequency y_n).
__global__ void k_sem_phi(SemTabArgs a) {
  const int Ny = 2 * a.h + 1, total = Ny * a.np;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int j = e % a.np, n = e / a.np - a.h, s = j / a.Q, q = j % a.Q;
    const double y = (double)n * a.dx;
    double sn, cs;
    sincos(2.0 * a.centre[s] * y / a.hbar, &sn, &cs);
    double re = 0.0, im = 0.0;
    for (int l = 0; l < a.Q; ++l) {
      const double2 o = osc_at(a.osc, a.Q, n, l);
      const double c = a.cheb[l * a.Q + q];
      re = fma(c, cs * o.x - sn * o.y, re);
      im = fma(c, cs * o.y + sn * o.x, im);
    }
    a.phir[e] = 0.5 * a.width * re;
    a.phii[e] = 0.5 * a.width * im;
  }
}

// Block operands of the complex products (see launch_sem_tables).
__global__ void k_sem_assemble(SemTabArgs a) {
  const int np = a.np, h = a.h, Ny = 2 * h + 1, Nyh = h + 1;
  const int nph = 2 * Nyh * 2 * np, neh = 2 * np * 2 * Nyh, nee = np * 2 * Ny;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nph + neh + nee; e += gridDim.x * blockDim.x) {
    if (e < nph) {  // ph[r][c] = [[Phr_h, -Phi_h], [Phi_h, Phr_h]], rows y1 = 0 .. h
      const int r = e / (2 * np), c = e % (2 * np);
      const int br = r / Nyh, rr = r % Nyh, bc = c / np, cc = c % np;
      const int src = (h + rr) * np + cc;
      double v;
      if (br == bc) v = a.phir[src]; else v = (br == 0) ? -a.phii[src] : a.phii[src];
      a.ph[e] = v;
    } else if (e < nph + neh) {  // eh[b][i][c]: b = 0: [Er_h | -Ei_h], b = 1: [Ei_h | Er_h]
      const int f = e - nph;
      const int b = f / (np * 2 * Nyh), i = (f / (2 * Nyh)) % np, c = f % (2 * Nyh);
      const int half = c / Nyh, n = c % Nyh;  // y1 = n dx, n = 0 .. h
      double sn, cs;
      sincos(-2.0 * a.p[i] * ((double)n * a.dx) / a.hbar, &sn, &cs);  // E = cs + i sn
      double v;
      if (b == 0) v = (half == 0) ? cs : -sn; else v = (half == 0) ? sn : cs;
      a.eh[f] = v;
    } else {  // eier[i][c] = [Ei | Er] over y2 = (n - h) dx
      const int f = e - nph - neh;
      const int i = f / (2 * Ny), c = f % (2 * Ny);
      const int n = (c % Ny) - h;
      double sn, cs;
      sincos(-2.0 * a.p[i] * ((double)n * a.dx) / a.hbar, &sn, &cs);
      a.eier[f] = (c < Ny) ? sn : cs;
    }
  }
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  __syncthreads();
  if (ln == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; ++i) s += red[i];
  return s;  // valid in thread 0
}

// xs[X] = sum_j1 w_j1 sum_j2 w_j2 f[X][j1][j2]: thread t keeps the column
// j2 = t % np and walks the rows j1 = t / np + R k (R = 256 / np rows in
// flight, np <= 256), one FP64 multiply-add per element; w_j2 is applied once.
__global__ void __launch_bounds__(256) k_sem_xsum(int np, const double *__restrict__ f, const double *__restrict__ w,
                                                  double *xs) {
  __shared__ double red[8];
  const long long X = blockIdx.x;
  const double *fx = f + X * np * np;
  const int R = 256 / np, j2 = threadIdx.x % np, r0 = threadIdx.x / np;
  double acc = 0.0;
  if (r0 < R)
    for (int j1 = r0; j1 < np; j1 += R) acc = fma(w[j1], fx[j1 * np + j2], acc);
  const double s = block_sum<256>(acc * w[j2], red);
  if (threadIdx.x == 0) xs[X] = s;
}

__global__ void k_sem_dens(int nx, double dx, const double *xs, double *n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nx) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < nx; ++k) {
    a += xs[(long long)i * nx + k];
    b += xs[(long long)k * nx + i];
  }
  n[i] = dx * a;
  n[nx + i] = dx * b;
}

__device__ __forceinline__ double phi_xc(int kind, double n) {
  if (kind == 1) return n;
  if (kind == 2) {  // Hedin-Lundqvist exchange-correlation potential, atomic units
    const double c = cbrt(n > 0.0 ? n : 0.0);
    return 0.985 * c + 0.985 * 0.034 * log1p(18.37 * c);
  }
  return 0.0;
}

// One block per particle: U, then its Toeplitz rows.
__global__ void __launch_bounds__(256) k_sem_potential(SemPotArgs a) {
  extern __shared__ double Us[];
  const int k = blockIdx.x, nx = a.nx, W0 = 2 * (nx - 1);
  const double *n = a.n + k * nx;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    double u = a.vext[i];
    if (a.c_h != 0.0) {
      double vh = 0.0;
      for (int q = 0; q < nx; ++q) vh = fma(a.wgrid[i - q + W0], n[q], vh);
      u += a.c_h * a.dx * vh;
    }
    if (a.c_xc != 0.0 && a.xc_kind) u += a.c_xc * phi_xc(a.xc_kind, n[i]);
    Us[i] = u;
    a.U[k * nx + i] = u;
  }
  __syncthreads();
  const int nd = 2 * nx - 1;
  for (long long e = threadIdx.x; e < (long long)nx * nd; e += blockDim.x) {
    const int m = (int)(e / nd), dd = (int)(e % nd);
    const int src = m + dd - (nx - 1);
    a.ut[((long long)k * nx + m) * nd + dd] = (src >= 0 && src < nx) ? Us[src] : 0.0;
  }
}

// Two-body weighting on a chunk of X: A_X holds [Ar; Ai] (2 Nyh x Ny) with
// rows y1 = r dx (r = 0 .. h) and columns y2 = (c - h) dx.
__global__ void k_sem_dmul(int nx, int h, int x0, int nb, const double *__restrict__ wgrid, double *A) {
  const int Ny = 2 * h + 1, Nyh = h + 1, W0 = 2 * (nx - 1);
  const long long per = (long long)2 * Nyh * Ny, total = per * nb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int bb = (int)(e / per);
    const int r = (int)((e % per) / Ny) % Nyh, c = (int)(e % Ny);
    const int X = x0 + bb, rho = X / nx - X % nx;
    const int u = r - (c - h);
    const double D = wgrid[rho + u + W0] - wgrid[rho - u + W0];
    A[e] *= (r == 0 ? 1.0 : 2.0) * D;
  }
}

// Natural-boundary cubic spline shift of C adjacent lines by 4 C threads:
// all threads load the lines into shared memory (coalesced rows of C
// values), one thread per line solves the interior (1,4,1)/6 system with
// eta_0 = f_0, eta_N = f_N by the Thomas recursion in place, then all threads
// evaluate the four B-spline terms at the feet and store; the ghosts are
// eta_{-1} = 2 eta_0 - eta_1, eta_{N+1} = 2 eta_N - eta_{N-1}, zero beyond.
template <int AXIS>
__global__ void __launch_bounds__(256) k_sem_adv(SemAdvArgs a) {
  extern __shared__ double sl[];
  const int nx = a.nx, np = a.np, C = a.C, N = nx - 1, T = 4 * C;
  const int tid = threadIdx.x;
  const int nchunk = (np + C - 1) / C;
  const int chunk = blockIdx.x % nchunk, j1 = (blockIdx.x / nchunk) % np, o = blockIdx.x / (nchunk * np);
  const int c0 = chunk * C, width = np - c0 < C ? np - c0 : C;
  const long long np2 = (long long)np * np;
  long long base, stride;
  if (AXIS == 0) { base = ((long long)o * np + j1) * np; stride = (long long)nx * np2; }  // o = i2
  else { base = (long long)o * nx * np2 + (long long)j1 * np; stride = np2; }          // o = i1
  double *ghost = sl + (size_t)nx * C;  // [2][C]: eta_{-1}, eta_{N+1}
  for (int e = tid; e < nx * C; e += T) {
    const int i = e / C, c = e % C;
    if (c < width) sl[e] = a.in[base + i * stride + c0 + c];
  }
  __syncthreads();
  if (tid < width) {
    const int c = tid;
    // forward: d'_i = (r_i - d'_{i-1}) c'_i, r_i = 6 f_i - [i==1] f_0 - [i==N-1] f_N
    double dprev = 0.0;
    const double f0 = sl[c], fN = sl[N * C + c];
    for (int i = 1; i <= N - 1; ++i) {
      double r = 6.0 * sl[i * C + c];
      if (i == 1) r -= f0;
      if (i == N - 1) r -= fN;
      dprev = (r - dprev) * a.cp[i];
      sl[i * C + c] = dprev;
    }
    // backward: eta_{N-1} = d'_{N-1}, eta_i = d'_i - c'_i eta_{i+1}
    double enext = sl[(N - 1) * C + c];
    for (int i = N - 2; i >= 1; --i) {
      enext = sl[i * C + c] - a.cp[i] * enext;
      sl[i * C + c] = enext;
    }
    ghost[c] = 2.0 * sl[c] - sl[C + c];
    ghost[C + c] = 2.0 * sl[N * C + c] - sl[(N - 1) * C + c];
  }
  __syncthreads();
  for (int e = tid; e < nx * C; e += T) {
    const int i = e / C, c = e % C;
    if (c >= width) continue;
    const int jm = (AXIS == 0) ? j1 : c0 + c;
    const int nu0 = i + a.k0[jm] - 1;
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int nu = nu0 + q;
      double eta = 0.0;
      if (nu >= 0 && nu <= N) eta = sl[nu * C + c];
      else if (nu == -1) eta = ghost[c];
      else if (nu == N + 1) eta = ghost[C + c];
      v = fma(a.wts[jm * 4 + q], eta, v);
    }
    a.out[base + i * stride + c0 + c] = v;
  }
}

// Double-float arithmetic on (hi, lo) FP32 pairs (Dekker / Knuth error-free
// transformations, w2_df.cuh), about 2^-47 relative per operation.
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float s, e;
  w2::two_sum(a.x, b.x, s, e);
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  float h, l;
  w2::fast_two_sum(s, e, h, l);
  return make_float2(h, l);
}
__device__ __forceinline__ float2 df_mulv(float2 a, float2 b) {
  float p, e;
  w2::df_mul(a.x, a.y, b.x, b.y, p, e);
  float h, l;
  w2::fast_two_sum(p, e, h, l);
  return make_float2(h, l);
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// The shift of k_sem_adv with the line values held as double-float pairs in
// shared memory: the FP64 pipe of this GPU runs at about 1/64 of the FP32
// rate, and the recursion plus the evaluation cost about seven FP64
// operations per value.  The solve runs on h = eta / 6 (the factor 6 of the
// (1, 4, 1) system moves into the B-spline weights, which the caller passes
// as 6 w): g_i = (f_i - [i==1] f_0/6 - [i==N-1] f_N/6 - g_{i-1}) c'_i,
// h_i = g_i - c'_i h_{i+1}, h_0 = f_0 / 6, h_N = f_N / 6.  Each column keeps
// three rows below and above the line (zero, zero, ghost | ghost, zero,
// zero), so a foot index is clamped into [-3, N + 3] instead of branched on;
// thread t works on column t % C and rows t / C + 4 k.
constexpr int kStart = 28, kPieceMin = 48;

// 8-byte asynchronous copy global -> shared; the wait covers the calling
// thread's own copies.
__device__ __forceinline__ void sem_cp_async8(void *dst, const void *src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void sem_cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <int AXIS>
__global__ void __launch_bounds__(256) k_sem_adv_df(SemAdvArgs a) {
  extern __shared__ float2 sf[];
  const int nx = a.nx, np = a.np, C = a.C, N = nx - 1;
  const int tid = threadIdx.x, c = tid % C, r0 = tid / C;  // 4 rows in flight per column
  const int nchunk = (np + C - 1) / C;
  const int chunk = blockIdx.x % nchunk, j1 = (blockIdx.x / nchunk) % np, o = blockIdx.x / (nchunk * np);
  const int c0 = chunk * C, width = np - c0 < C ? np - c0 : C;
  const long long np2 = (long long)np * np;
  long long base, stride;
  if (AXIS == 0) { base = ((long long)o * np + j1) * np; stride = (long long)nx * np2; }  // o = i2
  else { base = (long long)o * nx * np2 + (long long)j1 * np; stride = np2; }          // o = i1
  float2 *col = sf + 3 * C + c;  // row nu of this column at col[nu * C], nu in [-3, N + 3]
  const bool live = c < width;
  const double *src = a.in + base + c0 + c;
  // stage the column's rows with 8-byte asynchronous copies (all in flight at
  // once), then split each FP64 value into a pair in place (same 8 bytes)
  if (live) {
    for (int i = r0; i < nx; i += 4) sem_cp_async8(col + i * C, src + i * stride);
    sem_cp_async_wait_all();
    for (int i = r0; i < nx; i += 4) col[i * C] = w2::df_split(*reinterpret_cast<const double *>(col + i * C));
  }
  if (r0 == 0) {
    const float2 z = make_float2(0.f, 0.f);
    col[-3 * C] = z; col[-2 * C] = z; col[(N + 2) * C] = z; col[(N + 3) * C] = z;
  }
  __syncthreads();
  const float2 sixth = make_float2(0.1666666716337204f, -4.967053879312289e-09f), two = make_float2(2.f, 0.f);
  // P threads per column (P = 1 .. 4), one piece [lo, hi) of the interior
  // rows each; a piece holds at least kPieceMin rows.  Where c'_i has settled
  // to c* = 2 - sqrt(3), the recursions unroll into geometric sums, so piece
  // p > 0 starts its forward pass from
  // g_{lo-1} = sum_{k<kStart} (-1)^k c*^(k+1) f_{lo-1-k} and piece p < P - 1
  // its backward pass from h_hi = sum_k (-c*)^k g_{hi+k} (kStart = 28 terms:
  // the tail is below 2^-53 of the scale).  The start values are read before
  // any piece overwrites its rows.  With P = 1 this is the plain two-pass
  // solve.
  const int n = N - 1;
  const int P = max(1, min(4, n / kPieceMin));
  const bool work = live && r0 < P;
  const int lo = 1 + (r0 * n) / P, hi = 1 + ((r0 + 1) * n) / P;
  float2 dprev = make_float2(0.f, 0.f);
  if (work && r0 > 0)
    for (int k = 0; k < kStart; ++k) dprev = df_add(dprev, df_mulv(a.fwdc[k], col[(lo - 1 - k) * C]));
  const float2 f0 = df_mulv(col[0], sixth), fN = df_mulv(col[N * C], sixth);
  __syncthreads();
  if (work) {  // g_i = (r_i - g_{i-1}) c'_i, r_i = f_i - [i==1] f_0/6 - [i==N-1] f_N/6
    for (int i = lo; i < hi; ++i) {
      float2 r = col[i * C];
      if (i == 1) r = df_add(r, df_neg(f0));
      if (i == N - 1) r = df_add(r, df_neg(fN));
      dprev = df_mulv(df_add(r, df_neg(dprev)), a.cpdf[i]);
      col[i * C] = dprev;
    }
  }
  __syncthreads();
  float2 enext = make_float2(0.f, 0.f);
  if (work && r0 < P - 1)
    for (int k = 0; k < kStart && hi + k <= N - 1; ++k) enext = df_add(enext, df_mulv(a.bwdc[k], col[(hi + k) * C]));
  __syncthreads();
  if (work) {  // h_{N-1} = g_{N-1}, h_i = g_i - c'_i h_{i+1}
    int i = hi - 1;
    if (r0 == P - 1) {
      enext = col[i * C];
      --i;
    }
    for (; i >= lo; --i) {
      enext = df_add(col[i * C], df_neg(df_mulv(a.cpdf[i], enext)));
      col[i * C] = enext;
    }
  }
  __syncthreads();
  if (live && r0 == 0) {
    col[0] = f0;
    col[N * C] = fN;
    col[-C] = df_add(df_mulv(f0, two), df_neg(col[C]));
    col[(N + 1) * C] = df_add(df_mulv(fN, two), df_neg(col[(N - 1) * C]));
  }
  __syncthreads();
  if (!live) return;
  const int jm = (AXIS == 0) ? j1 : c0 + c;
  const int k0 = a.k0[jm];
  const float2 w0 = a.wtsdf[jm * 4], w1 = a.wtsdf[jm * 4 + 1], w2 = a.wtsdf[jm * 4 + 2], w3 = a.wtsdf[jm * 4 + 3];
  double *dst = a.out + base + c0 + c;
  for (int i = r0; i < nx; i += 4) {
    const int nu = i + k0 - 1;
    const float2 e0 = col[min(max(nu, -3), N + 3) * C], e1 = col[min(max(nu + 1, -3), N + 3) * C];
    const float2 e2 = col[min(max(nu + 2, -3), N + 3) * C], e3 = col[min(max(nu + 3, -3), N + 3) * C];
    // sum_q (6 w_q) h_q: exact products of the high parts plus cross terms,
    // accumulated without normalising in between (one normalisation at the end)
    float sh, se, ph, pe, h, l;
    w2::df_mul(w0.x, w0.y, e0.x, e0.y, sh, se);
    w2::df_mul(w1.x, w1.y, e1.x, e1.y, ph, pe);
    w2::df_acc(sh, se, ph, pe);
    w2::df_mul(w2.x, w2.y, e2.x, e2.y, ph, pe);
    w2::df_acc(sh, se, ph, pe);
    w2::df_mul(w3.x, w3.y, e3.x, e3.y, ph, pe);
    w2::df_acc(sh, se, ph, pe);
    w2::fast_two_sum(sh, se, h, l);
    dst[i * stride] = w2::df_join(h, l);
  }
}

__global__ void k_sem_erm(int np, int Ny, const double *eier, double *erm) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)np * 2 * Ny;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / (2 * Ny);
    const int c = (int)(e % (2 * Ny));
    erm[e] = c < Ny ? eier[i * 2 * Ny + Ny + c] : -eier[i * 2 * Ny + c - Ny];
  }
}

__global__ void k_sem_negcols(int rows, int cols, int c0, const double *in, double *out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)rows * cols;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (e % cols) < c0 ? in[e] : -in[e];
}

__global__ void k_sem_scale(long long n, double a, const double *__restrict__ in, double *out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = a * in[e];
}

__global__ void k_sem_axpy(long long n, const double *__restrict__ x, double a, const double *__restrict__ y,
                           const double *__restrict__ y2, double *out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double t = y2 ? y[e] + y2[e] : y[e];
    out[e] = fma(a, t, x[e]);
  }
}

// Per-X partials xp = [sum_j1 w r0, sum_j1 w (p^2 r0 + r2) / (2m), sum_j1 w r3, 0,
// r0(j1) for j1 < np] with r0(j1) = sum_j2 w f, r2 = sum_j2 w p^2 f,
// r3 = sum_j2 w f^2.  One block per X, one thread per row j1 (w and w p^2
// from shared tables: four FP64 operations per element, no per-row
// reductions).
__global__ void __launch_bounds__(256) k_sem_obs_x(SemObsArgs a) {
  __shared__ double red[3][8];
  extern __shared__ double sm[];  // w [np], w p^2 [np]
  const long long X = blockIdx.x;
  const int np = a.np, nt = blockDim.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double *ws = sm, *wp2 = sm + np;
  for (int j = threadIdx.x; j < np; j += nt) {
    ws[j] = a.w[j];
    wp2[j] = a.w[j] * a.p[j] * a.p[j];
  }
  __syncthreads();
  const double *fx = a.f + X * np * np;
  double *xp = a.xpart + X * (4 + np);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int j1 = threadIdx.x; j1 < np; j1 += nt) {
    const double *row = fx + (long long)j1 * np;
    double r0 = 0.0, r2 = 0.0, r3 = 0.0;
    int j2 = 0;
    if ((np & 1) == 0) {
      for (; j2 < np; j2 += 2) {
        const double2 v = *reinterpret_cast<const double2 *>(row + j2);
        const double w0 = ws[j2] * v.x, w1 = ws[j2 + 1] * v.y;
        r0 += w0;
        r0 += w1;
        r2 = fma(wp2[j2], v.x, r2);
        r2 = fma(wp2[j2 + 1], v.y, r2);
        r3 = fma(w0, v.x, r3);
        r3 = fma(w1, v.y, r3);
      }
    }
    for (; j2 < np; ++j2) {
      const double v = row[j2], wv = ws[j2] * v;
      r0 += wv;
      r2 = fma(wp2[j2], v, r2);
      r3 = fma(wv, v, r3);
    }
    xp[4 + j1] = r0;
    s0 = fma(ws[j1], r0, s0);
    s1 = fma(wp2[j1], r0, fma(ws[j1], r2, s1));
    s2 = fma(ws[j1], r3, s2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) {
    red[0][wid] = s0;
    red[1][wid] = s1;
    red[2][wid] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    for (int q = 0; q < nt / 32; ++q) {
      t0 += red[0][q];
      t1 += red[1][q];
      t2 += red[2][q];
    }
    xp[0] = t0;
    xp[1] = t1 / (2.0 * a.mass);
    xp[2] = t2;
    xp[3] = 0.0;
  }
}

// One block per x1 = x_i (256 threads): mid[i] = {sum_i2 xp[0], sum_i2 (xp[1] +
// xp[0] (V(x1) + V(x2) + gamma W(x1 - x2))), sum_i2 xp[2],
// sum_j1 w_j1 f1(x_i, p_j1)^2 with f1 = dx sum_i2 r0, and sum_i1 xp[0] at
// x2 = x_i}: the densities are dx times the first and the last.
__global__ void __launch_bounds__(256) k_sem_obs_mid(SemObsArgs a, double *mid) {
  __shared__ double red[8];
  const int nx = a.nx, np = a.np, W0 = 2 * (nx - 1), i1 = blockIdx.x;
  const double *xrow = a.xpart + (long long)i1 * nx * (4 + np);
  double m = 0.0, e = 0.0, l2 = 0.0, pu = 0.0, nc = 0.0;
  for (int i2 = threadIdx.x; i2 < nx; i2 += 256) {
    const double *xp = xrow + (long long)i2 * (4 + np);
    m += xp[0];
    l2 += xp[2];
    e += xp[1] + xp[0] * (a.vext[i1] + a.vext[i2] + a.gamma * a.wgrid[i1 - i2 + W0]);
    nc += a.xpart[((long long)i2 * nx + i1) * (4 + np)];
  }
  for (int b = 0; b < np; b += 64) {  // a quad of lanes per momentum row j1
    const int j1 = b + (threadIdx.x >> 2);
    double f1 = w2::quad_sum(j1 < np, nx, [&](int i2) { return xrow[(long long)i2 * (4 + np) + 4 + j1]; });
    if ((threadIdx.x & 3) == 0 && j1 < np) {
      f1 *= a.dx;
      pu = fma(a.w[j1] * f1, f1, pu);
    }
  }
  m = block_sum<256>(m, red);
  e = block_sum<256>(e, red);
  l2 = block_sum<256>(l2, red);
  pu = block_sum<256>(pu, red);
  nc = block_sum<256>(nc, red);
  if (threadIdx.x == 0) {
    mid[5 * i1] = m;
    mid[5 * i1 + 1] = e;
    mid[5 * i1 + 2] = l2;
    mid[5 * i1 + 3] = pu;
    mid[5 * i1 + 4] = nc;
  }
}

// One block: out = {mass, energy, purity, entropy_lin, l2norm, 0, 0, 0, n1[nx]}.
__global__ void __launch_bounds__(1024) k_sem_obs_fin(SemObsArgs a, const double *mid) {
  __shared__ double red[32];
  extern __shared__ double dens[];  // n1 [nx], n2 [nx]
  const int nx = a.nx, W0 = 2 * (nx - 1);
  double m = 0.0, e = 0.0, l2 = 0.0, pu = 0.0;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    m += mid[5 * i];
    e += mid[5 * i + 1];
    l2 += mid[5 * i + 2];
    pu += mid[5 * i + 3];
    dens[i] = a.dx * mid[5 * i];
    dens[nx + i] = a.dx * mid[5 * i + 4];
  }
  m = block_sum<1024>(m, red);
  e = block_sum<1024>(e, red);
  l2 = block_sum<1024>(l2, red);
  pu = block_sum<1024>(pu, red);  // its barriers also publish dens
  // Hartree energy (c_h / 2) dx sum_i n_k(x_i) V_H[n_k](x_i), both particles
  double eh = 0.0;
  for (int t = threadIdx.x; t < 2 * nx; t += blockDim.x) {
    const int k = t / nx, i = t % nx;
    const double *n = dens + k * nx;
    double vh = 0.0;
#pragma unroll 8
    for (int q = 0; q < nx; ++q) vh = fma(a.wgrid[i - q + W0], n[q], vh);
    eh += n[i] * a.dx * (a.dx * vh);  // n(x_i) dx V_H[n](x_i)
  }
  eh = block_sum<1024>(eh, red);
  if (threadIdx.x == 0) {
    const double dx2 = a.dx * a.dx;
    a.out[0] = dx2 * m;
    a.out[1] = dx2 * e + 0.5 * a.c_h * eh;
    a.out[2] = 2.0 * kPi * a.hbar * a.dx * pu;
    a.out[3] = 1.0 - a.out[2];
    a.out[4] = sqrt(dx2 * l2);
    a.out[5] = a.out[6] = a.out[7] = 0.0;
  }
  for (int i = threadIdx.x; i < nx; i += blockDim.x) a.out[8 + i] = dens[i];
}

// Occupation numbers: the reduced Wigner function (one block per (x, p)),
// its half points by the natural spline, and the density matrix.
__global__ void __launch_bounds__(128) k_sem_f1(int nx, int np, double dx, const double *__restrict__ f,
                                                const double *__restrict__ w, double *f1) {
  __shared__ double red[4];
  const int i = blockIdx.x / np, j = blockIdx.x % np;
  double acc = 0.0;
  for (int e = threadIdx.x; e < nx * np; e += 128) {
    const int i2 = e / np, j2 = e % np;
    acc = fma(w[j2], f[(((long long)i * nx + i2) * np + j) * np + j2], acc);
  }
  const double v = block_sum<128>(acc, red);
  if (threadIdx.x == 0) f1[(long long)i * np + j] = dx * v;
}

__global__ void k_sem_halfgrid(int nx, int np, const double *f1, const double *cp, double *eta, double *g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  const int N = nx - 1;
  double *E = eta + j;  // eta_nu at E[(nu + 1) * np], nu = -1 .. N + 1
  auto F = [&](int i) { return f1[(long long)i * np + j]; };
  E[np] = F(0);
  E[(N + 1) * np] = F(N);
  double dprev = 0.0;
  for (int i = 1; i <= N - 1; ++i) {
    double r = 6.0 * F(i);
    if (i == 1) r -= F(0);
    if (i == N - 1) r -= F(N);
    dprev = (r - dprev) * cp[i];
    E[(i + 1) * np] = dprev;
  }
  double enext = dprev;
  for (int i = N - 2; i >= 1; --i) {
    enext = E[(i + 1) * np] - cp[i] * enext;
    E[(i + 1) * np] = enext;
  }
  E[0] = 2.0 * E[np] - E[2 * np];
  E[(N + 2) * np] = 2.0 * E[(N + 1) * np] - E[N * np];
  for (int i = 0; i < nx; ++i) g[(long long)(2 * i) * np + j] = F(i);
  // B-spline weights at theta = 1/2: 1/48, 23/48, 23/48, 1/48
  for (int i = 0; i < N; ++i) {
    const double v = (E[i * np] + E[(i + 3) * np]) * (1.0 / 48.0) + (E[(i + 1) * np] + E[(i + 2) * np]) * (23.0 / 48.0);
    g[(long long)(2 * i + 1) * np + j] = v;
  }
}

__global__ void k_sem_rho(int nx, int np, double dx, const double *g, const double *phr, const double *phi,
                          double2 *rho) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nx * nx) return;
  const int b = e / nx, c = e % nx;
  if (b > c) return;
  const double *gr = g + (long long)(b + c) * np;
  const long long m = (long long)(c - b + nx - 1) * np;
  double re = 0.0, im = 0.0;
  for (int j = 0; j < np; ++j) {
    re = fma(gr[j], phr[m + j], re);
    im = fma(-gr[j], phi[m + j], im);
  }
  rho[(long long)b * nx + c] = make_double2(dx * re, b == c ? 0.0 : dx * im);
  rho[(long long)c * nx + b] = make_double2(dx * re, b == c ? 0.0 : -dx * im);
}

inline int grid_for(long long n, int nt) {
  long long g = (n + nt - 1) / nt;
  return (int)(g < 152LL * 32 ? (g > 0 ? g : 1) : 152LL * 32);
}

}  // namespace

cudaError_t launch_sem_osc(const SemTabArgs &a, cudaStream_t s) {
  if (a.Q > 32) return cudaErrorInvalidValue;
  k_sem_osc<<<(a.nx + 63) / 64, 64, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sem_tables(const SemTabArgs &a, cudaStream_t s) {
  const long long npsi = (long long)(2 * a.nx - 1) * a.np * a.np;
  k_sem_psi<<<grid_for(npsi, 256), 256, 0, s>>>(a);
  k_sem_phi<<<grid_for((long long)(2 * a.h + 1) * a.np, 256), 256, 0, s>>>(a);
  const long long nas = (long long)4 * (a.h + 1) * a.np * 2 + (long long)a.np * 2 * (2 * a.h + 1);
  k_sem_assemble<<<grid_for(nas, 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sem_phi(const SemTabArgs &a, cudaStream_t s) {
  k_sem_phi<<<grid_for((long long)(2 * a.h + 1) * a.np, 256), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sem_marginal(int nx, int np, double dx, const double *f, const double *w, double *xs,
                                double *n, cudaStream_t s) {
  k_sem_xsum<<<nx * nx, 256, 0, s>>>(np, f, w, xs);
  k_sem_dens<<<(nx + 127) / 128, 128, 0, s>>>(nx, dx, xs, n);
  return cudaGetLastError();
}

cudaError_t launch_sem_potential(const SemPotArgs &a, cudaStream_t s) {
  k_sem_potential<<<2, 256, sizeof(double) * a.nx, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sem_dmul(int nx, int h, int x0, int nb, const double *wgrid, double *A, cudaStream_t s) {
  const long long total = (long long)2 * (h + 1) * (2 * h + 1) * nb;
  k_sem_dmul<<<grid_for(total, 256), 256, 0, s>>>(nx, h, x0, nb, wgrid, A);
  return cudaGetLastError();
}

int sem_adv_cols(int nx, int np) {
  int C = 64;
  while (C > 8 && (size_t)C * (nx + 6) * sizeof(double) > 56 * 1024) C >>= 1;
  while (C > 8 && C / 2 >= np) C >>= 1;
  return C;
}

cudaError_t launch_sem_adv(int axis, const SemAdvArgs &a, cudaStream_t s, int df) {
  const size_t smem = sizeof(double) * a.C * (a.nx + 6);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  const long long nblk = (long long)a.nx * a.np * ((a.np + a.C - 1) / a.C);
  if (nblk > 0x7fffffffLL) return cudaErrorInvalidValue;
  cudaError_t e;
  if (df) {
    if (!a.cpdf || !a.wtsdf) return cudaErrorInvalidValue;
    auto kern = axis == 0 ? k_sem_adv_df<0> : k_sem_adv_df<1>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)nblk, 4 * a.C, smem, s>>>(a);
    return cudaGetLastError();
  }
  if (axis == 0) {
    e = cudaFuncSetAttribute(k_sem_adv<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sem_adv<0><<<(unsigned)nblk, 4 * a.C, smem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_sem_adv<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sem_adv<1><<<(unsigned)nblk, 4 * a.C, smem, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_sem_axpy(long long n, const double *x, double a, const double *y, const double *y2, double *out,
                            cudaStream_t s) {
  k_sem_axpy<<<grid_for(n, 256), 256, 0, s>>>(n, x, a, y, y2, out);
  return cudaGetLastError();
}

cudaError_t launch_sem_rdm(int nx, int np, double dx, const double *f, const double *w, const double *cp, double *f1,
                           double *eta, double *g, const double *phr, const double *phi, double2 *rho, cudaStream_t s) {
  k_sem_f1<<<nx * np, 128, 0, s>>>(nx, np, dx, f, w, f1);
  k_sem_halfgrid<<<(np + 63) / 64, 64, 0, s>>>(nx, np, f1, cp, eta, g);
  k_sem_rho<<<(nx * nx + 127) / 128, 128, 0, s>>>(nx, np, dx, g, phr, phi, rho);
  return cudaGetLastError();
}

cudaError_t launch_sem_erm(int np, int Ny, const double *eier, double *erm, cudaStream_t s) {
  k_sem_erm<<<grid_for((long long)np * 2 * Ny, 256), 256, 0, s>>>(np, Ny, eier, erm);
  return cudaGetLastError();
}

cudaError_t launch_sem_negcols(int rows, int cols, int c0, const double *in, double *out, cudaStream_t s) {
  k_sem_negcols<<<grid_for((long long)rows * cols, 256), 256, 0, s>>>(rows, cols, c0, in, out);
  return cudaGetLastError();
}

cudaError_t launch_sem_scale(long long n, double a, const double *in, double *out, cudaStream_t s) {
  k_sem_scale<<<grid_for(n, 256), 256, 0, s>>>(n, a, in, out);
  return cudaGetLastError();
}

cudaError_t launch_sem_obs(const SemObsArgs &a, cudaStream_t s) {
  const int nt = a.np >= 256 ? 256 : 32 * ((a.np + 31) / 32);  // a thread per row
  k_sem_obs_x<<<a.nx * a.nx, nt, sizeof(double) * 2 * a.np, s>>>(a);
  double *mid = a.xpart + (long long)a.nx * a.nx * (4 + a.np);
  k_sem_obs_mid<<<a.nx, 256, 0, s>>>(a, mid);
  k_sem_obs_fin<<<1, 1024, sizeof(double) * 2 * a.nx, s>>>(a, mid);
  return cudaGetLastError();
}

}  // namespace w2sem
