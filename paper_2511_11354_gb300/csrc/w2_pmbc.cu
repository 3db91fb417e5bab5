// Distributed characteristic shift: local cubic splines joined by perfectly
// matched boundary conditions (PMBC, Sec. 4.2).
//
// The axis being shifted is cut into np patches of M = nx / np points.  A
// patch (a rank of a distributed run) holds its own M points; it solves a
// local spline over its points plus G ghost points on each side, with the
// spline's slope at the two ends of that range as boundary conditions
// (the first and last rows of the local system of Sec. 4.2).  The slope of
// the global periodic spline at a point is a fixed stencil of the samples,
//   s'(r_k) = sum_{|j| <= nnb} D_j f(r_{k+j}),
//   D_j = (beta_{j-1} - beta_{j+1}) / (2h),  beta = the inverse of the (1,4,1)/6 circulant,
// whose coefficients decay as |z|^|j| (z = sqrt(3) - 2); with nnb = 26 the
// truncation is below 2^-52 of the line, so the local splines give the
// global spline's coefficients and the shift equals the global one to FP64
// rounding.  Each end's stencil straddles a junction: the part over the
// neighbour's points is summed by the neighbour and sent (one number per line
// and junction, the paper's split of phi into left and right sums), together
// with the G ghost samples the local system needs.  Here every patch runs in
// one process on one device: kernel k_pmbc_send writes each patch's
// outgoing values into exchange buffers (what a rank would hand to its
// neighbours), and k_pmbc_solve reads only its own points and the buffers of
// its two neighbours.  FP64 arithmetic throughout.
#include "w2_internal.cuh"

namespace w2 {
namespace {

// k_pmbc_send: per patch l and line, for each shifted array q:
//   xs[q][l][0] = part of the left neighbour's right-end slope over this patch,
//                 sum_{n = lM}^{lM + G - 1 + nnb} D_{n - (lM + G - 1)} f(n);
//   xs[q][l][1] = part of the right neighbour's left-end slope over this patch,
//                 sum_{n = (l+1)M - G - nnb}^{(l+1)M - 1} D_{n - ((l+1)M - G)} f(n);
//   gh[q][l][0][g] = f(lM + g), gh[q][l][1][g] = f((l+1)M - G + g), g < G.
// Block (patch, line group); one thread per momentum column.
template <int NK, int DIR, int TWO>
__global__ void __launch_bounds__(NK) k_pmbc_send(PatchArgs a) {
  const int l = blockIdx.x % a.np, n1 = (blockIdx.x / a.np) % NK, fixed = blockIdx.x / (a.np * NK);
  const int t = threadIdx.x, M = a.M, G = a.G, nnb = a.nnb, nx = a.nx;
  const size_t lineStride = (DIR == 0) ? (size_t)NK * NK : (size_t)nx * NK * NK;
  const size_t base = (DIR == 0) ? ((size_t)fixed * nx * NK + n1) * NK : ((size_t)fixed * NK + n1) * NK;
  const size_t line = ((size_t)fixed * NK + n1) * NK + t, lines = (size_t)nx * NK * NK;
  const double *D = a.D + nnb;  // D[j], |j| <= nnb
#pragma unroll
  for (int q = 0; q < 1 + TWO; ++q) {
    const double *f = (q == 0 ? a.in0 : a.in1) + base + t;
    double sl = 0.0, sr = 0.0;
    const int cl = l * M + G - 1, cr = (l + 1) * M - G;
    for (int n = l * M; n <= cl + nnb; ++n) sl = fma(D[n - cl], f[n * lineStride], sl);
    for (int n = cr - nnb; n < (l + 1) * M; ++n) sr = fma(D[n - cr], f[n * lineStride], sr);
    double *xs = a.xs + ((size_t)(q * a.np + l) * 2) * lines;
    xs[line] = sl;
    xs[lines + line] = sr;
    double *gh = a.gh + ((size_t)(q * a.np + l) * 2) * G * lines;
    for (int g = 0; g < G; ++g) {
      gh[(size_t)g * lines + line] = f[(size_t)(l * M + g) * lineStride];
      gh[(size_t)(G + g) * lines + line] = f[(size_t)((l + 1) * M - G + g) * lineStride];
    }
  }
}

// k_pmbc_solve: per patch l and line, for each array: the local spline on
// points lo = lM - G .. hi = (l+1)M + G - 1 (n = M + 2G) with the slopes
// phi_L at lo and phi_R at hi as boundary rows,
//   (eta_1 - eta_-1)/(2h) = phi_L,  (eta_{v-1} + 4 eta_v + eta_{v+1})/6 = f_v,
//   (eta_n - eta_{n-2})/(2h) = phi_R,
// eliminated to the tridiagonal (4,2), (1,4,1), (2,4) system and solved with
// the host's Thomas factors; then the value at each own point's foot
// x_i - tau p / m (|shift| < G - 1 cells).  DIR 1 with TWO writes
// out0 = a + tau b and out1 = a + tau/2 b, DIR 0 with TWO out0 = a, out1 = b.
template <int NK, int DIR, int TWO>
__global__ void __launch_bounds__(NK) k_pmbc_solve(PatchArgs a) {
  extern __shared__ double smp[];
  const int l = blockIdx.x % a.np, n1 = (blockIdx.x / a.np) % NK, fixed = blockIdx.x / (a.np * NK);
  const int t = threadIdx.x, M = a.M, G = a.G, nnb = a.nnb, nx = a.nx, n = M + 2 * G;
  const size_t lineStride = (DIR == 0) ? (size_t)NK * NK : (size_t)nx * NK * NK;
  const size_t base = (DIR == 0) ? ((size_t)fixed * nx * NK + n1) * NK : ((size_t)fixed * NK + n1) * NK;
  const size_t line = ((size_t)fixed * NK + n1) * NK + t, lines = (size_t)nx * NK * NK;
  const int lL = (l + a.np - 1) % a.np, lR = (l + 1) % a.np;
  const double *D = a.D + nnb;
  const int sidx = (DIR == 0) ? t : n1;
  const int k0 = a.k0tab[sidx];
  const double w0 = a.wb[4 * sidx], w1 = a.wb[4 * sidx + 1], w2 = a.wb[4 * sidx + 2], w3 = a.wb[4 * sidx + 3];
  const double h = a.h;
  // column of this thread: eta at local index v + 1 for v = -1 .. n (n + 2 rows)
  double *col0 = smp + t, *col1 = smp + (size_t)(n + 2) * NK + t;
#pragma unroll
  for (int q = 0; q < 1 + TWO; ++q) {
    double *col = q == 0 ? col0 : col1;
    const double *f = (q == 0 ? a.in0 : a.in1) + base + t;
    const double *ghL = a.gh + ((size_t)(q * a.np + lL) * 2) * G * lines + (size_t)G * lines;  // left neighbour's right strip
    const double *ghR = a.gh + ((size_t)(q * a.np + lR) * 2) * G * lines;                      // right neighbour's left strip
    // samples of points lo .. hi
    for (int g = 0; g < G; ++g) {
      col[(size_t)(g + 1) * NK] = ghL[(size_t)g * lines + line];
      col[(size_t)(G + M + g + 1) * NK] = ghR[(size_t)g * lines + line];
    }
    for (int v = 0; v < M; ++v) col[(size_t)(G + v + 1) * NK] = f[(size_t)(l * M + v) * lineStride];
    // end slopes: own part plus the neighbour's part
    const int lo = l * M - G, hi = (l + 1) * M + G - 1;
    double pl = a.xs[((size_t)(q * a.np + lL) * 2 + 1) * lines + line];
    for (int m = l * M; m <= lo + nnb; ++m) pl = fma(D[m - lo], f[(size_t)m * lineStride], pl);
    double pr = a.xs[((size_t)(q * a.np + lR) * 2) * lines + line];
    for (int m = hi - nnb; m < (l + 1) * M; ++m) pr = fma(D[m - hi], f[(size_t)m * lineStride], pr);
    // forward sweep on the (x6) system: 4 e0 + 2 e1 = 6 f0 + 2h phi_L, ..., 2 e_{n-2} + 4 e_{n-1} = 6 f_{n-1} - 2h phi_R
    double d = (6.0 * col[NK] + 2.0 * h * pl) * a.inv_m[0];
    col[NK] = d;
    for (int v = 1; v < n; ++v) {
      double r = 6.0 * col[(size_t)(v + 1) * NK];
      if (v == n - 1) r -= 2.0 * h * pr;
      d = (r - (v == n - 1 ? 2.0 : 1.0) * d) * a.inv_m[v];
      col[(size_t)(v + 1) * NK] = d;
    }
    // back substitution eta_v = d_v - c'_v eta_{v+1}
    double e = d;
    for (int v = n - 2; v >= 0; --v) {
      e = fma(-a.cp[v], e, col[(size_t)(v + 1) * NK]);
      col[(size_t)(v + 1) * NK] = e;
    }
    col[0] = col[2 * NK] - 2.0 * h * pl;                                  // eta_-1
    col[(size_t)(n + 1) * NK] = col[(size_t)(n - 1) * NK] + 2.0 * h * pr;  // eta_n
  }
  // values at the feet of the own points i = lM + v: foot cell k = i + k0,
  // local index k - lo = G + v + k0, eta rows (k - lo - 1 .. k - lo + 2) + 1
  for (int v = 0; v < M; ++v) {
    const int r = G + v + k0;  // row of eta_{k - 1}
    const double va = fma(w3, col0[(size_t)(r + 3) * NK],
                          fma(w2, col0[(size_t)(r + 2) * NK], fma(w1, col0[(size_t)(r + 1) * NK], w0 * col0[(size_t)r * NK])));
    const size_t o = base + (size_t)(l * M + v) * lineStride + t;
    if (!TWO) {
      a.out0[o] = va;
    } else {
      const double vb = fma(w3, col1[(size_t)(r + 3) * NK],
                            fma(w2, col1[(size_t)(r + 2) * NK], fma(w1, col1[(size_t)(r + 1) * NK], w0 * col1[(size_t)r * NK])));
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
cudaError_t run_pmbc(int dir, int two, const PatchArgs &a, cudaStream_t s) {
  const int grid = a.np * NK * a.nx;
  const size_t smem = sizeof(double) * (size_t)(two ? 2 : 1) * (a.M + 2 * a.G + 2) * NK;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
#define W2_PM(D, T)                                                                                    \
  if (dir == D && two == T) {                                                                          \
    cudaError_t e = cudaFuncSetAttribute(k_pmbc_solve<NK, D, T>,                                       \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);     \
    if (e != cudaSuccess) return e;                                                                    \
    k_pmbc_send<NK, D, T><<<grid, NK, 0, s>>>(a);                                                      \
    k_pmbc_solve<NK, D, T><<<grid, NK, smem, s>>>(a);                                                  \
    return cudaGetLastError();                                                                         \
  }
  W2_PM(0, 0) W2_PM(0, 1) W2_PM(1, 0) W2_PM(1, 1)
#undef W2_PM
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_adv_pmbc(int nk, int dir, int two, const PatchArgs &a, cudaStream_t s) {
  switch (nk) {
    case 8: return run_pmbc<8>(dir, two, a, s);
    case 16: return run_pmbc<16>(dir, two, a, s);
    case 24: return run_pmbc<24>(dir, two, a, s);
    case 32: return run_pmbc<32>(dir, two, a, s);
    case 40: return run_pmbc<40>(dir, two, a, s);
    case 48: return run_pmbc<48>(dir, two, a, s);
    case 56: return run_pmbc<56>(dir, two, a, s);
    case 64: return run_pmbc<64>(dir, two, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace w2
