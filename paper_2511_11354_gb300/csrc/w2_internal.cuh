// Internal declarations shared by the w2 library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/w2.h"

namespace w2 {

// Static one-body / pair potential samples and the per-call densities that
// build the kernels K(x, j) of the pseudo-difference operator (Sec. 3.1):
//   K(x, j) = 1/(hbar nk) sum_{l=1}^{nk-1} [U(x + l h') - U(x - l h')] sin(pi l j / nk)
// with h' = L / (2 nk); K(x, -j) = -K(x, j), K(x, 0) = 0.
struct TabArgs {
  int nx, nk, M;
  double dx, dp, hbar;
  double gamma, c_h, c_xc;
  int xc_kind;
  int pair_mode;            // 1: U = gamma W(d dx + l h') for row d (the pair kernel K12)
  const double *xsum;       // [nx][nx] per-X momentum sums of the state (or null)
  const double *vext_fine;  // [nx][M]
  const double *w_fine;     // [nx][M]
  const double *d_fine;     // [nx][M] trigonometric interpolation weights (xc only)
  const double *sintab;     // [M] sin(pi m / nk)
  double *K;                // pair_mode 0: [2][nx][2nk-1]; pair_mode 1: [nx][2nk-1]
};

struct ThetaArgs {
  int nx;
  const double *in;         // state the operator acts on
  const double *h;          // corrector base (mode 1) or null
  double *out;              // mode 0: Theta[in]; mode 1: h + half_tau Theta[in]
  double *xsum;             // mode 1: per-X sums of out
  const double *K1, *K2, *K12;
  double half_tau;
};

struct AdvArgs {
  int nx;
  const double *in0, *in1;  // arrays to shift (in1 may be null)
  double *out0, *out1;      // outputs
  const int *k0tab;         // [nk] integer part of the foot offset
  const double *wtab;       // [nk][4] B-spline weights times -6 z
  double z, zscale;         // pole z = sqrt(3) - 2 and 1/(1 - z^n) (or 1)
  int nterm;                // terms of the periodic initial sums
  double tau;               // combination weight (x1 pass with two arrays)
};

struct ObsArgs {
  int nx, nk, M;
  double dx, dp, hbar, mass, gamma, c_h;
  const double *f;
  const double *vext_grid;  // [nx]
  const double *w_fine;     // [nx][M]; column 0 is W(fold(d dx))
  double *xpart;            // [nx*nx][3 + nk] per-X partials
  double *out;              // [8 + nx + nx*nx]
};

// Launchers (return the launch error).
cudaError_t launch_tables(const TabArgs &a, cudaStream_t s);
cudaError_t launch_theta_f64(int nk, int mode, const ThetaArgs &a, cudaStream_t s);
cudaError_t launch_adv_f64(int nk, int dir, int two, const AdvArgs &a, cudaStream_t s);
cudaError_t launch_xsum_f64(int nx, int nk, const double *f, double *xsum, cudaStream_t s);
cudaError_t launch_obs_f64(const ObsArgs &a, cudaStream_t s);
cudaError_t prepare_kernels_f64(int nk);
bool nk_supported_f64(int nk);

}  // namespace w2
