/*
 * w2_sem.h -- C ABI of the non-periodic path of the w2 library: the Wigner
 * equation of the two-body reduced density matrix on a bounded box, with the
 * momentum axes discretised by Chebyshev spectral elements.
 *
 * The equation is the one of w2.h (arXiv:2511.11354, Sec. 2.4,
 * Eq. two_body_truncated_Wigner),
 *
 *   d_t f + (p1/m) d_x1 f + (p2/m) d_x2 f
 *       = Theta_{U1}[f] + Theta_{U2}[f] + Theta_{gamma W}[f],
 *
 * now on the box [-L/2, L/2]^2 outside which the density vanishes:
 *   - Theta_U (one body) is the Chebyshev spectral approximation of
 *     Sec. 3.2.1 (Eq. Chebyshev_PDO): f is expanded in Chebyshev polynomials
 *     on each momentum cell, the momentum integral of every basis function is
 *     done exactly through O_l(z) = int_{-1}^{1} e^{i z eta} T_l(eta) deta
 *     (Eq. basic_osc_int), and the position integral is the sum over the
 *     spatial grid (Poisson summation, periodic images dropped);
 *   - Theta_{gamma W} (two body) is the Poisson-summation form of Sec. 3.2.2:
 *     a sum over a uniform (y1, y2) grid of e^{-2i p.y/hbar} D_V(y) times the
 *     exact transform of the cell expansions (the two-body tensor
 *     O_{s1,s2,l1,l2});
 *   - U_i = V_ext + c_H V_H[n_i] + c_xc phi(n_i), with the Hartree potential
 *     V_H[n](x) = dx sum_q W(x - x_q) n(x_q) -- the zero-padded convolution
 *     of the remark in Sec. 3.2.1, which for 3-fold padding equals this
 *     direct sum;
 *   - a step is the Lawson predictor-corrector of Sec. 4.1 with the shift
 *     X -> X - tau P / m by cubic B-splines under the natural boundary
 *     condition (Sec. 4.1, matrix A_nat, ghost values 0).
 *
 * Readings of the paper fixed by this library:
 *   - each momentum cell holds nq Chebyshev-Gauss points (roots of T_nq);
 *     cells share no point;
 *   - Theta_U f(x,p) = (1/(i hbar)) (1/(pi hbar)) int dy int dp'
 *       e^{-2i(p-p')y/hbar} [U(x+y) - U(x-y)] f(p')  (classical limit
 *     U'(x) d_p f), the same sign as the periodic path;
 *   - the two-body y grid is y_n = n dx, |n| <= (nx-1)/2, and
 *     D_V(y) = W(r + y1 - y2) - W(r - y1 + y2), r = x1 - x2;
 *   - the Hartree term (c_H) and the pair term (gamma) have separate
 *     strengths;
 *   - the spline sum over nu = -1 .. nx runs wherever the departure point
 *     falls, with zero coefficients beyond (zero inflow).
 *
 * Grid:
 *   x_i = -L/2 + i dx, dx = L / (nx - 1), i in [0, nx)  (both ends included)
 *   momentum cells s in [0, ncell): [-Lp/2 + s w, -Lp/2 + (s+1) w], w = Lp/ncell;
 *   p_{s nq + q} = -Lp/2 + (s + 1/2) w - (w/2) cos((2q+1) pi / (2 nq)), ascending;
 *   np = ncell * nq momenta per axis;
 *   phase-space arrays are f[i1][i2][j1][j2], j2 fastest, C order, FP64,
 *   nx*nx*np*np elements.
 *
 * Conventions are those of w2.h: every call returns a w2_status; the first
 * CUDA error of a context sticks until w2_sem_destroy; the caller owns every
 * pointer it passes and nothing is retained after a call, except the stream
 * (borrowed); device pointers are CUDA global-memory addresses on the
 * context's device; work is queued on the stream except where a function says
 * it synchronises; there is no CPU fallback.
 */
#ifndef W2_SEM_H
#define W2_SEM_H

#include "w2.h"

#ifdef __cplusplus
extern "C" {
#endif

/* nx   : spatial points per axis, 8 <= nx <= 1024
 * ncell: momentum cells per axis, >= 1;  nq: points per cell, 2 <= nq <= 32;
 *        ncell * nq <= 256
 * L    : box length (> 0);  Lp: momentum window length (> 0), with
 *        (Lp / ncell) * L / hbar <= 4096
 * dt   : time step tau (> 0);  hbar, mass: > 0
 * xc_kind: a w2_xc_kind
 * precision: W2_F64 -- the operator's products on the FP64 pipe; or
 *   W2_F64_SLICED -- the same products from exact 8-bit slices of the FP64
 *   operands on the BF16 tensor cores (six digits per value, the 21 digit
 *   pairs above 2^-48 of the line scales kept, integer recombination;
 *   nx <= 256); FP64 state and results either way */
typedef struct {
  int32_t nx, ncell, nq;
  double L, Lp, dt, hbar, mass;
  int32_t xc_kind;
  int32_t precision;
} w2_sem_config;

typedef struct w2_sem_ctx w2_sem_ctx;

/* Create a context on the current CUDA device; builds the static tables
 * (oscillatory integrals by the Jacobi-Anger expansion with Bessel values
 * from Miller's backward recurrence, cell transforms, spline weights) on the
 * device and synchronises.  W2_ERR_ARG for sizes outside the limits above,
 * W2_ERR_OOM when device memory runs out. */
w2_status w2_sem_create(const w2_sem_config *cfg, void *cuda_stream, w2_sem_ctx **out);

/* Potentials, evaluated on the host once: vext at the grid points and vee at
 * the multiples k dx, |k| <= 2 (nx - 1).  gamma scales the pair term, c_h the
 * Hartree term, c_xc the exchange-correlation term.  Synchronises. */
w2_status w2_sem_set_potentials(w2_sem_ctx *ctx, w2_fn vext, void *ue, w2_fn vee, void *ui,
                                double gamma, double c_h, double c_xc);

/* Collocation momenta p[np] and the weights w[np] of the momentum integral
 * (the exact integral of the cell expansion), host arrays. */
w2_status w2_sem_momenta(const w2_sem_ctx *ctx, double *p, double *w);

/* Copy a state in or out (device or host pointer).  get_state with
 * on_device = 0 synchronises. */
w2_status w2_sem_set_state(w2_sem_ctx *ctx, const double *f, int32_t on_device);
w2_status w2_sem_get_state(w2_sem_ctx *ctx, double *f, int32_t on_device);

/* out = Theta_{U1}[in] + Theta_{U2}[in] + Theta_{gamma W}[in], with U built
 * from the densities of `in` (device arrays of the state's shape; they must
 * not overlap). */
w2_status w2_sem_theta(w2_sem_ctx *ctx, const double *in, double *out);

/* out = in(X - tau P / m, P) by the natural-boundary spline shift, x1 first
 * then x2 (device arrays; they must not overlap). */
w2_status w2_sem_advect(w2_sem_ctx *ctx, const double *in, double *out);

/* nsteps Lawson steps of the state.  W2_ERR_STATE before set_potentials and
 * set_state. */
w2_status w2_sem_step(w2_sem_ctx *ctx, int32_t nsteps);

/* Observables of the state (definitions of w2_obs with every momentum sum
 * replaced by the momentum quadrature w, and the Hartree energy
 * (c_h/2) dx sum_i n(x_i) V_H[n](x_i) for each particle); n1 (host, [nx]) may
 * be NULL.  Synchronises. */
w2_status w2_sem_observables(w2_sem_ctx *ctx, w2_obs *out, double *n1);

/* Occupation numbers and correlation entropy of the one-body density matrix
 * of the state (the strongly correlated example, Sec. 5.4, and the appendix
 * on the correlation entropy): f1 = dx sum_{x2} int f dp2; the inverse Wigner
 * transform rho1(x_b, x_c) = int f1((x_b + x_c)/2, p) e^{-i p (x_c - x_b)/hbar} dp
 * taken exactly over the cell expansions (the transform of the two-body term
 * at half the offset), f1 at half points from the natural cubic spline;
 * occ[nx] (host, may be NULL) receives the eigenvalues of rho1 dx, largest
 * first, by the eigensolver of w2_hermitian_eigvals, and *entropy
 * (may be NULL) s = sum n ln n / sum n over the occupations above 1e-14 of
 * the largest.  The first call allocates its work arrays (about
 * 16 nx^2 + 40 nx np bytes).  Synchronises. */
w2_status w2_sem_occupations(w2_sem_ctx *ctx, double *occ, double *entropy);

void w2_sem_destroy(w2_sem_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* W2_SEM_H */
