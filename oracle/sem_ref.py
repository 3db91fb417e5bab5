"""Plain numpy oracle of the non-periodic path (TEST INFRASTRUCTURE ONLY:
tests/, the smoke check and the benchmark's CPU baseline may import it; the
product path never does).

It follows, step by step and in the paper's order:

* Sec. 3.2 -- the momentum window split into cells, each carrying a
  Chebyshev expansion of f (Eqs. spectral_representation, eq:base); the
  one-body operator through the tensors T+- of Eq. Chebyshev_PDO and the
  oscillatory integrals O_l(z) = int_{-1}^{1} e^{i z eta} T_l(eta) deta of
  Eq. basic_osc_int; the two-body operator through the Poisson-summation
  form of Sec. 3.2.2 (sum over a uniform y grid of e^{-2i p.y} D_V(y) times
  the exact transform of the cell expansions, the two-body tensor
  O_{s1,s2,l1,l2});
* the remark of Sec. 3.2.1 -- the Hartree potential by the zero-padded FFT
  with N~ = 3 N_x;
* Sec. 4.1 -- the Lawson predictor-corrector and the cubic B-spline shift
  with the natural boundary condition (matrix A_nat, ghost values 0).

Everything is FP64.  Library primitives used as steps: Gauss-Legendre nodes
(numpy), matrix products, FFTs and one LU factorisation (scipy).

Readings where the paper is silent, garbled or inconsistent (the design
notes list them as R17-R24):
  R17 nodes: each cell holds nq Chebyshev-Gauss points (roots of T_nq), so
      cells share no point (8 cells x 16 points = 128 per axis as printed);
      coefficients come from the exact discrete Chebyshev transform at those
      points; integrals over p use the exact integral of the cell expansion
      (Fejer's first rule).
  R18 operator: Theta_U f(x,p) = (1/(i hbar)) (1/(pi hbar)) int dy int dp'
      e^{-2i(p-p')y/hbar} [U(x+y) - U(x-y)] f(p'), the sign reading of the
      periodic path (classical limit +U' d_p f); printed |P|/2 vs |P| and the
      position of hbar are taken from this form (they matter only for
      hbar != 1).  The y integral is the paper's sum over the spatial grid
      (y = x_n - x for the one-body term; the potential is sampled on the
      grid only).
  R19 two-body term: D_V(y) = W(r + y1 - y2) - W(r - y1 + y2), r = x1 - x2,
      with the y grid spacing equal to dx (the paper's dy = pi hbar / L_p
      equals dx in every run it reports) and y_n = n dx, |n| <= (nx-1)/2.
  R20 strengths: the Hartree term is c_H dx sum_q W(x - x_q) n(x_q) and the
      pair term gamma W(x1 - x2), two separate switches (Hamiltonians I and
      II carry a Hartree term and no pair term).
  R21 Hartree by zero padding: N~ = 3 (nx - 1), kernel W(nu dx) for
      nu in the centred range of N~, V_H = dx * cyclic convolution; for
      N~ >= 2 nx - 1 this equals the direct sum dx sum_q W(x_m - x_q) n_q.
  R22 spline: the B-spline sum over nu = -1 .. nx (paper's N_x + 1 with
      N_x = nx - 1 intervals) is evaluated wherever the departure point
      falls, with eta = 0 beyond that range (zero inflow further out).
  R23 x quadrature: dx sum over the nx points (f vanishes at both ends).
  R24 initial data: the Gaussian parameter a of the strongly correlated
      example is 1/4 (unit spatial width, as the other workloads).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


def osc_integral(lmax: int, z: np.ndarray) -> np.ndarray:
    """O_l(z) = int_{-1}^{1} e^{i z eta} T_l(eta) deta for l < lmax (Eq.
    basic_osc_int), by Gauss-Legendre quadrature with enough nodes that the
    entire integrand is integrated to rounding.  Returns [lmax][*z.shape]."""
    z = np.asarray(z, dtype=np.float64)
    n = int(math.ceil(float(np.abs(z).max(initial=0.0)))) + 2 * lmax + 64
    t, w = np.polynomial.legendre.leggauss(n)
    T = np.cos(np.outer(np.arange(lmax), np.arccos(t)))          # [l][k]
    E = np.exp(1j * np.multiply.outer(z.reshape(-1), t))        # [z][k]
    O = (T * w[None, :]) @ E.T                                   # [l][z]
    return O.reshape((lmax,) + z.shape)


def phi_xc(kind: int, n):
    n = np.asarray(n, dtype=np.float64)
    if kind == 1:
        return n.copy()
    if kind == 2:  # Hedin-Lundqvist exchange-correlation potential, atomic units
        c = np.cbrt(np.maximum(n, 0.0))
        return 0.985 * c + 0.985 * 0.034 * np.log1p(18.37 * c)
    return np.zeros_like(n)


class SemOracle:
    """Oracle of one non-periodic problem (an inputs.SemProblem)."""

    def __init__(self, prob):
        self.P = prob
        nx, M, Q = prob.nx, prob.ncell, prob.nq
        self.nx, self.M, self.Q, self.np_ = nx, M, Q, M * Q
        self.hbar, self.mass = prob.hbar, prob.mass
        self.dx = prob.L / (nx - 1)
        self.x = -0.5 * prob.L + self.dx * np.arange(nx)
        # cells [d_s, d_{s+1}], width |P_s|, centre d^_s (Eq. eq:base)
        self.width = prob.Lp / M
        self.centre = -0.5 * prob.Lp + self.width * (np.arange(M) + 0.5)
        self.eta = -np.cos((2 * np.arange(Q) + 1) * np.pi / (2 * Q))
        self.p = (self.centre[:, None] + 0.5 * self.width * self.eta[None, :]).reshape(-1)
        # discrete Chebyshev transform at the Gauss points: b_l = sum_q C[l][q] f_q
        T = np.cos(np.outer(np.arange(Q), np.arccos(self.eta)))  # T_l(eta_q)
        self.Tq = T
        self.C = T * np.where(np.arange(Q) == 0, 1.0, 2.0)[:, None] / Q
        l = np.arange(Q)
        intT = np.array([2.0 / (1.0 - k * k) if k % 2 == 0 else 0.0 for k in l])  # int_{-1}^{1} T_l
        self.w = np.tile(0.5 * self.width * (intT @ self.C), M)   # weights of int dp
        self.h = (nx - 1) // 2
        self.y2 = self.dx * np.arange(-self.h, self.h + 1)        # two-body y grid
        self.vext = np.array([prob.vext(float(v)) for v in self.x])
        self._Wcache = {}
        # natural-spline matrix A_nat (Sec. 4.1), LU-factorised once
        N = nx - 1
        A = np.zeros((N + 3, N + 3))
        A[0, 0:3] = np.array([6.0, -12.0, 6.0]) / self.dx ** 2
        for nu in range(N + 1):
            A[nu + 1, nu:nu + 3] = [1.0, 4.0, 1.0]
        A[N + 2, N:N + 3] = np.array([6.0, -12.0, 6.0]) / self.dx ** 2
        self.Anat_lu = sla.lu_factor(A / 6.0)

    # ------------------------------------------------------------------ helpers
    def W(self, r):
        r = np.asarray(r, dtype=np.float64)
        return np.vectorize(lambda v: float(self.P.vee(float(v))), otypes=[np.float64])(r)

    def cell_coeffs(self, f, axis):
        """Chebyshev coefficients b_{s,l} of the cell expansions along ``axis``
        (momentum index s*Q + q -> (s, l))."""
        f = np.moveaxis(f, axis, -1)
        sh = f.shape[:-1]
        b = np.einsum("lq,...sq->...sl", self.C, f.reshape(sh + (self.M, self.Q)))
        return np.moveaxis(b.reshape(sh + (self.np_,)), -1, axis)

    def basis_transform(self, y):
        """(|P|/2) e^{2i d^_s y / hbar} O_l(|P| y / hbar): the exact
        int_{P_s} e^{2i p' y / hbar} C_l(p') dp' of one cell basis function;
        returns [len(y)][s*Q + l]."""
        y = np.asarray(y, dtype=np.float64)
        O = osc_integral(self.Q, self.width * y / self.hbar)               # [l][y]
        ph = np.exp(2j * np.outer(y, self.centre) / self.hbar)              # [y][s]
        return (0.5 * self.width * ph[:, :, None] * O.T[:, None, :]).reshape(len(y), self.np_)

    # ------------------------------------------------------------ potentials
    def marginal(self, f):
        """n1(x_i) = dx sum_{i2} int int f dp1 dp2 (and n2 = the same with the
        roles swapped)."""
        n1 = self.dx * np.einsum("abcd,c,d->a", f, self.w, self.w)
        n2 = self.dx * np.einsum("abcd,c,d->b", f, self.w, self.w)
        return n1, n2

    def hartree(self, n):
        """Zero-padded FFT Hartree (remark of Sec. 3.2.1), N~ = 3 (nx-1)."""
        Nt = 3 * (self.nx - 1)
        nu = np.rint(np.fft.fftfreq(Nt) * Nt)
        k = self.W(nu * self.dx)
        npad = np.zeros(Nt)
        npad[: self.nx] = n
        return self.dx * np.real(np.fft.ifft(np.fft.fft(k) * np.fft.fft(npad)))[: self.nx]

    def potential(self, n):
        P = self.P
        U = self.vext.copy()
        if P.c_hartree != 0.0:
            U += P.c_hartree * self.hartree(n)
        if P.c_xc != 0.0 and P.xc_kind:
            U += P.c_xc * phi_xc(P.xc_kind, n)
        return U

    # ---------------------------------------------------------------- Theta
    def T_tensors(self, U, ms=None):
        """T+-[m][i][s*Q+l] = sum_n U(x_n) e^{+-2i (p_i - d^_s)(x_n - x_m)/hbar}
        |P| O_l(-+|P| (x_n - x_m)/hbar) (Sec. 3.2.1), for the targets ms
        (all grid points by default)."""
        nx, hb = self.nx, self.hbar
        ms = range(nx) if ms is None else ms
        d = np.arange(-(nx - 1), nx) * self.dx                     # all x_n - x_m
        O = osc_integral(self.Q, self.width * d / hb)               # [l][d]
        Tp = np.zeros((len(ms), self.np_, self.np_), dtype=np.complex128)
        Tm = np.zeros_like(Tp)
        dps = self.p[:, None] - self.centre[None, :]                # p_i - d^_s   [i][s]
        for k, m in enumerate(ms):
            y = self.x - self.x[m]                                  # x_n - x_m
            idx = np.arange(nx) - m + (nx - 1)
            Opos = O[:, idx]                                        # O_l(+|P| y)   [l][n]
            ph = np.exp(2j * dps[:, :, None] * y[None, None, :] / hb)   # [i][s][n]
            # O_l(-z) = conj(O_l(z)) for real z
            tp = np.einsum("n,isn,ln->isl", U, ph, np.conj(Opos))
            tm = np.einsum("n,isn,ln->isl", U, np.conj(ph), Opos)
            Tp[k] = self.width * tp.reshape(self.np_, self.np_)
            Tm[k] = self.width * tm.reshape(self.np_, self.np_)
        return Tp, Tm

    def theta_one_body(self, f, U1, U2):
        """Mean-field part: sum over cells and degrees of the coefficient
        b_{s,l} (along p1 for particle 1, p2 for particle 2) times
        (dx / (2 i pi hbar^2)) (T-_{s,l} - T+_{s,l})."""
        pref = self.dx / (2j * math.pi * self.hbar ** 2)
        # the kernel pref (T- - T+) is real for real U (T+ = conj T-); its
        # imaginary part is rounding and is dropped before the contraction
        Tp1, Tm1 = self.T_tensors(U1)
        G1 = (pref * (Tm1 - Tp1)).real                               # [i1][p1][s1 l1]
        b1 = self.cell_coeffs(f, 2)                                 # [i1][i2][s1 l1][p2]
        out = np.matmul(G1[:, None], b1)
        Tp2, Tm2 = (Tp1, Tm1) if U2 is U1 else self.T_tensors(U2)
        G2 = (pref * (Tm2 - Tp2)).real                               # [i2][p2][s2 l2]
        b2 = self.cell_coeffs(f, 3)                                 # [i1][i2][p1][s2 l2]
        out += np.matmul(b2, np.swapaxes(G2, 1, 2)[None])
        return out

    def _two_body_parts(self):
        y = self.y2
        B = self.basis_transform(y)                                 # [y][s l]
        E = np.exp(-2j * np.outer(self.p, y) / self.hbar)           # [p][y]
        Y1, Y2 = np.meshgrid(y, y, indexing="ij")
        pref = self.P.gamma * self.dx * self.dx / (1j * self.hbar * (math.pi * self.hbar) ** 2)
        return B, E, Y1 - Y2, pref

    def _two_body_block(self, parts, i1, i2, a):
        """Theta_{gamma W} at X = (x_i1, x_i2) from the block's coefficients a."""
        B, E, U12, pref = parts
        D = self._D(self.x[i1] - self.x[i2], U12)
        Fh = B @ a @ B.T                                             # F^(y1, y2)
        return (pref * (E @ (D * Fh) @ E.T)).real

    def theta_two_body(self, f):
        """Sec. 3.2.2: (gamma dy^2 / (i hbar (pi hbar)^2)) sum_{y1,y2}
        e^{-2i (p1 y1 + p2 y2)/hbar} D_V(y1, y2) sum a_{s1 s2 l1 l2}
        O_{s1 s2 l1 l2}(y1, y2), with the two-body tensor a product of two
        one-cell transforms."""
        if self.P.gamma == 0.0:
            return np.zeros_like(f)
        parts = self._two_body_parts()
        a = self.cell_coeffs(self.cell_coeffs(f, 2), 3)              # [i1][i2][s1 l1][s2 l2]
        out = np.zeros(f.shape)
        for i1 in range(self.nx):
            for i2 in range(self.nx):
                out[i1, i2] = self._two_body_block(parts, i1, i2, a[i1, i2])
        return out

    def theta_sample(self, f, xs):
        """Theta at the flat spatial indices xs (X = i1 nx + i2) only; the
        potentials come from the densities of the whole state."""
        n1, n2 = self.marginal(f)
        U1, U2 = self.potential(n1), self.potential(n2)
        pref = self.dx / (2j * math.pi * self.hbar ** 2)
        i1s = [int(X) // self.nx for X in xs]
        i2s = [int(X) % self.nx for X in xs]
        Tp1, Tm1 = self.T_tensors(U1, i1s)
        Tp2, Tm2 = self.T_tensors(U2, i2s)
        parts = self._two_body_parts() if self.P.gamma != 0.0 else None
        out = np.zeros((len(xs), self.np_, self.np_))
        for k, (i1, i2) in enumerate(zip(i1s, i2s)):
            blk = f[i1, i2]
            G1 = (pref * (Tm1[k] - Tp1[k])).real
            G2 = (pref * (Tm2[k] - Tp2[k])).real
            out[k] = G1 @ self.cell_coeffs(blk, 0) + self.cell_coeffs(blk, 1) @ G2.T
            if parts is not None:
                out[k] += self._two_body_block(parts, i1, i2, self.cell_coeffs(self.cell_coeffs(blk, 0), 1))
        return out

    def _D(self, r, u):
        key = round(r / self.dx)
        if key not in self._Wcache:
            self._Wcache[key] = self.W(r + u) - self.W(r - u)
        return self._Wcache[key]

    def theta_with(self, f, U1, U2, one_body=True, two_body=True):
        out = np.zeros(f.shape)
        if one_body:
            out += self.theta_one_body(f, U1, U2)
        if two_body:
            out += self.theta_two_body(f)
        return out

    def theta(self, f):
        n1, n2 = self.marginal(f)
        return self.theta_with(f, self.potential(n1), self.potential(n2))

    # ------------------------------------------------------------- advection
    @staticmethod
    def _bspline(r, rnu, h):
        """B_nu(r) of Sec. 4.1, the four printed pieces."""
        t = (r - rnu) / h
        out = np.zeros_like(t)
        m = (t >= -2) & (t < -1)
        out[m] = (t[m] + 2) ** 3 / 6
        m = (t >= -1) & (t < 0)
        a = t[m] + 1
        out[m] = -a ** 3 / 2 + a ** 2 / 2 + a / 2 + 1.0 / 6
        m = (t >= 0) & (t < 1)
        a = 1 - t[m]
        out[m] = -a ** 3 / 2 + a ** 2 / 2 + a / 2 + 1.0 / 6
        m = (t >= 1) & (t <= 2)
        out[m] = (2 - t[m]) ** 3 / 6
        return out

    def spline_coeffs(self, f, axis):
        """eta_{-1..N+1} along ``axis`` from A_nat eta = (0, f_0..f_N, 0)."""
        g = np.moveaxis(f, axis, 0)
        rhs = np.zeros((self.nx + 2,) + g.shape[1:])
        rhs[1:-1] = g
        eta = sla.lu_solve(self.Anat_lu, rhs.reshape(self.nx + 2, -1)).reshape(rhs.shape)
        return eta                                                  # axis 0 = nu + 1

    def shift_matrix(self, s):
        """S[i][nu+1] = B_nu(x_i - s), nu = -1..N+1."""
        rnu = self.x[0] + self.dx * np.arange(-1, self.nx + 1)
        return self._bspline((self.x - s)[:, None], rnu[None, :], self.dx)

    def advect(self, f):
        """f(X - tau P / m, P): x1 pass then x2 pass."""
        tau = self.P.dt
        out = np.empty_like(f)
        eta = self.spline_coeffs(f, 0)                              # [nu][i2][p1][p2]
        for j in range(self.np_):
            S = self.shift_matrix(tau * self.p[j] / self.mass)
            out[:, :, j, :] = np.einsum("in,nbd->ibd", S, eta[:, :, j, :])
        g = out
        out = np.empty_like(f)
        eta = self.spline_coeffs(g, 1)                              # [nu][i1][p1][p2]
        for j in range(self.np_):
            S = self.shift_matrix(tau * self.p[j] / self.mass)
            out[:, :, :, j] = np.einsum("in,nac->aic", S, eta[:, :, :, j])
        return out

    # ------------------------------------------------------------------ step
    def step(self, f, nsteps=1):
        """Lawson predictor-corrector (Sec. 4.1); the mean-field potential of
        each Theta comes from that Theta's input."""
        tau = self.P.dt
        for _ in range(nsteps):
            g = self.theta(f)
            a = self.advect(f)
            b = self.advect(g)
            ft = a + tau * b
            c = self.theta(ft)
            f = a + 0.5 * tau * (b + c)
        return f

    # ----------------------------------------------------------- observables
    def observables(self, f):
        P, dx, w = self.P, self.dx, self.w
        n1, n2 = self.marginal(f)
        ww = np.outer(w, w)
        mass = dx * dx * np.einsum("abcd,cd->", f, ww)
        x = self.x
        r = x[:, None] - x[None, :]
        Wr = self.W(r)
        pe = (self.p[:, None] ** 2 + self.p[None, :] ** 2) / (2 * self.mass)
        e = dx * dx * (np.einsum("abcd,cd,cd->", f, ww, pe)
                       + np.einsum("abcd,cd,a->", f, ww, self.vext)
                       + np.einsum("abcd,cd,b->", f, ww, self.vext)
                       + P.gamma * np.einsum("abcd,cd,ab->", f, ww, Wr))
        if P.c_hartree != 0.0:
            e += 0.5 * P.c_hartree * dx * (np.dot(n1, self.hartree(n1)) + np.dot(n2, self.hartree(n2)))
        f1 = dx * np.einsum("abcd,d->ac", f, w)
        purity = 2 * math.pi * self.hbar * dx * np.einsum("ac,c->", f1 * f1, w)
        l2 = math.sqrt(dx * dx * np.einsum("abcd,cd->", f * f, ww))
        return {"mass": mass, "energy": e, "purity": purity, "entropy_lin": 1.0 - purity,
                "l2norm": l2, "n1": n1}


# ---------------------------------------------------------------------------
# Occupation numbers and correlation entropy of the one-body density matrix
# (the strongly correlated example of Sec. 5.4 and the appendix on the
# correlation entropy), on the bounded box.
#
# Readings (R25): the inverse Wigner transform
#   rho1(r - y/2, r + y/2) = int f1(r, p) e^{-i p y / hbar} dp
# is taken exactly over the cell expansions of f1 (the same transform as the
# two-body term's, at y/2), with f1 = dx sum_{x2} int f dp2; rho1(x_b, x_c)
# uses r = (x_b + x_c)/2, which for odd b + c is a half point where f1 comes
# from the natural cubic spline of Sec. 4.1; rho1 is made Hermitian as
# (rho1 + rho1^H)/2 and its occupations are the eigenvalues of rho1 dx.
# ---------------------------------------------------------------------------

def _sem_f1(o, f):
    """f1[i][j] = dx sum_{i2} sum_{j2} w_{j2} f[i][i2][j][j2]."""
    return o.dx * np.einsum("abcd,d->ac", f, o.w)


def _sem_f1_halfgrid(o, f1):
    """g[k] = f1 at x_0 + k dx/2, k = 0 .. 2 (nx - 1): the grid values and the
    natural-spline values at the half points."""
    nx = o.nx
    eta = o.spline_coeffs(f1, 0)                       # [nu][j]
    half = o.shift_matrix(-0.5 * o.dx) @ eta           # f1 at x_i + dx/2, i = 0 .. nx-1
    g = np.empty((2 * nx - 1, f1.shape[1]))
    g[0::2] = f1
    g[1::2] = half[: nx - 1]
    return g


def sem_rho1_from_f1(o, f1):
    """rho1[b][c] (complex nx x nx, Hermitian) from the reduced Wigner
    function f1[nx][np]."""
    nx = o.nx
    g = _sem_f1_halfgrid(o, f1)
    coef = o.cell_coeffs(g, 1)                          # [k][s l]
    m = np.arange(-(nx - 1), nx)
    B = o.basis_transform(0.5 * o.dx * m)               # int e^{2 i p y / hbar} C_l dp at y = m dx / 2
    rho = np.empty((nx, nx), dtype=np.complex128)
    for b in range(nx):
        for c in range(nx):
            rho[b, c] = np.dot(coef[b + c], np.conj(B[c - b + nx - 1]))
    return 0.5 * (rho + rho.conj().T)


def sem_rho1(o, f):
    """rho1 of the state f."""
    return sem_rho1_from_f1(o, _sem_f1(o, f))


def sem_occupations(o, f=None, f1=None):
    """Eigenvalues of rho1 dx, largest first (from the state f, or from f1)."""
    rho = sem_rho1(o, f) if f1 is None else sem_rho1_from_f1(o, f1)
    return np.sort(np.linalg.eigvalsh(rho * o.dx))[::-1]


SemOracle.f1 = _sem_f1
SemOracle.rho1 = sem_rho1
SemOracle.rho1_from_f1 = sem_rho1_from_f1
SemOracle.occupations = sem_occupations
