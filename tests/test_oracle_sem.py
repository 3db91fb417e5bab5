"""Pins of the non-periodic (spectral-element) oracle against things other
than itself: the paper's closed forms for the exchange and the two-body
operators (Sec. 5.1.1, 5.1.2), Moyal's terminating expansion for a quadratic
potential, the spherical-Bessel form of the oscillatory integrals (Sec. 3.2),
the paper's own check of the zero-padded Hartree potential against a
Gauss-Laguerre quadrature (Sec. 5.1.3), scipy's natural cubic spline, and
exact identities (polynomial reproduction, linearity, exchange symmetry).
"""
import math

import numpy as np
import pytest
from scipy.interpolate import CubicSpline
from scipy.special import roots_genlaguerre, spherical_jn

from oracle import SemOracle
from oracle.sem_ref import osc_integral
from paper_2511_11354_gb300 import inputs


def _sem(nx=21, ncell=2, nq=6, L=20.0, Lp=None, **kw):
    Lp = math.pi * (nx - 1) / L if Lp is None else Lp   # dx = pi hbar / Lp
    base = dict(dt=0.01, vext=inputs.zero_potential(), vee=inputs.zero_potential(), gamma=0.0,
                c_hartree=0.0, c_xc=0.0)
    base.update(kw)
    return inputs.SemProblem(nx=nx, ncell=ncell, nq=nq, L=L, Lp=Lp, **base)


def _grid4(o):
    return np.meshgrid(o.x, o.x, o.p, o.p, indexing="ij")


# ---------------------------------------------------------------------------
# Oscillatory integrals and the cell expansion
# ---------------------------------------------------------------------------

def test_osc_integral_is_a_sum_of_spherical_bessel_functions():
    """T_l = sum_k c_lk P_k (Legendre) and int P_k e^{i z eta} = 2 i^k j_k(z)."""
    z = np.concatenate([np.linspace(-80.0, 80.0, 161), [0.0, 1e-3, -2.5]])
    O = osc_integral(16, z)
    for l in range(16):
        c = np.polynomial.Chebyshev.basis(l).convert(kind=np.polynomial.Legendre).coef
        ref = sum(ck * 2 * (1j ** k) * spherical_jn(k, z) for k, ck in enumerate(c))
        np.testing.assert_allclose(O[l], ref, rtol=0, atol=1e-13)
    # z = 0: int T_l = 2 / (1 - l^2) for even l, 0 for odd l
    O0 = osc_integral(16, np.zeros(1))[:, 0]
    ref0 = [2.0 / (1 - l * l) if l % 2 == 0 else 0.0 for l in range(16)]
    np.testing.assert_allclose(O0.real, ref0, atol=1e-15)


def test_nodes_weights_and_cell_transform():
    prob = _sem(ncell=3, nq=7, Lp=6.0)
    o = SemOracle(prob)
    np.testing.assert_allclose(o.p, prob.p(), rtol=0, atol=1e-15)
    assert np.all(np.diff(o.p) > 0)
    # the weights integrate every cell polynomial of degree < nq exactly
    for deg in range(7):
        exact = (3.0 ** (deg + 1) - (-3.0) ** (deg + 1)) / (deg + 1)
        assert abs(np.dot(o.w, o.p ** deg) - exact) < 1e-12 * max(1.0, abs(exact))
    # the coefficients of T_l in one cell are (0, .., 1, .., 0)
    eta = (o.p - np.repeat(o.centre, 7)) / (0.5 * o.width)
    for l in range(7):
        b = o.cell_coeffs(np.cos(l * np.arccos(np.clip(eta, -1, 1)))[None, :], 1)[0]
        want = np.tile(np.eye(7)[l], 3)
        np.testing.assert_allclose(b, want, atol=1e-14)


# ---------------------------------------------------------------------------
# Closed forms (Sec. 5.1) on the paper's test domain
# ---------------------------------------------------------------------------

def test_xc_closed_form_spectral_elements():
    """Exchange potential V_XC[n] = n on f = pi^-2 exp(-u1^2/2 - 2p1^2)
    exp(-u2^2/2 - 2p2^2), domain [-10, 10]^2 x [-5pi/2, 5pi/2]^2, 101 points
    per axis; the error falls spectrally with the points per cell (the paper
    prints 7e-7 and 6e-12 for 8 and 16 points; this reading's Gauss points
    carry one degree less per cell)."""
    r10, r20 = 1.0, -0.5
    errs = []
    for nq in (6, 10):
        prob = _sem(nx=101, ncell=8, nq=nq, L=20.0, Lp=5 * math.pi, c_xc=1.0, xc_kind=1)
        o = SemOracle(prob)
        X1, X2, P1, P2 = _grid4(o)
        u1, u2 = X1 + r10, X2 + r20
        f = np.pi ** -2 * np.exp(-u1 ** 2 / 2 - 2 * P1 ** 2) * np.exp(-u2 ** 2 / 2 - 2 * P2 ** 2)
        exact = (np.pi ** -2.5 * np.exp(-0.75 * u1 ** 2 - P1 ** 2) * np.exp(-u2 ** 2 / 2 - 2 * P2 ** 2) * np.sin(u1 * P1)
                 + np.pi ** -2.5 * np.exp(-0.75 * u2 ** 2 - P2 ** 2) * np.exp(-u1 ** 2 / 2 - 2 * P1 ** 2) * np.sin(u2 * P2))
        n1, _ = o.marginal(f)
        th = o.theta(f)
        errs.append(np.abs(th - exact).max() / np.abs(exact).max())
        if nq == 10:
            np.testing.assert_allclose(n1, np.exp(-(o.x + r10) ** 2 / 2) / math.sqrt(2 * math.pi), atol=2e-6)
            assert np.abs(th + exact).max() / np.abs(exact).max() > 1.9   # the sign reading
    assert errs[0] < 3e-3 and errs[1] < 2e-5 and errs[1] < errs[0] / 50, errs


def test_two_body_closed_form_spectral_elements():
    """Gaussian pair H_B exp(-r^2/2) on f = pi^-2 exp(-u1^2 - p1^2)
    exp(-u2^2 - p2^2): Theta = sqrt(2) H_B / pi^2 exp(-u1^2 - u2^2 - r^2/4)
    exp(-p1^2 - p2^2 + (p1-p2)^2/4) sin(r (p1-p2)/2)."""
    HB, r10, r20 = 0.7, 0.5, -0.8
    errs = []
    for nq in (6, 10):
        prob = _sem(nx=61, ncell=8, nq=nq, L=12.0, vee=inputs.gaussian_potential(HB, 2.0), gamma=1.0)
        o = SemOracle(prob)
        X1, X2, P1, P2 = _grid4(o)
        u1, u2, r, q = X1 + r10, X2 + r20, X1 - X2, P1 - P2
        f = np.pi ** -2 * np.exp(-u1 ** 2 - P1 ** 2) * np.exp(-u2 ** 2 - P2 ** 2)
        exact = (np.sqrt(2) * HB / np.pi ** 2 * np.exp(-u1 ** 2 - u2 ** 2 - r ** 2 / 4)
                 * np.exp(-P1 ** 2 - P2 ** 2 + q ** 2 / 4) * np.sin(r * q / 2))
        th = o.theta_two_body(f)
        errs.append(np.abs(th - exact).max() / np.abs(exact).max())
        if nq == 10:
            assert np.abs(th + exact).max() / np.abs(exact).max() > 1.9
    assert errs[0] < 5e-3 and errs[1] < 1e-6 and errs[1] < errs[0] / 100, errs


def test_moyal_quadratic_potential_spectral_elements():
    """For V = omega^2 x^2 / 2 the operator is exactly V'(x) d_p f (Moyal);
    checked on a packet well inside the box."""
    om = 1.3
    prob = _sem(nx=51, ncell=8, nq=14, L=10.0, Lp=5 * math.pi)
    o = SemOracle(prob)
    X1, X2, P1, P2 = _grid4(o)
    g = np.exp(-2 * (X1 - 0.3) ** 2 - (P1 + 0.4) ** 2 / 2) * np.exp(-X2 ** 2 - P2 ** 2)
    dp1 = -(P1 + 0.4) * g
    exact = om * om * X1 * dp1
    U = 0.5 * om * om * o.x ** 2
    th = o.theta_one_body(g, U, np.zeros_like(U))
    err = np.abs(th - exact).max() / np.abs(exact).max()
    assert err < 2e-8, err


# ---------------------------------------------------------------------------
# Zero-padded Hartree (Sec. 3.2.1 remark; the paper's check in Sec. 5.1.3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("eps", [1.0, 0.25])
def test_zero_padded_hartree(eps):
    """n = exp(-r^2): V_H(r) = (1/2) int_0^inf [W(r - sqrt s) + W(r + sqrt s)]
    s^{-1/2} e^{-s} ds by generalised Gauss-Laguerre quadrature (alpha = -1/2);
    and the 3-fold padded FFT equals the direct linear sum exactly."""
    W = inputs.soft_coulomb(eps)
    prob = _sem(nx=161, L=16.0, vee=W, c_hartree=1.0)
    o = SemOracle(prob)
    n = np.exp(-o.x ** 2)
    vh = o.hartree(n)
    direct = o.dx * np.array([sum(W(xm - xq) * nq for xq, nq in zip(o.x, n)) for xm in o.x])
    np.testing.assert_allclose(vh, direct, rtol=1e-13, atol=0)
    s, ws = roots_genlaguerre(200, -0.5)
    ref = np.array([0.5 * np.sum(ws * (np.array([W(xm - math.sqrt(v)) + W(xm + math.sqrt(v)) for v in s])))
                    for xm in o.x])
    tol = 1e-9 if eps == 1.0 else 1e-4
    assert np.abs(vh - ref).max() / np.abs(ref).max() < tol
    # unpadded (cyclic of length nx - 1) is visibly wrong near the ends
    k = np.array([W(v * o.dx) for v in np.rint(np.fft.fftfreq(o.nx - 1) * (o.nx - 1))])
    wrap = o.dx * np.real(np.fft.ifft(np.fft.fft(k) * np.fft.fft(n[:-1])))
    assert np.abs(wrap - ref[:-1]).max() / np.abs(ref).max() > 1e-3


# ---------------------------------------------------------------------------
# Natural cubic spline shift (Sec. 4.1, A_nat)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nx", [9, 24])
def test_natural_spline_matches_scipy(nx):
    prob = _sem(nx=nx, L=10.0)
    o = SemOracle(prob)
    rng = np.random.default_rng(nx)
    f = rng.standard_normal(nx)
    eta = o.spline_coeffs(f, 0)
    cs = CubicSpline(o.x, f, bc_type="natural")
    for s in (0.0, 0.37, -1.9, 3.3 * o.dx, -0.5 * o.dx):
        pts = o.x - s
        inside = (pts >= o.x[0]) & (pts <= o.x[-1])
        val = o.shift_matrix(s) @ eta
        np.testing.assert_allclose(val[inside], cs(pts[inside]), rtol=0, atol=1e-12 * np.abs(f).max())
    # zero shift reproduces the data; far shifts see zero inflow
    np.testing.assert_allclose(o.shift_matrix(0.0) @ eta, f, atol=1e-13)
    far = o.shift_matrix(prob.L + 4 * o.dx)
    assert np.all(far == 0.0)


def test_advection_identity_linear_and_commuting():
    prob = _sem(nx=13, ncell=2, nq=3, L=12.0, Lp=6.0, dt=0.3)
    o = SemOracle(prob)
    X1, X2, P1, P2 = _grid4(o)
    # linear functions of x are reproduced wherever the departure point stays in the box
    f = 0.5 + 0.2 * X1 - 0.1 * X2
    g = o.advect(f)
    ref = 0.5 + 0.2 * (X1 - prob.dt * P1) - 0.1 * (X2 - prob.dt * P2)
    inside = (np.abs(X1 - prob.dt * P1) <= 6.0) & (np.abs(X2 - prob.dt * P2) <= 6.0)
    np.testing.assert_allclose(g[inside], ref[inside], atol=1e-12)
    prob0 = _sem(nx=13, ncell=2, nq=3, L=12.0, Lp=6.0, dt=0.0)
    r = np.random.default_rng(0).standard_normal(f.shape)
    np.testing.assert_allclose(SemOracle(prob0).advect(r), r, atol=1e-13)


# ---------------------------------------------------------------------------
# Step identities
# ---------------------------------------------------------------------------

def test_step_linear_without_mean_field_and_exchange_symmetric():
    prob = _sem(nx=15, ncell=2, nq=4, L=14.0, Lp=math.pi * 14 / 14.0, dt=0.05,
                vext=lambda x: 0.1 * x * x, vee=inputs.soft_coulomb(1.0), gamma=1.0)
    o = SemOracle(prob)
    rng = np.random.default_rng(3)
    a = rng.standard_normal((15, 15, 8, 8))
    b = rng.standard_normal((15, 15, 8, 8))
    lhs = o.step(2.0 * a - 0.5 * b, 2)
    rhs = 2.0 * o.step(a, 2) - 0.5 * o.step(b, 2)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()
    s = 0.5 * (a + a.transpose(1, 0, 3, 2))
    prob2 = _sem(nx=15, ncell=2, nq=4, L=14.0, Lp=math.pi, dt=0.05, vext=lambda x: 0.1 * x * x,
                 vee=inputs.soft_coulomb(1.0), gamma=1.0, c_hartree=1.0, c_xc=1.0, xc_kind=2)
    g = SemOracle(prob2).step(np.abs(s), 3)
    assert np.abs(g - g.transpose(1, 0, 3, 2)).max() < 1e-13 * np.abs(g).max()


def test_correlated_state_and_observables():
    prob, f = inputs.workload_correlated(nx=31, ncell=8, nq=12)
    o = SemOracle(prob)
    ob = o.observables(f)
    # without the correlation factor the state is a product of two unit-mass
    # mixtures: mass 1, n1 the mixture's density
    x, p = o.x, o.p
    f1 = sum(np.exp(-0.5 * (x[:, None] - c) ** 2 - 2 * p[None, :] ** 2) for c in (-2.0, 2.0)) / (2 * math.pi)
    fp = np.einsum("ac,bd->abcd", f1, f1)
    op = o.observables(fp)
    assert abs(op["mass"] - 1.0) < 1e-6
    dens = sum(np.exp(-0.5 * (x - c) ** 2) for c in (-2.0, 2.0)) / (2 * math.sqrt(2 * math.pi))
    np.testing.assert_allclose(op["n1"], dens, atol=1e-6)
    # purity of the 50/50 mixture of two Gaussian pure states 4 apart:
    # (1 + |<1|2>|^2) / 2 with |<1|2>|^2 = e^-4
    assert abs(op["purity"] - 0.5 * (1.0 + math.exp(-4.0))) < 1e-4   # dx = 1 limits the x sum of f1^2
    # the correlation factor vanishes on the diagonal and removes mass
    assert np.all(f[np.arange(31), np.arange(31)] == 0.0)
    assert 0.5 < ob["mass"] < 1.0
    # kinetic energy of the product state: 2 x <p^2>/2 with <p^2> = 1/4
    prob0 = inputs.SemProblem(nx=31, ncell=8, nq=12, L=prob.L, Lp=prob.Lp, dt=0.01, vext=inputs.zero_potential(),
                              vee=inputs.zero_potential(), gamma=0.0, c_hartree=0.0)
    assert abs(SemOracle(prob0).observables(fp)["energy"] - 0.25) < 1e-5


# ---------------------------------------------------------------------------
# Occupation numbers of the one-body density matrix (appendix on the
# correlation entropy; strongly correlated example)
# ---------------------------------------------------------------------------

def _pure(o, x0, p0):
    """Wigner function of a unit-width Gaussian pure state (mass 1)."""
    return (1 / math.pi) * np.exp(-0.5 * (o.x[:, None] - x0) ** 2 - 2 * (o.p[None, :] - p0) ** 2)


def test_occupations_of_a_pure_state_and_of_a_mixture():
    """A pure state has one occupation 1 (rho1 = psi psi*); the 50/50
    mixture of two unit-width Gaussians 4 apart has (1 +- e^-2)/2 (their
    overlap is e^-2); the rest vanish as the mesh is refined."""
    from oracle.rdm_ref import correlation_entropy
    e = math.exp(-2.0)
    errs = []
    for nx in (61, 121):
        prob = inputs.sem_correlated_problem("I", nx=nx, ncell=8, nq=12, L=30.0)
        o = SemOracle(prob)
        occ = o.occupations(f1=_pure(o, -1.0, 0.3))
        assert abs(occ[0] - 1.0) < 1e-4 and occ[1] < 3e-4, occ[:3]
        mix = 0.5 * (_pure(o, -2.0, 0.0) + _pure(o, 2.0, 0.0))
        occ = o.occupations(f1=mix)
        errs.append(max(abs(occ[0] - 0.5 * (1 + e)), abs(occ[1] - 0.5 * (1 - e))))
        s = correlation_entropy(occ)
        exact = sum(v * math.log(v) for v in (0.5 * (1 + e), 0.5 * (1 - e)))
        assert abs(s - exact) < 5e-3, (s, exact)
        # rho1 is Hermitian before the symmetrisation up to rounding
        assert abs(occ.sum() - np.dot(o.w, mix.sum(axis=0)) * o.dx) < 1e-10
    assert errs[1] < 1e-5 and errs[1] < errs[0] / 5, errs


def test_reduced_wigner_function_of_the_state():
    prob, f = inputs.workload_correlated("IV", nx=15, ncell=2, nq=4, L=30.0)
    o = SemOracle(prob)
    f1 = o.f1(f)
    ref = np.array([[o.dx * sum(o.w[d] * f[a, b, c, d] for b in range(15) for d in range(8)) for c in range(8)]
                    for a in range(15)])
    np.testing.assert_allclose(f1, ref, rtol=1e-13, atol=1e-16)
    # the trace of rho1 dx is the mass of f1
    occ = o.occupations(f)
    assert abs(occ.sum() - o.dx * np.dot(f1.sum(axis=0), o.w)) < 1e-12 * abs(occ.sum())
