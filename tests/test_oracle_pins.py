"""Pins of the FP64 oracle against things other than itself.

Each test below checks one oracle function against a value fixed by the
paper or by mathematics: the paper's closed forms for the pseudo-difference
operators (Sec. 5.1), Moyal's terminating expansions for polynomial
potentials, the FFT form of the periodic operator that the paper points to
(Sec. 3.1), scipy's periodic cubic interpolating spline, exact discrete
identities, and a brute-force two-particle Schroedinger evolution.
"""
import math

import numpy as np
import pytest
from scipy.interpolate import make_interp_spline

import oracle
from paper_2511_11354_gb300 import inputs


def _grid4(prob):
    x = prob.x()
    p = prob.p()
    X1, X2, P1, P2 = np.meshgrid(x, x, p, p, indexing="ij")
    return X1, X2, P1, P2


# ---------------------------------------------------------------------------
# Closed forms, Sec. 5.1
# ---------------------------------------------------------------------------

def test_xc_closed_form():
    """Sec. 5.1.1: f = pi^-2 exp(-u1^2/2 - 2 p1^2) exp(-u2^2/2 - 2 p2^2) with
    the exchange potential V_XC[n] = n gives
    Theta = pi^-5/2 exp(-3u1^2/4 - p1^2) exp(-u2^2/2 - 2 p2^2) sin(u1 p1) + (1<->2)."""
    r10, r20 = 1.0, -0.5
    prob = inputs.Problem(nx=48, nk=48, L=20.0, dt=0.01, vext=inputs.zero_potential(),
                          vee=inputs.zero_potential(), gamma=0.0, c_hartree=0.0, c_xc=1.0, xc_kind=1)
    X1, X2, P1, P2 = _grid4(prob)
    u1, u2 = X1 + r10, X2 + r20
    f = np.pi ** -2 * np.exp(-u1 ** 2 / 2 - 2 * P1 ** 2) * np.exp(-u2 ** 2 / 2 - 2 * P2 ** 2)
    exact = (np.pi ** -2.5 * np.exp(-0.75 * u1 ** 2 - P1 ** 2) * np.exp(-u2 ** 2 / 2 - 2 * P2 ** 2) * np.sin(u1 * P1)
             + np.pi ** -2.5 * np.exp(-0.75 * u2 ** 2 - P2 ** 2) * np.exp(-u1 ** 2 / 2 - 2 * P1 ** 2) * np.sin(u2 * P2))
    o = oracle.Oracle(prob)
    # the densities of f are exactly the Gaussians of the closed form
    n1, n2 = o.marginals(f)
    x = prob.x()
    np.testing.assert_allclose(n1, np.exp(-(x + r10) ** 2 / 2) / np.sqrt(2 * np.pi), atol=1e-13)
    np.testing.assert_allclose(n2, np.exp(-(x + r20) ** 2 / 2) / np.sqrt(2 * np.pi), atol=1e-13)
    th = o.theta(f)
    err = np.abs(th - exact).max() / np.abs(exact).max()
    assert err < 1e-9, err


def test_two_body_closed_form():
    """Sec. 5.1.2: Gaussian pair interaction H_B exp(-r^2/2) on
    f = pi^-2 exp(-u1^2 - p1^2) exp(-u2^2 - p2^2) gives
    Theta = sqrt(2) H_B / pi^2 exp(-u1^2 - u2^2 - r^2/4) exp(-p1^2 - p2^2 + (p1-p2)^2/4) sin(r (p1-p2)/2)."""
    HB, r10, r20 = 0.7, 0.5, -0.8
    prob = inputs.Problem(nx=16, nk=56, L=16.0, dt=0.01, vext=inputs.zero_potential(),
                          vee=inputs.gaussian_potential(HB, 2.0), gamma=1.0, c_hartree=0.0)
    X1, X2, P1, P2 = _grid4(prob)
    u1, u2, r, q = X1 + r10, X2 + r20, X1 - X2, P1 - P2
    f = np.pi ** -2 * np.exp(-u1 ** 2 - P1 ** 2) * np.exp(-u2 ** 2 - P2 ** 2)
    exact = (np.sqrt(2) * HB / np.pi ** 2 * np.exp(-u1 ** 2 - u2 ** 2 - r ** 2 / 4)
             * np.exp(-P1 ** 2 - P2 ** 2 + q ** 2 / 4) * np.sin(r * q / 2))
    o = oracle.Oracle(prob)
    U0 = np.zeros((prob.nx, 2 * prob.nk))
    th = o.theta_with(f, U0, U0, terms=4)
    err = np.abs(th - exact).max() / np.abs(exact).max()
    assert err < 1e-10, err
    # a sign error in the reading would flip the whole term
    assert np.abs(th + exact).max() / np.abs(exact).max() > 1.0


@pytest.mark.parametrize("kind", ["harmonic", "quartic"])
def test_moyal_polynomial(kind):
    """Moyal expansion terminates for polynomial V:
    Theta f = V' d_p f - (hbar^2/24) V''' d_p^3 f  (exact for cubic/quartic).
    Checked away from the fold of the periodised polynomial."""
    prob = inputs.Problem(nx=24, nk=64, L=12.0, dt=0.01,
                          vext=(inputs.harmonic(1.3) if kind == "harmonic" else (lambda x: 0.25 * x ** 4)),
                          vee=inputs.zero_potential(), gamma=0.0, c_hartree=0.0)
    X1, X2, P1, P2 = _grid4(prob)
    s2 = 0.25  # x-width^2 of the Gaussian; p-width^2 = 1/(4 s2)
    a, b = 1.0 / (2 * s2), 2 * s2
    x0, p0 = 0.3, -0.4
    g = np.exp(-a * (X1 - x0) ** 2 - b * (P1 - p0) ** 2) * np.exp(-a * X2 ** 2 - b * P2 ** 2)
    dp1 = -2 * b * (P1 - p0) * g
    dp3 = (-(2 * b) ** 3 * (P1 - p0) ** 3 + 3 * (2 * b) ** 2 * (P1 - p0)) * g
    if kind == "harmonic":
        V1, V3 = 1.3 ** 2 * X1, 0.0 * X1
    else:
        V1, V3 = X1 ** 3, 6 * X1
    exact = V1 * dp1 - (prob.hbar ** 2 / 24) * V3 * dp3
    o = oracle.Oracle(prob)
    U1 = o.potential_fine(None)
    th = o.theta_with(g, U1, np.zeros_like(U1), terms=1)
    mask = np.abs(X1) <= 2.0
    err = np.abs(th - exact)[mask].max() / np.abs(exact).max()
    assert err < 1e-9, err


# ---------------------------------------------------------------------------
# FFT form of the periodic operator (Sec. 3.1: accelerated by FFTs when f
# vanishes outside the momentum window)
# ---------------------------------------------------------------------------

def _theta_fft(prob, f, U1, U2, u12):
    """Theta by zero padding to M = 2 nk, multiplying the 2-D DFT by the
    symbol (i/hbar)[U(x + l h') - U(x - l h')] per axis (and along l1 - l2
    for the pair term), inverse DFT, crop."""
    nx, nk, M = prob.nx, prob.nk, 2 * prob.nk
    l = np.arange(M)
    sym = lambda u: (1j / prob.hbar) * (u[..., l] - u[..., (-l) % M])
    s1, s2, s12 = sym(U1), sym(U2), sym(u12)
    out = np.empty_like(f)
    k1, k2 = np.meshgrid(l, l, indexing="ij")
    for i1 in range(nx):
        for i2 in range(nx):
            F = np.zeros((M, M))
            F[:nk, :nk] = f[i1, i2]
            Fh = np.fft.fft2(F)
            d = (i1 - i2) % nx
            S = s1[i1][k1] + s2[i2][k2] + s12[d][(k1 - k2) % M]
            out[i1, i2] = np.real(np.fft.ifft2(S * Fh))[:nk, :nk]
    return out


def test_theta_fft_form():
    prob, f = inputs.workload_small(nx=8, nk=12)
    o = oracle.Oracle(prob)
    n1, n2 = o.marginals(f)
    U1, U2 = o.potential_fine(n1), o.potential_fine(n2)
    M = 2 * prob.nk
    u12 = np.array([[prob.gamma * prob.vee(float(inputs.fold(d * prob.dx + l * prob.L / M, prob.L)))
                     for l in range(M)] for d in range(prob.nx)])
    ref = _theta_fft(prob, f, U1, U2, u12)
    th = o.theta(f)
    assert np.abs(th - ref).max() / np.abs(ref).max() < 1e-13


def test_hartree_quadrature():
    """V_H(y) = gamma dx sum_q W(fold(y - x_q)) n(x_q) at the fine points."""
    prob, f = inputs.workload_small(nx=8, nk=6)
    o = oracle.Oracle(prob)
    n = np.linspace(0.1, 0.9, prob.nx) ** 2
    U = o.potential_fine(n)
    M, x = 2 * prob.nk, prob.x()
    for i in range(prob.nx):
        for l in range(M):
            y = x[i] + l * prob.L / M
            vh = prob.gamma * prob.dx * sum(prob.vee(float(inputs.fold(y - x[q], prob.L))) * n[q]
                                            for q in range(prob.nx))
            assert abs(U[i, l] - (prob.vext(float(inputs.fold(y, prob.L))) + vh)) < 1e-13


def test_theta_antisymmetry_and_mass_leak():
    """Theta is skew per X: sum_P f Theta f = 0.  On the padded lattice the
    symbol vanishes at zero frequency, so the window mass of Theta f equals
    minus the mass it sends outside the window."""
    prob, f = inputs.workload_small(nx=8, nk=12)
    o = oracle.Oracle(prob)
    th = o.theta(f)
    s = np.einsum("abcd,abcd->ab", f, th)
    assert np.abs(s).max() < 1e-15 * np.abs(f).max() * np.abs(th).max() * prob.nk ** 2
    # leaked mass, from the uncropped padded operator
    n1, n2 = o.marginals(f)
    U1, U2 = o.potential_fine(n1), o.potential_fine(n2)
    nx, nk, M = prob.nx, prob.nk, 2 * prob.nk
    l = np.arange(M)
    u12 = np.array([[prob.gamma * prob.vee(float(inputs.fold(d * prob.dx + ll * prob.L / M, prob.L)))
                     for ll in l] for d in range(nx)])
    sym = lambda u: (1j / prob.hbar) * (u[..., l] - u[..., (-l) % M])
    k1, k2 = np.meshgrid(l, l, indexing="ij")
    for i1, i2 in [(0, 0), (3, 5), (7, 2)]:
        F = np.zeros((M, M))
        F[:nk, :nk] = f[i1, i2]
        S = sym(U1)[i1][k1] + sym(U2)[i2][k2] + sym(u12)[(i1 - i2) % nx][(k1 - k2) % M]
        full = np.real(np.fft.ifft2(S * np.fft.fft2(F)))
        outside = full.sum() - full[:nk, :nk].sum()
        assert abs(th[i1, i2].sum() + outside) < 1e-12 * np.abs(full).sum()


# ---------------------------------------------------------------------------
# Periodic cubic spline (Sec. 4.1) against scipy's periodic interpolant
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nx", [5, 8, 17, 32])
def test_spline_shift_matches_scipy(nx):
    L = 7.0
    prob = inputs.Problem(nx=nx, nk=4, L=L, dt=0.01, vext=inputs.zero_potential(),
                          vee=inputs.zero_potential(), gamma=0.0, c_hartree=0.0)
    o = oracle.Oracle(prob)
    rng = np.random.default_rng(nx)
    y = rng.standard_normal(nx)
    x = prob.x()
    xs = np.append(x, x[0] + L)
    spl = make_interp_spline(xs, np.append(y, y[0]), k=3, bc_type="periodic")
    for shift in [0.0, 0.37 * prob.dx, -1.6 * prob.dx, 3.25 * prob.dx, 2.0 * L + 0.1]:
        got = o.shift_line(y, shift)
        t = x - shift
        t = x[0] + np.mod(t - x[0], L)
        np.testing.assert_allclose(got, spl(t), rtol=0, atol=1e-13)


def test_spline_integer_shift_is_roll_and_fourier_multiplier():
    nx, L = 16, 10.0
    prob = inputs.Problem(nx=nx, nk=4, L=L, dt=0.01, vext=inputs.zero_potential(),
                          vee=inputs.zero_potential(), gamma=0.0, c_hartree=0.0)
    o = oracle.Oracle(prob)
    y = np.random.default_rng(1).standard_normal(nx)
    np.testing.assert_allclose(o.shift_line(y, 3 * prob.dx), np.roll(y, 3), atol=1e-13)
    np.testing.assert_allclose(o.shift_line(y, 0.0), y, atol=1e-14)
    # e^{i w j} is an eigenvector of the shift: closed-form multiplier
    j = np.arange(nx)
    for q in [1, 3, 5]:
        w = 2 * np.pi * q / nx
        s = 0.3
        th = (-s) - math.floor(-s)
        k0 = math.floor(-s)
        b = [(1 - th) ** 3 / 6, (3 * th ** 3 - 6 * th ** 2 + 4) / 6, (-3 * th ** 3 + 3 * th ** 2 + 3 * th + 1) / 6, th ** 3 / 6]
        mu = np.exp(1j * w * k0) * sum(b[a + 1] * np.exp(1j * w * a) for a in range(-1, 3)) / ((4 + 2 * np.cos(w)) / 6)
        re = o.shift_line(np.cos(w * j), s * prob.dx)
        im = o.shift_line(np.sin(w * j), s * prob.dx)
        np.testing.assert_allclose(re + 1j * im, mu * np.exp(1j * w * j), atol=1e-13)


# ---------------------------------------------------------------------------
# Step-level identities
# ---------------------------------------------------------------------------

def test_free_streaming_integer_roll():
    """No potential: the step is the shift; with tau dp/(m dx) = 1 it is an
    exact roll of every (p1, p2) plane by the momentum index."""
    L, nx, nk = 2 * np.pi, 8, 6
    tau = L * L / (np.pi * nx)
    prob = inputs.Problem(nx=nx, nk=nk, L=L, dt=tau, vext=inputs.zero_potential(),
                          vee=inputs.zero_potential(), gamma=0.0, c_hartree=0.0)
    o = oracle.Oracle(prob)
    f = np.random.default_rng(3).standard_normal((nx, nx, nk, nk))
    g = o.step(f, 1)
    for a in range(nk):
        for b in range(nk):
            ref = np.roll(np.roll(f[:, :, a, b], a - nk // 2, axis=0), b - nk // 2, axis=1)
            np.testing.assert_allclose(g[:, :, a, b], ref, atol=1e-12)


def test_free_streaming_converges_at_fourth_order():
    """No potential, a non-integer shift: after a few steps the state is the
    initial one moved along its characteristics, f(x - t p/m, p) on the
    torus; the cubic-spline error falls as dx^4 (ratio near 16 per halving)."""
    L, nk, steps = 10.0, 4, 5
    errs = []
    for nx in (24, 48):
        prob = inputs.Problem(nx=nx, nk=nk, L=L, dt=0.37, vext=inputs.zero_potential(),
                              vee=inputs.zero_potential(), gamma=0.0, c_hartree=0.0)
        o = oracle.Oracle(prob)
        x, p = prob.x(), prob.p()
        k = 2 * np.pi / L
        prof = lambda y: np.exp(np.cos(k * y) + 0.5 * np.sin(2 * k * y))
        f = np.einsum("a,b,c,d->abcd", prof(x), prof(x - 1.0), np.ones(nk), np.ones(nk))
        g = o.step(f, steps)
        t = steps * prob.dt
        X1, X2, P1, P2 = np.meshgrid(x, x, p, p, indexing="ij")
        exact = prof(X1 - t * P1) * prof(X2 - 1.0 - t * P2)
        errs.append(np.abs(g - exact).max() / np.abs(exact).max())
    assert errs[0] < 1e-2 and 10.0 < errs[0] / errs[1] < 24.0, errs


def test_exchange_symmetry_and_parity_preserved():
    prob, f = inputs.workload_small(nx=8, nk=10)
    o = oracle.Oracle(prob)
    g = o.step(f, 3)
    assert np.abs(g - g.transpose(1, 0, 3, 2)).max() < 1e-14 * np.abs(g).max()
    # torus parity sector f(x + L/2, p_n) = (-1)^n f(x, p_n) is invariant
    nx, nk = prob.nx, prob.nk
    sgn = (-1.0) ** np.arange(nk)
    h = f.copy()
    h[nx // 2:] = sgn[None, None, :, None] * f[:nx // 2]
    h[:, nx // 2:] = sgn[None, None, None, :] * h[:, :nx // 2]
    h = 0.5 * (h + h.transpose(1, 0, 3, 2))
    hs = o.step(h, 2)
    half = hs[nx // 2:] - sgn[None, None, :, None] * hs[:nx // 2]
    assert np.abs(half).max() < 1e-13 * np.abs(hs).max()


def test_step_linear_without_mean_field():
    prob, f = inputs.workload_small(nx=8, nk=8)
    prob.c_hartree = 0.0
    o = oracle.Oracle(prob)
    g = np.random.default_rng(5).standard_normal(f.shape) * 0.01
    lhs = o.step(2.0 * f - 3.0 * g, 2)
    rhs = 2.0 * o.step(f, 2) - 3.0 * o.step(g, 2)
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(lhs).max()


def test_advection_conserves_mass_exactly():
    prob, f = inputs.workload_small(nx=12, nk=8)
    o = oracle.Oracle(prob)
    a = o.advect(f)
    m0 = f.sum(axis=(0, 1))
    m1 = a.sum(axis=(0, 1))
    np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-13 * np.abs(m0).max())


def test_observables_definitions():
    prob, f = inputs.workload_small(nx=8, nk=8)
    o = oracle.Oracle(prob)
    ob = o.observables(f)
    dV = prob.dx ** 2 * prob.dp ** 2
    assert abs(ob["mass"] - 1.0) < 1e-13
    assert abs(ob["l2norm"] - np.sqrt((f * f).sum() * dV)) < 1e-14
    f1 = f.sum(axis=(1, 3)) * prob.dx * prob.dp
    pur = 2 * np.pi * prob.hbar * (f1 ** 2).sum() * prob.dx * prob.dp
    assert abs(ob["purity"] - pur) < 1e-13 and abs(ob["entropy_lin"] - (1 - pur)) < 1e-13
    np.testing.assert_allclose(ob["n12"], f.sum(axis=(2, 3)) * prob.dp ** 2, atol=1e-15)
    np.testing.assert_allclose(ob["n1"], f.sum(axis=(1, 2, 3)) * prob.dx * prob.dp ** 2, atol=1e-15)
    # pure single Gaussian packet per particle: purity of rho1 is 1
    x, p = prob.x(), prob.p()
    big = inputs.Problem(nx=32, nk=48, L=20.0, dt=0.01, vext=inputs.zero_potential(),
                         vee=inputs.zero_potential(), gamma=0.0, c_hartree=0.0)
    x, p = big.x(), big.p()
    g1 = inputs.gaussian_1body(x[:, None], p[None, :], 0.0, 0.0, 1.0, 1.0, big.L)
    g = np.einsum("ac,bd->abcd", g1, g1)
    ob = oracle.Oracle(big).observables(g)
    assert abs(ob["purity"] - 1.0) < 1e-8 and abs(ob["mass"] - 1.0) < 1e-8


def test_literal_double_well_blows_up_capped_does_not():
    """Reading of the double-well workload: the uncapped well makes the
    explicit step unstable (tau * max|dU| ~ 8), the capped one does not."""
    pl, fl = inputs.workload_dwell(nx=16, nk=16, literal=True)
    pc, fc = inputs.workload_dwell(nx=16, nk=16, literal=False)
    gl = oracle.Oracle(pl).step(fl, 12)
    gc = oracle.Oracle(pc).step(fc, 12)
    assert not np.isfinite(gl).all() or np.abs(gl).max() > 1e3 * np.abs(fl).max()
    assert np.abs(gc).max() < 2.0 * np.abs(fc).max()
