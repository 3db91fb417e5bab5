"""Pins of the oracle's energy, pair-kernel Hartree potential, stage-wise
potential (Lawson reading R8) and of its whole step under a harmonic
potential, each against mathematics rather than a restatement of the oracle:

* energy: product Gaussian packets with a cosine well and a Gaussian pair
  kernel have closed-form kinetic, external, pair and Hartree energies;
* Hartree: a Gaussian kernel convolved with a Gaussian density is a
  Gaussian;
* R8: the Lawson predictor-corrector (Sec. 4.1) is second order in tau only
  if each pseudo-difference operator takes its mean-field potential from its
  own stage input; with exact (integer-cell) shifts the time error is the
  only error, and a step that freezes U^n for the corrector is first order;
* harmonic rotation: for V = x^2/2 the Wigner flow is the classical rotation
  of phase space, reached at order tau^2 and dx^4 (cubic spline).

Each pin is also run on a copy of the oracle with a planted mistake (built by
``oracle.variant``) to show that it fails there.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2511_11354_gb300 import inputs

# ---------------------------------------------------------------------------
# Energy of product Gaussian packets
# ---------------------------------------------------------------------------

SIG = 1.5            # spatial width of both packets
XA, PA = -1.5, 0.4   # particle 1
XB, PB = 2.0, -0.3   # particle 2
AMP = 0.7            # external potential AMP cos(2 pi x / L)
HW, W2 = 1.3, 3.0    # pair kernel HW exp(-r^2 / W2)
GAMMA, MASS = 0.8, 1.3


def _energy_problem(vext_on, gamma, c_h):
    L = 30.0
    return inputs.Problem(nx=40, nk=64, L=L, dt=0.01, mass=MASS,
                          vext=inputs.cos_potential(AMP, L) if vext_on else inputs.zero_potential(),
                          vee=inputs.gaussian_potential(HW, W2), gamma=gamma, c_hartree=c_h)


def _product_state(prob):
    x, p = prob.x(), prob.p()
    ga = inputs.gaussian_1body(x[:, None], p[None, :], XA, PA, SIG, prob.hbar, prob.L)
    gb = inputs.gaussian_1body(x[:, None], p[None, :], XB, PB, SIG, prob.hbar, prob.L)
    return np.ascontiguousarray(np.einsum("ac,bd->abcd", ga, gb))


def _energy_exact(prob, vext_on, gamma, c_h):
    """Closed forms for G(x, p) = exp(-(x-x0)^2/(2 s^2) - 2 s^2 (p-p0)^2/hbar^2)/(pi hbar):
    <p^2> = p0^2 + hbar^2/(4 s^2);  <cos(k x)> = cos(k x0) exp(-k^2 s^2/2);
    for r ~ N(mu, v): <exp(-r^2/c)> = (1 + 2 v/c)^(-1/2) exp(-mu^2/(c + 2 v))."""
    hb = prob.hbar
    kin = sum((p0 ** 2 + hb ** 2 / (4 * SIG ** 2)) / (2 * MASS) for p0 in (PA, PB))
    k = 2 * math.pi / prob.L
    ext = sum(AMP * math.cos(k * x0) * math.exp(-k * k * SIG ** 2 / 2) for x0 in (XA, XB)) if vext_on else 0.0
    v = 2 * SIG ** 2
    pair = gamma * HW * math.exp(-(XA - XB) ** 2 / (W2 + 2 * v)) / math.sqrt(1 + 2 * v / W2)
    # Hartree: (c_H/2) gamma sum_particles <W(x - y)>, x, y independent draws of the same density
    hart = c_h * gamma * HW / math.sqrt(1 + 2 * v / W2)
    return kin + ext + pair + hart


ENERGY_CASES = [(False, 0.0, 0.0), (True, 0.0, 0.0), (True, GAMMA, 0.0), (True, GAMMA, 1.0)]


def _energy_errors(lib=None):
    errs = []
    for vext_on, gamma, c_h in ENERGY_CASES:
        prob = _energy_problem(vext_on, gamma, c_h)
        f = _product_state(prob)
        ob = oracle.Oracle(prob, lib=lib).observables(f)
        errs.append(abs(ob["energy"] - _energy_exact(prob, vext_on, gamma, c_h)))
    return errs


def test_energy_closed_form():
    """Kinetic, then + external, then + pair, then + Hartree energy, each to
    5e-12 (the oracle's sums run over 6.6M points in one accumulator)."""
    prob = _energy_problem(True, GAMMA, 1.0)
    f = _product_state(prob)
    ob = oracle.Oracle(prob).observables(f)
    assert abs(ob["mass"] - 1.0) < 5e-12
    errs = _energy_errors()
    assert max(errs) < 5e-12, errs


@pytest.mark.parametrize("name,old,new", [
    ("hartree_energy_factor", "eh += 0.5 * P->c_h * fac", "eh += P->c_h * fac"),
    ("pair_energy_dropped", "+ P->gamma * P->w_shift[d * M + 0];", "+ 0.0 * P->w_shift[d * M + 0];"),
    ("kinetic_mass", "/ (2 * P->mass) * dV", "/ 2 * dV"),
    ("external_energy_one_particle", "P->vext_grid[i1] + P->vext_grid[i2]", "P->vext_grid[i1] + P->vext_grid[i1]"),
])
def test_energy_pin_catches_planted_mistakes(name, old, new):
    errs = _energy_errors(oracle.variant(name, [(old, new)]))
    assert max(errs) > 1e-3, (name, errs)


# ---------------------------------------------------------------------------
# Pair-kernel Hartree potential (reading R6)
# ---------------------------------------------------------------------------

def _hartree_error(lib=None):
    """U = c_H gamma dx sum_q W(fold(y - x_q)) n(x_q) at the fine points
    y = x_i + l h' against the Gaussian convolution
    H (1 + 2 a^2/c)^(-1/2) exp(-(y - c0)^2/(c + 2 a^2)) for W = H exp(-r^2/c),
    n = N(c0, a^2); the box is wide enough for the periodic images to vanish."""
    L, H, c, a, c0, gamma, c_h = 30.0, 1.3, 1.62, 1.1, 1.3, 0.8, 0.75
    prob = inputs.Problem(nx=64, nk=8, L=L, dt=0.01, vext=inputs.zero_potential(),
                          vee=inputs.gaussian_potential(H, c), gamma=gamma, c_hartree=c_h)
    x = prob.x()
    n = np.exp(-(x - c0) ** 2 / (2 * a * a)) / (a * math.sqrt(2 * math.pi))
    U = oracle.Oracle(prob, lib=lib).potential_fine(n)
    y = x[:, None] + np.arange(2 * prob.nk)[None, :] * prob.L / (2 * prob.nk)
    u = inputs.fold(y - c0, L)
    exact = c_h * gamma * H / math.sqrt(1 + 2 * a * a / c) * np.exp(-u * u / (c + 2 * a * a))
    return np.abs(U - exact).max() / np.abs(exact).max()


def test_pair_hartree_closed_form():
    err = _hartree_error()
    assert err < 1e-12, err


@pytest.mark.parametrize("name,new", [
    ("hartree_dropped_dx", "u += P->c_h * P->gamma * vh;"),
    ("hartree_flipped_sign", "u -= P->c_h * P->gamma * P->dx * vh;"),
])
def test_hartree_pin_catches_planted_mistakes(name, new):
    lib = oracle.variant(name, [("u += P->c_h * P->gamma * P->dx * vh;", new)])
    assert _hartree_error(lib) > 1e-2


# ---------------------------------------------------------------------------
# Reading R8: each stage's potential from its own input -> second order in tau
# ---------------------------------------------------------------------------

def _r8_setup():
    """Exact shifts: tau_min dp / (m dx) = 1, so every step moves each
    momentum plane by whole cells for tau = k tau_min; a Hartree term with
    W = cos(r) couples the moving density to the momentum kicks."""
    L, nx, nk, m = 2 * math.pi, 256, 4, 0.1
    dx, dp = L / nx, math.pi / L
    tmin = m * dx / dp

    def prob(tau):
        return inputs.Problem(nx=nx, nk=nk, L=L, dt=tau, mass=m, vext=inputs.zero_potential(),
                              vee=lambda r: math.cos(r), gamma=5.0, c_hartree=1.0)

    x = -L / 2 + dx * np.arange(nx)
    p = (np.arange(nk) - nk // 2) * dp
    X1, X2, P1, P2 = np.meshgrid(x, x, p, p, indexing="ij")
    f0 = ((1 + 0.6 * np.cos(X1 - 0.3) + 0.3 * np.sin(2 * X1)) * (1 + 0.5 * np.cos(X2 + 0.7))
          * np.exp(-2 * (P1 - 0.2) ** 2 - 2 * (P2 + 0.1) ** 2))
    f0 = f0 + f0.transpose(1, 0, 3, 2)
    f0 /= f0.sum() * dx * dx * dp * dp
    return prob, tmin, np.ascontiguousarray(f0)


def _frozen_step(o, f, nsteps):
    """The oracle's Lawson step from its own parts with one planted mistake:
    the corrector's pseudo-difference operator reuses the potential of f^n."""
    tau = o.prob.dt
    for _ in range(nsteps):
        n1, n2 = o.marginals(f)
        U1, U2 = o.potential_fine(n1), o.potential_fine(n2)
        g = o.theta_with(f, U1, U2, 7)
        a, b = o.advect(f, tau), o.advect(g, tau)
        c = o.theta_with(a + tau * b, U1, U2, 7)
        f = a + 0.5 * tau * (b + c)
    return f


def _r8_ratios(frozen):
    prob, tmin, f0 = _r8_setup()
    run = (lambda o, f, n: _frozen_step(o, f, n)) if frozen else (lambda o, f, n: o.step(f, n))
    ref = run(oracle.Oracle(prob(tmin)), f0, 16)
    errs = [np.linalg.norm(run(oracle.Oracle(prob(k * tmin)), f0, 16 // k) - ref) / np.linalg.norm(ref)
            for k in (2, 4, 8)]
    # e(k tau) - e(tau) ~ (k^2 - 1) tau^2 for a second-order step: ratios 5.0 and 4.2;
    # ~ (k - 1) tau for a first-order one: ratios 3.0 and 2.3
    return errs[1] / errs[0], errs[2] / errs[1]


def test_stage_potential_is_second_order():
    r = _r8_ratios(frozen=False)
    assert min(r) > 4.0 and max(r) < 6.0, r


def test_frozen_stage_potential_is_caught():
    r = _r8_ratios(frozen=True)
    assert max(r) < 3.6, r


# ---------------------------------------------------------------------------
# Harmonic potential, interaction off: exact classical rotation of phase space
# ---------------------------------------------------------------------------

OMEGA, X0 = 1.0, 1.0


def _harmonic_error(nx, nk, tau, nsteps, lib=None):
    """Particle 1 starts as the coherent state displaced to X0, particle 2 in
    the ground state (width^2 = hbar/(2 m omega)); for V = m omega^2 x^2/2 the
    Wigner function rotates rigidly: f(x, p, t) = f0(x cos wt - p sin wt / (m w),
    p cos wt + m w x sin wt).  Both packets stay far from the fold."""
    L = 12.0
    prob = inputs.Problem(nx=nx, nk=nk, L=L, dt=tau, vext=inputs.harmonic(OMEGA), vee=inputs.zero_potential(),
                          gamma=0.0, c_hartree=0.0)
    s2 = 1.0 / (2 * OMEGA)
    x, p = prob.x(), prob.p()

    def g(xx, pp, xc):
        return np.exp(-(xx - xc) ** 2 / (2 * s2) - 2 * s2 * pp ** 2) / np.pi

    X1, X2, P1, P2 = np.meshgrid(x, x, p, p, indexing="ij")
    f0 = np.ascontiguousarray(g(X1, P1, X0) * g(X2, P2, 0.0))
    t = tau * nsteps
    c, s = math.cos(OMEGA * t), math.sin(OMEGA * t)
    exact = g(X1 * c - P1 * s / OMEGA, P1 * c + OMEGA * X1 * s, X0) * g(X2, P2, 0.0)
    got = oracle.Oracle(prob, lib=lib).step(f0, nsteps)
    return np.linalg.norm(got - exact) / np.linalg.norm(exact)


def test_harmonic_rotation_second_order_in_tau():
    e1 = _harmonic_error(48, 40, 0.2, 2)
    e2 = _harmonic_error(48, 40, 0.1, 4)
    assert e2 < 1e-2 and 3.4 < e1 / e2 < 5.0, (e1, e2)


def test_harmonic_rotation_fourth_order_in_dx():
    """One short step: the time error (tau^3) is far below the spline's."""
    e1 = _harmonic_error(20, 40, 0.02, 1)
    e2 = _harmonic_error(40, 40, 0.02, 1)
    assert e2 < 1e-4 and 12.0 < e1 / e2 < 24.0, (e1, e2)


def test_harmonic_rotation_catches_flipped_operator_sign():
    lib = oracle.variant("theta_flipped_sign", [("out[idx4(P, i1, i2, n1, n2)] = creal((I / hb) * s);",
                                                 "out[idx4(P, i1, i2, n1, n2)] = creal((-I / hb) * s);")])
    assert _harmonic_error(24, 32, 0.1, 2) < 1e-2
    assert _harmonic_error(24, 32, 0.1, 2, lib=lib) > 0.1
