"""Pins of the oracle's neutralised periodic Poisson Hartree term (the 1-D
Coulomb example under an ion background, used by the plasma workloads):
closed-form solutions of -V'' = n - mean(n) for trigonometric densities,
including the Nyquist mode's convention, and the conservation laws of a step
with it."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_11354_gb300 import inputs


def _prob(nx=16, nk=8):
    return inputs.Problem(nx=nx, nk=nk, L=inputs.PLASMA_L, dt=0.01, vext=inputs.zero_potential(),
                          vee=inputs.zero_potential(), gamma=0.0, c_hartree=1.0, hartree="poisson")


@pytest.mark.parametrize("nx", [16, 20, 15])
def test_poisson_hartree_closed_form(nx):
    """n(x) = 3 + A cos(k_a x) + B sin(k_b x) gives V_H(y) = A cos(k_a y)/k_a^2 +
    B sin(k_b y)/k_b^2 at every fine point y = x_i + l h' (the constant is
    neutralised)."""
    prob = _prob(nx)
    x = prob.x()
    ka, kb = 2 * math.pi * 2 / prob.L, 2 * math.pi * 5 / prob.L
    n = 3.0 + 0.7 * np.cos(ka * x) - 0.4 * np.sin(kb * x)
    U = oracle.Oracle(prob).potential_fine(n)
    M = 2 * prob.nk
    y = x[:, None] + np.arange(M)[None, :] * prob.L / M
    want = 0.7 * np.cos(ka * y) / ka ** 2 - 0.4 * np.sin(kb * y) / kb ** 2
    assert np.abs(U - want).max() < 1e-12 * np.abs(want).max()


def test_poisson_hartree_nyquist_mode():
    """The grid's alternating density (-1)^q, i.e. cos(k_N x_q) with
    k_N = pi N / L (N divisible by 4), is solved by cos(k_N y)/k_N^2 between
    the grid points too (the Nyquist mode read as its cosine)."""
    prob = _prob(16)
    x = prob.x()
    kN = math.pi * prob.nx / prob.L
    n = np.cos(kN * x)
    assert np.allclose(n, (-1.0) ** np.arange(prob.nx))
    U = oracle.Oracle(prob).potential_fine(n)
    M = 2 * prob.nk
    y = x[:, None] + np.arange(M)[None, :] * prob.L / M
    assert np.abs(U - np.cos(kN * y) / kN ** 2).max() < 1e-12 / kN ** 2


def test_poisson_hartree_is_the_second_antiderivative():
    """A random density: the spectral second derivative of V_H on the grid
    equals -(n - mean n) (the Poisson equation itself, checked with numpy's
    FFT, independent of the convolution the oracle uses)."""
    prob = _prob(32)
    rng = np.random.default_rng(4)
    n = rng.random(prob.nx)
    n[prob.nx // 2] = n[prob.nx // 2]
    U = oracle.Oracle(prob).potential_fine(n)[:, 0]  # on the grid
    k = 2 * math.pi * np.fft.fftfreq(prob.nx, d=prob.dx)
    # drop the Nyquist mode on both sides (its sine part is not representable)
    nh, uh = np.fft.fft(n - n.mean()), np.fft.fft(U)
    keep = np.abs(np.fft.fftfreq(prob.nx)) < 0.5
    assert np.abs((k[keep] ** 2) * uh[keep] - nh[keep]).max() < 1e-10 * np.abs(nh).max()


def test_plasma_step_conserves_mass_and_exchange_symmetry():
    """Three Lawson steps of two-stream data with Poisson Hartree, H-L XC and
    the smoothed Coulomb pair on a box small enough (L = 3) that the momentum
    window (|p| < 7.3) holds the whole distribution: the operator conserves
    mass on the symmetric initial state, the steps keep the exchange symmetry
    to rounding and the mass to the window's leak (~1e-9)."""
    L = 3.0
    prob = inputs.Problem(nx=12, nk=16, L=L, dt=0.01, vext=inputs.zero_potential(), vee=inputs.soft_coulomb(1.0),
                          gamma=1.0, c_hartree=1.0, c_xc=1.0, xc_kind=2, hartree="poisson")
    x, p = prob.x(), prob.p()
    a = 1.0 + 0.02 * np.cos(2 * math.pi * x / L)
    b = (1.0 + 5.0 * p * p) * np.exp(-0.5 * p * p) / (6.0 * math.sqrt(2.0 * math.pi))
    f0 = np.ascontiguousarray(a[:, None, None, None] * a[None, :, None, None] * b[None, None, :, None]
                              * b[None, None, None, :])
    o = oracle.Oracle(prob)
    th = o.theta(f0)
    assert abs(th.sum()) < 1e-12 * np.abs(th).sum()
    f1 = o.step(f0, 3)
    assert np.abs(f1 - f1.transpose(1, 0, 3, 2)).max() < 1e-13 * np.abs(f1).max()
    m0, m1 = o.observables(f0)["mass"], o.observables(f1)["mass"]
    assert abs(m1 - m0) < 1e-7 * m0
