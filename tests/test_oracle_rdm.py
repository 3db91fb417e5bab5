"""Pins of the occupation-number reference (oracle/rdm_ref.py): the inverse
Wigner transform on the half grid against closed forms — the density matrix
of a pure Gaussian state, the occupations and correlation entropy of a
two-component mixture — and the trace identity."""
import math

import numpy as np

from oracle import rdm_ref


def _grid(nx=64, nk=64, L=20.0):
    dx, dp = L / nx, math.pi / L
    x = -0.5 * L + dx * np.arange(nx)
    p = (np.arange(nk) - nk // 2) * dp
    return x, p, dx, dp


def _wigner(x, p, x0, p0, sigma):
    """Wigner function of psi = (2 pi s^2)^(-1/4) exp(-(x-x0)^2/(4 s^2) + i p0 x)."""
    return np.exp(-(x[:, None] - x0) ** 2 / (2 * sigma ** 2) - 2 * sigma ** 2 * (p[None, :] - p0) ** 2) / math.pi


def _psi(x, x0, p0, sigma):
    return (2 * math.pi * sigma ** 2) ** -0.25 * np.exp(-(x - x0) ** 2 / (4 * sigma ** 2) + 1j * p0 * x)


def test_pure_gaussian_density_matrix():
    """rho1(x_b, x_c) of a Gaussian wave packet is psi(x_b) psi*(x_c),
    including the odd-index entries built from the half-point values (box
    large enough that the periodic images at |x_b - x_c| ~ L/2 are below
    1e-9)."""
    x, p, dx, dp = _grid(nx=96, nk=64, L=30.0)
    f1 = _wigner(x, p, 1.5, 0.7, 1.2)
    rho = rdm_ref.rho1_from_f1(f1, x.size, p.size, dp)
    ps = _psi(x, 1.5, 0.7, 1.2)
    want = np.outer(ps, ps.conj())
    assert np.abs(rho - want).max() < 1e-8 * np.abs(want).max()
    n = rdm_ref.occupations(rho, dx)
    assert abs(n[0] - 1.0) < 1e-8 and np.abs(n[1:]).max() < 1e-8
    assert abs(rdm_ref.correlation_entropy(n)) < 1e-7


def test_mixture_occupations_and_entropy():
    """A mixture 0.7 |psi_a><psi_a| + 0.3 |psi_b><psi_b| of two far-apart
    packets (orthogonal to 1e-13): occupations 0.7 and 0.3, entropy
    0.7 ln 0.7 + 0.3 ln 0.3."""
    x, p, dx, dp = _grid(nx=96, nk=64, L=24.0)
    f1 = 0.7 * _wigner(x, p, -5.0, 0.3, 0.9) + 0.3 * _wigner(x, p, 5.0, -0.4, 0.9)
    n = rdm_ref.occupations(rdm_ref.rho1_from_f1(f1, x.size, p.size, dp), dx)
    assert abs(n[0] - 0.7) < 1e-8 and abs(n[1] - 0.3) < 1e-8 and np.abs(n[2:]).max() < 1e-8
    s = rdm_ref.correlation_entropy(n)
    assert abs(s - (0.7 * math.log(0.7) + 0.3 * math.log(0.3))) < 1e-7


def test_trace_is_the_mass_and_hermiticity():
    x, p, dx, dp = _grid(nx=33, nk=20)
    rng = np.random.default_rng(2)
    f1 = rng.random((x.size, p.size))
    rho = rdm_ref.rho1_from_f1(f1, x.size, p.size, dp)
    assert np.allclose(rho, rho.conj().T)
    assert abs(np.trace(rho).real * dx - f1.sum() * dx * dp) < 1e-12 * f1.sum() * dx * dp
    assert abs(rdm_ref.occupations(rho, dx).sum() - f1.sum() * dx * dp) < 1e-10


def test_reduced_wigner_function_of_a_product_state():
    x, p, dx, dp = _grid(nx=16, nk=16, L=16.0)
    w1, w2 = _wigner(x, p, -1.0, 0.2, 1.0), _wigner(x, p, 2.0, -0.3, 0.8)
    f = w1[:, None, :, None] * w2[None, :, None, :]
    f1 = rdm_ref.f1_from_state(f, dx, dp)
    assert np.allclose(f1, w1 * w2.sum() * dx * dp, rtol=1e-14, atol=0)
