"""Pin of the whole oracle time step against brute-force quantum mechanics.

Two particles on a ring of length L: exact evolution of the two-particle
wavefunction in a plane-wave basis (scipy expm), with band-limited external
and pair potentials, then the exact torus Wigner transform on the momentum
lattice p_n = n dp, dp = pi hbar / L (Sec. 3.1: periodisation in x makes
momentum discrete with this spacing).  For such states the pseudo-difference
operator is exact, so the oracle's only errors are the cubic spline (order 4
in dx) and the Lawson predictor-corrector (order 2 in dt).  With no pair
potential and a product state this is also the product-of-one-body check.
"""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_2511_11354_gb300 import inputs

L = 2 * np.pi
V1, V2 = 0.3, 0.2


def _evolve(T, w1, sym, K=10, seed=7):
    ms = np.arange(-K, K + 1)
    nb = len(ms)
    Vq = {1: V1 / 2, -1: V1 / 2, 2: V2 / 2j, -2: -V2 / 2j}   # 0.3 cos x + 0.2 sin 2x
    Wq = {1: w1 / 2, -1: w1 / 2}                            # w1 cos(x1 - x2)
    H = np.zeros((nb * nb, nb * nb), complex)
    idx = lambda a, b: (a + K) * nb + (b + K)
    for a in ms:
        for b in ms:
            i = idx(a, b)
            H[i, i] += 0.5 * (2 * np.pi / L) ** 2 * (a * a + b * b)
            for q, v in Vq.items():
                if abs(a + q) <= K:
                    H[idx(a + q, b), i] += v
                if abs(b + q) <= K:
                    H[idx(a, b + q), i] += v
            for q, w in Wq.items():
                if abs(a + q) <= K and abs(b - q) <= K:
                    H[idx(a + q, b - q), i] += w
    rng = np.random.default_rng(seed)
    c0 = np.zeros((nb, nb), complex)
    if sym:
        sub = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        sub = sub + sub.T
    else:  # product of two one-body states
        u = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        v = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        sub = np.outer(u, v)
    c0[K - 1:K + 2, K - 1:K + 2] = sub
    c0 /= np.linalg.norm(c0)
    cT = (sl.expm(-1j * H * T) @ c0.reshape(-1)).reshape(nb, nb)
    return c0, cT


def _wigner(c, nx, nk, Ke=7):
    """Exact torus Wigner function of the two-particle pure state with
    plane-wave coefficients c[m1][m2] (|m| <= K):
    f(x1,x2,p_{n1},p_{n2}) = (L dp)^-2 sum_{m1+m1'=n1, m2+m2'=n2}
        c[m1,m2] c*[m1',m2'] exp(2 pi i ((m1-m1') x1 + (m2-m2') x2) / L)."""
    K = (c.shape[0] - 1) // 2
    c = c[K - Ke:K + Ke + 1, K - Ke:K + Ke + 1]
    ms = np.arange(-Ke, Ke + 1)
    dp = np.pi / L
    x = -L / 2 + (L / nx) * np.arange(nx)
    e = np.exp(2j * np.pi * np.outer(x, np.arange(-2 * Ke, 2 * Ke + 1)) / L)
    # R[a, a2][x2, n2] = sum_{b + b2 = n2} c[a,b] c*[a2,b2] e(x2, b - b2)
    S = np.zeros((len(ms), len(ms), nk))
    E2 = np.zeros((nx, len(ms), len(ms)), complex)
    for bi, b in enumerate(ms):
        for b2i, b2 in enumerate(ms):
            n2 = b + b2 + nk // 2
            if 0 <= n2 < nk:
                S[bi, b2i, n2] = 1.0
            E2[:, bi, b2i] = e[:, b - b2 + 2 * Ke]
    R = np.einsum("ab,cd,xbd,bdn->acxn", c, np.conj(c), E2, S, optimize=True)
    f = np.zeros((nx, nx, nk, nk), complex)
    for ai, a in enumerate(ms):
        for a2i, a2 in enumerate(ms):
            n1 = a + a2 + nk // 2
            if 0 <= n1 < nk:
                f[:, :, n1, :] += e[:, a - a2 + 2 * Ke][:, None, None] * R[ai, a2i][None, :, :]
    return (f / (L * dp) ** 2).real


def _oracle_error(c0, cT, T, nx, nk, nsteps, w1):
    prob = inputs.Problem(nx=nx, nk=nk, L=L, dt=T / nsteps,
                          vext=lambda x: V1 * np.cos(2 * np.pi * x / L) + V2 * np.sin(4 * np.pi * x / L),
                          vee=lambda r: w1 * np.cos(2 * np.pi * r / L), gamma=1.0, c_hartree=0.0)
    f0, fT = _wigner(c0, nx, nk), _wigner(cT, nx, nk)
    assert abs(f0.sum() * prob.dx ** 2 * prob.dp ** 2 - 1.0) < 1e-12
    fn = oracle.Oracle(prob).step(f0, nsteps)
    return np.linalg.norm(fn - fT) / np.linalg.norm(fT)


@pytest.mark.parametrize("w1,sym", [(0.5, True), (0.0, False)])
def test_schroedinger_spatial_order(w1, sym):
    T = 0.2
    c0, cT = _evolve(T, w1, sym)
    e16 = _oracle_error(c0, cT, T, 16, 24, 40, w1)
    e32 = _oracle_error(c0, cT, T, 32, 24, 40, w1)
    assert e32 < 4e-5, e32
    assert e16 / e32 > 10.0, (e16, e32)   # ~16 for a 4th-order spline


def test_schroedinger_time_order():
    T, w1 = 0.6, 0.5
    c0, cT = _evolve(T, w1, True)
    e_a = _oracle_error(c0, cT, T, 48, 24, 6, w1)
    e_b = _oracle_error(c0, cT, T, 48, 24, 12, w1)
    assert e_a / e_b > 3.0, (e_a, e_b)     # ~4 for a 2nd-order step
