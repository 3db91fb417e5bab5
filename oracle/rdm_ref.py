"""Plain numpy reference of the occupation numbers and the correlation
entropy of the one-body density matrix (test infrastructure only).

Follows the paper's appendix on the calculation of the correlation entropy
through the Wigner function:

* f1(x, p) = sum_{x2, p2} f(x, x2, p, p2) dx dp, the reduced one-body Wigner
  function of particle 1;
* the inverse Wigner transform rho1(r - hbar y/2, r + hbar y/2) =
  int f1(r, p) e^{-i p y} dp on the grid (the inverse of the paper's
  definition f1 = (1/2 pi) int rho1(r - y/2, r + y/2) e^{i p y / hbar} dy):
  with r = x_mu and hbar y / 2 = nu dx, rho1(x_{mu-nu}, x_{mu+nu}) =
  dp sum_n f1(x_mu, p_n) e^{-2 pi i (n - nk/2) nu / nx};
* occupation numbers n_k = eigenvalues of the discretised integral operator
  rho1 dx, and s = (1 / N) sum_k n_k ln n_k with N = sum_k n_k.

Readings (listed in the design notes as R16): the quadrature weight of the
p integral is dp (the printed prefactor is garbled); entries with an odd
index sum need mu = (b + c)/2 half-integer, where f1 is taken from its
periodic trigonometric interpolant in x (Nyquist mode halved), the "half
grid"; the pair offset c - b is the minimal image on the torus (in
[-nx/2, nx/2)), and rho1 is made Hermitian as (rho1 + rho1^H)/2 (the
offset -nx/2 has no partner); eigenvalues below 1e-14 of the largest do not
enter the logarithm.
"""
import numpy as np


def f1_from_state(f, dx, dp):
    """f[i1][i2][n1][n2] -> f1[i][n] = sum_{i2, n2} f dx dp."""
    return f.sum(axis=(1, 3)) * dx * dp


def trig_half_points(g):
    """Values of the periodic trigonometric interpolant of the columns of
    g[nx][...] at the half points x_a + dx/2: every mode m is advanced by the
    phase e^{i pi m / nx}; for even nx the Nyquist mode, taken as its cosine,
    vanishes there."""
    nx = g.shape[0]
    m = np.fft.fftfreq(nx, d=1.0 / nx)
    ph = np.exp(1j * np.pi * m / nx)
    if nx % 2 == 0:
        ph[nx // 2] = 0.0
    c = np.fft.fft(g, axis=0) * ph.reshape((nx,) + (1,) * (g.ndim - 1))
    return np.real(np.fft.ifft(c, axis=0))


def rho1_from_f1(f1, nx, nk, dp):
    """rho1[b][c] (complex nx x nx) from f1[nx][nk] by the rules above."""
    fh = trig_half_points(f1)  # f1 at x_a + dx/2
    n = np.arange(nk) - nk // 2
    rho = np.zeros((nx, nx), dtype=np.complex128)
    for b in range(nx):
        for c in range(nx):
            d = (c - b) % nx
            if d >= (nx + 1) // 2:
                d -= nx  # minimal image: b = mu - d/2, c = mu + d/2
            s2 = 2 * b + d  # twice the midpoint index mu
            row = f1[(s2 // 2) % nx] if s2 % 2 == 0 else fh[((s2 - 1) // 2) % nx]
            rho[b, c] = dp * np.sum(row * np.exp(-2j * np.pi * n * (d / 2.0) / nx))
    return 0.5 * (rho + rho.conj().T)


def occupations(rho, dx):
    """Eigenvalues of rho dx, largest first (numpy's Hermitian eigensolver)."""
    return np.sort(np.linalg.eigvalsh(rho * dx))[::-1]


def correlation_entropy(nk_vals, cut=1e-14):
    lam = np.asarray(nk_vals, dtype=np.float64)
    N = lam.sum()
    pos = lam[lam > cut * lam.max()]
    return float(np.sum(pos * np.log(pos)) / N)
