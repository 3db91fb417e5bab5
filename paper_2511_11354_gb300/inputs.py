"""Seeded synthetic inputs for the periodic 1-D two-body Wigner 2-RDM step.

This module is shared by the CUDA path's callers (tests, bench) and by the
CPU oracle.  It holds problem *inputs* only -- the potentials as plain
functions of one coordinate, the initial 2-RDM Wigner function and the
random numbers -- and none of the method's arithmetic (no pseudo-difference
operator, no spline, no time step).  It imports nothing from the package.

Workloads (Sec. 5 of arXiv:2511.11354 runs Gaussian-type synthetic data; no
dataset is involved):

* ``small``  -- 32^4 grid, L = 20, V = 0.5 cos(2 pi x / L), W = 1/sqrt(r^2+1),
  packets (x0=-3, p0=+0.5) x (x0=+3, p0=-0.5), dt = 0.01.
* ``dwell``  -- 64^4 grid, L = 24, capped double well min(0.05 (x^2-16)^2, 20)
  folded periodic, packet centres drawn U[-4, 4] from the seed, dt = 0.005.
* ``dwell_literal`` -- the same with the uncapped well (explicitly unstable
  for the Lawson step; kept as a negative test case).

Initial data: a product of pure-state Gaussians
G(x, p) = 1/(pi hbar) exp(-(x-x0)^2/(2 s^2) - 2 s^2 (p-p0)^2 / hbar^2)
(the pure-state form used for the strongly correlated example, Sec. 5.3,
with a = 1/(4 s^2)), plus 1e-3 max|g| uniform noise from SplitMix64, then
exchange-symmetrised, then normalised to unit mass.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """SplitMix64 output for stream ``seed`` at positions ``index`` (uint64).

    The published SplitMix64 finaliser (Steele, Lea & Flood, 2014) applied
    to the counter ``seed * golden + (index + 1) * golden``.
    """
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) * _GOLDEN + (index.astype(np.uint64) + np.uint64(1)) * _GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, index: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, index) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def fold(x, L):
    """Min-image fold of x into [-L/2, L/2) (x = +L/2 maps to -L/2)."""
    return x - L * np.floor((x + 0.5 * L) / L)


# ----------------------------------------------------------------------------
# Potentials (plain functions of one coordinate in [-L/2, L/2))
# ----------------------------------------------------------------------------

def cos_potential(amplitude: float, L: float) -> Callable[[float], float]:
    return lambda x: amplitude * math.cos(2.0 * math.pi * x / L)


def soft_coulomb(eps: float = 1.0) -> Callable[[float], float]:
    """Smoothed Coulomb kernel 1/sqrt(r^2 + eps) (Sec. 2, 1-D example)."""
    return lambda r: 1.0 / math.sqrt(r * r + eps)


def double_well(cap: float | None = 20.0) -> Callable[[float], float]:
    """0.05 (x^2 - 16)^2, optionally capped at ``cap``."""
    if cap is None:
        return lambda x: 0.05 * (x * x - 16.0) ** 2
    return lambda x: min(0.05 * (x * x - 16.0) ** 2, cap)


def harmonic(omega: float) -> Callable[[float], float]:
    return lambda x: 0.5 * omega * omega * x * x


def gaussian_potential(height: float, width2: float = 2.0) -> Callable[[float], float]:
    """height * exp(-x^2 / width2); the Gaussian two-body interaction of the
    two-body convergence test uses height H_B and width2 = 2."""
    return lambda x: height * math.exp(-x * x / width2)


def zero_potential() -> Callable[[float], float]:
    return lambda x: 0.0


# ----------------------------------------------------------------------------
# Problem description
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    nx: int
    nk: int
    L: float
    dt: float
    vext: Callable[[float], float]
    vee: Callable[[float], float]
    gamma: float = 1.0
    c_hartree: float = 1.0
    c_xc: float = 0.0
    xc_kind: int = 0          # 0 none, 1 phi(n) = n, 2 Hedin-Lundqvist
    hbar: float = 1.0
    mass: float = 1.0
    hartree: str = "pair"     # "pair": gamma dx sum W n; "poisson": neutralised periodic Poisson
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def dx(self) -> float:
        return self.L / self.nx

    @property
    def dp(self) -> float:
        # momentum lattice spacing fixed by the spatial period (Sec. 3.1)
        return math.pi * self.hbar / self.L

    def x(self) -> np.ndarray:
        return -0.5 * self.L + self.dx * np.arange(self.nx)

    def p(self) -> np.ndarray:
        return (np.arange(self.nk) - self.nk // 2) * self.dp

    @property
    def points(self) -> int:
        return self.nx * self.nx * self.nk * self.nk


def gaussian_1body(x, p, x0, p0, sigma, hbar, L):
    """Pure-state Gaussian Wigner function, min-image in x."""
    u = fold(x - x0, L)
    return (1.0 / (math.pi * hbar)) * np.exp(-u * u / (2 * sigma * sigma)
                                             - 2 * sigma * sigma * (p - p0) ** 2 / (hbar * hbar))


def initial_state(prob: Problem, centres, momenta=(0.5, -0.5), sigma: float = 1.0,
                  noise: float = 1e-3, seed: int = 0) -> np.ndarray:
    """Exchange-symmetrised product of two Gaussian packets plus seeded noise.

    Returns f[i1][i2][n1][n2] (float64, C order), normalised to unit mass
    sum(f) dx^2 dp^2 = 1.
    """
    x = prob.x()
    p = prob.p()
    ga = gaussian_1body(x[:, None], p[None, :], centres[0], momenta[0], sigma, prob.hbar, prob.L)
    gb = gaussian_1body(x[:, None], p[None, :], centres[1], momenta[1], sigma, prob.hbar, prob.L)
    # g(x1, x2, p1, p2) = ga(x1, p1) gb(x2, p2) in layout [i1][i2][n1][n2]
    g = np.einsum("ac,bd->abcd", ga, gb)
    if noise:
        idx = np.arange(g.size, dtype=np.uint64).reshape(g.shape)
        g = g + noise * np.max(np.abs(g)) * (2.0 * uniform01(seed, idx) - 1.0)
    f = 0.5 * (g + g.transpose(1, 0, 3, 2))
    mass = f.sum() * prob.dx ** 2 * prob.dp ** 2
    return np.ascontiguousarray(f / mass)


def initial_state_chunked(prob: Problem, centres, momenta=(0.5, -0.5), sigma: float = 1.0,
                          noise: float = 1e-3, seed: int = 0, dtype=np.float32) -> np.ndarray:
    """initial_state() for grids too large for whole-array temporaries: the
    same values (the noise is a counter-based function of the linear index,
    evaluated at both the index and its exchange image), built one x1-slab at
    a time and returned in ``dtype``."""
    nx, nk = prob.nx, prob.nk
    x, p = prob.x(), prob.p()
    ga = gaussian_1body(x[:, None], p[None, :], centres[0], momenta[0], sigma, prob.hbar, prob.L)
    gb = gaussian_1body(x[:, None], p[None, :], centres[1], momenta[1], sigma, prob.hbar, prob.L)
    amp = noise * float(np.max(np.abs(ga)) * np.max(np.abs(gb)))
    out = np.empty((nx, nx, nk, nk), dtype=dtype)
    i2 = np.arange(nx, dtype=np.uint64)[:, None, None]
    n1 = np.arange(nk, dtype=np.uint64)[None, :, None]
    n2 = np.arange(nk, dtype=np.uint64)[None, None, :]
    NX, NK = np.uint64(nx), np.uint64(nk)
    total = 0.0
    for a in range(nx):
        i1 = np.uint64(a)
        g = ga[a][None, :, None] * gb[:, None, :]     # g(x1=a, x2, p1, p2)     [i2][n1][n2]
        gt = gb[a][None, :, None] * ga[:, None, :]    # g(x2, x1=a, p2, p1)     exchange image
        f = g + gt
        if noise:
            idx = ((i1 * NX + i2) * NK + n1) * NK + n2
            idt = ((i2 * NX + i1) * NK + n2) * NK + n1
            f = f + amp * (2.0 * uniform01(seed, idx) - 1.0) + amp * (2.0 * uniform01(seed, idt) - 1.0)
        f *= 0.5
        total += float(f.sum())
        out[a] = f
    out /= dtype(total * prob.dx ** 2 * prob.dp ** 2)
    return out


def draw_centres(seed: int, lo: float = -4.0, hi: float = 4.0):
    u = uniform01(seed + 0x5EED, np.arange(2, dtype=np.uint64))
    c = np.sort(lo + (hi - lo) * u)
    return float(c[0]), float(c[1])


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

def workload_small(nx: int = 32, nk: int = 32) -> tuple[Problem, np.ndarray]:
    """32^4, L=20, cosine external potential, soft-Coulomb pair, 20 steps of dt=0.01."""
    L = 20.0
    prob = Problem(nx=nx, nk=nk, L=L, dt=0.01, vext=cos_potential(0.5, L), vee=soft_coulomb(1.0),
                   gamma=1.0, c_hartree=1.0, name=f"small_{nx}x{nk}", meta={"steps": 20, "seed": 0})
    f0 = initial_state(prob, centres=(-3.0, 3.0), seed=0)
    return prob, f0


def workload_dwell(nx: int = 64, nk: int = 64, literal: bool = False, seed: int = 1,
                   dtype=np.float64) -> tuple[Problem, np.ndarray]:
    """64^4 capped double well on L=24, soft-Coulomb pair, dt = 0.005."""
    L = 24.0
    prob = Problem(nx=nx, nk=nk, L=L, dt=0.005, vext=double_well(None if literal else 20.0),
                   vee=soft_coulomb(1.0), gamma=1.0, c_hartree=1.0,
                   name=("dwell_literal" if literal else "dwell") + f"_{nx}x{nk}",
                   meta={"steps": 1000, "seed": seed, "obs_every": 10})
    f0 = initial_state(prob, centres=draw_centres(seed), seed=seed)
    return prob, f0.astype(dtype, copy=False)


def workload_batch(n: int = 64, seed: int = 3):
    """Independent problems of uneven size and pair strength: per instance
    nx in {24, 32, 48, 64}, nk in {32, 48, 64} and gamma in U[0.2, 2.0], all
    drawn from the seed; L = 20, V = 0.5 cos(2 pi x / L), soft-Coulomb pair
    scaled by gamma, Hartree on, dt = 0.01, two Gaussian packets with centres
    drawn U[-4, 4] and momenta +-0.5.  Returns (problems, states)."""
    L = 20.0
    u = uniform01(seed, np.arange(3 * n, dtype=np.uint64)).reshape(n, 3)
    nxs, nks = (24, 32, 48, 64), (32, 48, 64)
    probs, states = [], []
    for i in range(n):
        nx = nxs[min(int(u[i, 0] * 4), 3)]
        nk = nks[min(int(u[i, 1] * 3), 2)]
        gamma = 0.2 + 1.8 * float(u[i, 2])
        prob = Problem(nx=nx, nk=nk, L=L, dt=0.01, vext=cos_potential(0.5, L), vee=soft_coulomb(1.0),
                       gamma=gamma, c_hartree=1.0, name=f"batch{i}_{nx}x{nk}", meta={"steps": 500, "seed": seed})
        probs.append(prob)
        states.append(initial_state(prob, centres=draw_centres(seed * 1000 + i), seed=seed * 1000 + i))
    return probs, states


# ---------------------------------------------------------------------------
# Periodic plasma workloads (the quantum Landau damping and two-stream
# examples): box [-5 pi, 5 pi)^2, momentum spacing 0.1 (= pi hbar / L),
# Hartree from the neutralised periodic Poisson equation, Hedin-Lundqvist
# XC, smoothed Coulomb pair 1/sqrt(r^2 + soft), dt = 0.01.  The paper's mesh
# is 257^2 x 128^2 with the endpoint; the periodic grid drops it: 256^2 x 128^2.
# ---------------------------------------------------------------------------

PLASMA_L = 10.0 * math.pi
PLASMA_K = 0.4


def plasma_problem(kind: str = "landau", nx: int = 256, nk: int = 128, soft: float = 1.0, xc: bool = True,
                   two_body: bool = True) -> Problem:
    if kind not in ("landau", "two_stream"):
        raise ValueError(kind)
    return Problem(nx=nx, nk=nk, L=PLASMA_L, dt=0.01, vext=zero_potential(), vee=soft_coulomb(soft),
                   gamma=1.0 if two_body else 0.0, c_hartree=1.0, c_xc=1.0 if xc else 0.0, xc_kind=2 if xc else 0,
                   hartree="poisson", name=f"plasma_{kind}", meta={"eps": 0.1 if kind == "landau" else 0.02})


def plasma_factors(prob: Problem, kind: str, eps: float | None = None):
    """The separable initial 2-RDM f = a(x1) a(x2) b(p1) b(p2) of the plasma
    examples: a = 1 + eps cos(0.4 x); Landau: b = exp(-p^2/2) / sqrt(2 pi);
    two-stream: b = (1 + 5 p^2) exp(-p^2/2) / (6 sqrt(2 pi))."""
    eps = prob.meta.get("eps", 0.1) if eps is None else eps
    a = 1.0 + eps * np.cos(PLASMA_K * prob.x())
    p = prob.p()
    if kind == "landau":
        b = np.exp(-0.5 * p * p) / math.sqrt(2.0 * math.pi)
    else:
        b = (1.0 + 5.0 * p * p) * np.exp(-0.5 * p * p) / (6.0 * math.sqrt(2.0 * math.pi))
    return a, b


def workload_plasma(kind: str = "landau", nx: int = 256, nk: int = 128, soft: float = 1.0, xc: bool = True,
                    two_body: bool = True, eps: float | None = None, dtype=np.float64):
    """(problem, initial state) of a plasma example (host array; for the full
    256^2 x 128^2 mesh build the state from plasma_factors on the device)."""
    prob = plasma_problem(kind, nx, nk, soft, xc, two_body)
    a, b = plasma_factors(prob, kind, eps)
    f = (a[:, None, None, None] * a[None, :, None, None] * b[None, None, :, None] * b[None, None, None, :])
    return prob, np.ascontiguousarray(f, dtype=dtype)



# ---------------------------------------------------------------------------
# Non-periodic problems (Sec. 3.2 and the strongly correlated example of
# Sec. 5.4): a bounded box [-L/2, L/2]^2 sampled with its endpoints, and a
# momentum window [-Lp/2, Lp/2] split into ncell equal cells of nq
# Chebyshev-Gauss collocation points each.
# ---------------------------------------------------------------------------

@dataclass
class SemProblem:
    nx: int                   # spatial points per axis, both ends included
    ncell: int                # momentum cells per axis
    nq: int                   # Chebyshev-Gauss points per cell
    L: float                  # box [-L/2, L/2]
    Lp: float                 # momentum window [-Lp/2, Lp/2]
    dt: float
    vext: Callable[[float], float]
    vee: Callable[[float], float]
    gamma: float = 1.0        # strength of the two-body term gamma W(x1 - x2)
    c_hartree: float = 1.0    # Hartree term c_H dx sum_q W(x - x_q) n(x_q)
    c_xc: float = 0.0
    xc_kind: int = 0          # 0 none, 1 phi(n) = n, 2 Hedin-Lundqvist
    hbar: float = 1.0
    mass: float = 1.0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def dx(self) -> float:
        return self.L / (self.nx - 1)

    @property
    def np_(self) -> int:
        return self.ncell * self.nq

    def x(self) -> np.ndarray:
        return -0.5 * self.L + self.dx * np.arange(self.nx)

    def p(self) -> np.ndarray:
        """Collocation momenta, ascending: cell s spans
        [-Lp/2 + s Lp/ncell, -Lp/2 + (s+1) Lp/ncell], its points sit at the
        Chebyshev-Gauss abscissae -cos((2q+1) pi / (2 nq)) of the cell."""
        w = self.Lp / self.ncell
        c = -0.5 * self.Lp + w * (np.arange(self.ncell) + 0.5)
        eta = -np.cos((2 * np.arange(self.nq) + 1) * np.pi / (2 * self.nq))
        return (c[:, None] + 0.5 * w * eta[None, :]).reshape(-1)

    @property
    def points(self) -> int:
        return self.nx * self.nx * self.np_ * self.np_


def correlated_state(prob: SemProblem, r0=(-2.0, 2.0), p0=(0.0, 0.0), a: float = 0.25,
                     alpha: float = 0.1, beta: float = 0.1) -> np.ndarray:
    """Initial 2-RDM of the strongly correlated example:
    f(x1, x2, p1, p2) = f1(x1, p1) f1(x2, p2) g12(|x1 - x2|) with
    f1(r, p) = (1 / (2 pi hbar)) sum_k exp(-2a (r - r0_k)^2 - (p - p0_k)^2 / (2 a hbar^2))
    and g12(r) = exp(-beta exp(-alpha r) / r) (zero at r = 0)."""
    x, p, hb = prob.x(), prob.p(), prob.hbar
    f1 = np.zeros((x.size, p.size))
    for rc, pc in zip(r0, p0):
        f1 += np.exp(-2 * a * (x[:, None] - rc) ** 2 - (p[None, :] - pc) ** 2 / (2 * a * hb * hb))
    f1 /= 2 * math.pi * hb
    r = np.abs(x[:, None] - x[None, :])
    with np.errstate(divide="ignore"):
        g = np.where(r > 0, np.exp(-beta * np.exp(-alpha * r) / np.where(r > 0, r, 1.0)), 0.0)
    f = np.einsum("ac,bd->abcd", f1, f1) * g[:, :, None, None]
    return np.ascontiguousarray(f)


def sem_correlated_problem(hamiltonian: str = "IV", soft: float = 1.0, nx: int = 201, ncell: int = 8,
                           nq: int = 16, L: float = 30.0, Lp: float = 20.0 * math.pi / 3.0) -> SemProblem:
    """The strongly correlated example: box [-15, 15]^2, momenta
    [-10 pi/3, 10 pi/3]^2, dx = 0.15 (201 points), 8 cells x 16 points per
    momentum axis, dt = 0.01, smoothed Coulomb 1/sqrt(r^2 + soft).
    Hamiltonians: I Hartree; II + Hedin-Lundqvist XC; III + the pair term;
    IV + the external well -2/sqrt(x^2 + soft)."""
    if hamiltonian not in ("I", "II", "III", "IV"):
        raise ValueError(hamiltonian)
    xc = hamiltonian != "I"
    pair = hamiltonian in ("III", "IV")
    vext = (lambda x: -2.0 / math.sqrt(x * x + soft)) if hamiltonian == "IV" else zero_potential()
    return SemProblem(nx=nx, ncell=ncell, nq=nq, L=L, Lp=Lp, dt=0.01, vext=vext, vee=soft_coulomb(soft),
                      gamma=1.0 if pair else 0.0, c_hartree=1.0, c_xc=1.0 if xc else 0.0, xc_kind=2 if xc else 0,
                      name=f"correlated_{hamiltonian}_{nx}x{ncell * nq}", meta={"soft": soft, "T": 4.0})


def workload_correlated(hamiltonian: str = "IV", soft: float = 1.0, nx: int = 201, ncell: int = 8, nq: int = 16,
                        L: float = 30.0, Lp: float = 20.0 * math.pi / 3.0):
    prob = sem_correlated_problem(hamiltonian, soft, nx, ncell, nq, L, Lp)
    return prob, correlated_state(prob)
