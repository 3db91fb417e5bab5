"""FP64 CPU oracle for the 1-D two-body Wigner 2-RDM step: the periodic path
(``oracle.py`` over ``w2_oracle.c``) and the non-periodic spectral-element
path (``sem_ref.py``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may use this package; the product path never
does.  It shares no code with the CUDA path (see ``w2_oracle.c``).

Every function is pinned by ``tests/test_oracle_*.py`` against something other
than itself: the paper's two closed forms (Sec. 5.1), a numpy FFT form of the
pseudo-difference operator, exact discrete identities (antisymmetry, mass
leak, exchange symmetry, integer rolls, spline Fourier multipliers),
convergence to classical rotation in a harmonic well, and a brute-force
two-particle Schroedinger evolution.
"""
from .oracle import Oracle, build, lib_path, variant  # noqa: F401
from .sem_ref import SemOracle  # noqa: F401
