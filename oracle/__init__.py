"""CPU FP64 oracle for the TDSE-Z Crank-Nicolson propagation path (arXiv 2608.18472).

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package. The
product path (``paper_2608_18472_b300``) never calls it and shares no code with it.

Everything here is a plain, slow, obviously correct restatement of the paper in
numpy/scipy double precision:

* ``bspline``   - Cox-de Boor B-spline recursion and Gauss-Legendre rules
                  (Sec. "Weak form", Eq. tensor3d; Sec. "Parallel assembly").
* ``assemble``  - Galerkin matrices M(=S), T_BDD, V, D, plus the acceleration
                  matrices G = <m^-1 dV> and K = <m^-1> (Eqs. mass_elem, bdd_elem,
                  the potential/dipole element formulas, Eq. pdm_acceleration),
                  assembled by plain element-by-element quadrature, in 1-D, 2-D
                  and 3-D (full tensor quadrature, no sum factorisation).
* ``propagate`` - Crank-Nicolson (Eq. cn_system) with an exact direct solve per
                  step (LAPACK banded LU with partial pivoting in 1-D, SuperLU in
                  2-D/3-D), and the per-step observables of Sec. "Dipoles".
* ``eigen``     - ground state of Eq. gen_ev, phase-realigned (Sec. "Wavefunction
                  realignment").
* ``hhg``       - windowed spectrum S(w) and per-harmonic yields (Sec. "Dipoles").

Parity status: every function is pinned by a ``-m "not gpu"`` test against what
the paper or the mathematics fixes. The non-separable 2-D/3-D potential and mass
terms (soft core, elliptical dot), whose matrix elements have no closed form, are
pinned by the cases that reduce to something independent: an ellipse covering or
missing the domain is the constant medium, a dot stretched into a stripe is the
Kronecker product of the layered 1-D assembly, exchange symmetries of circular
and soft-core media, and soft-core gradients against finite differences of the
assembled potential.
"""
from . import bspline, assemble, propagate, eigen, hhg  # noqa: F401
