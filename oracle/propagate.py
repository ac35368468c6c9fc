"""Crank-Nicolson propagation with an exact solve per step, and per-step observables.

TEST INFRASTRUCTURE (oracle). Paper Sec. "Time propagation", Eq. cn_system:
    (M + i dt/2 H^{n+1/2}) c^{n+1} = (M - i dt/2 H^{n+1/2}) c^n,
    H^{n+1/2} = (H^{n+1} + H^n)/2,   H(t) = T_BDD + V + E(t).D   (length gauge, Eq. laser).
Since H depends on t only through E(t).D, H^{n+1/2} = H0 + Ebar_n.D with
Ebar_n = (E(t_n) + E(t_{n+1}))/2. With an absorbing layer (CAP matrix -i W of Sec. "Parallel assembly")
the Hamiltonian is H^{n+1/2} - i W, i.e. A_n = S + dt/2 W + i dt/2 H^{n+1/2}: still complex symmetric, and
the norm c^H S c decays by the flux the layer absorbs.

Each step is solved directly: LAPACK banded LU with partial pivoting
(scipy.linalg.solve_banded) in 1-D, SuperLU (scipy.sparse.linalg.splu) in 2-D/3-D.

Observables after each step (Sec. "Dipoles"), raw (not divided by the norm):
    norm  = c^H S c
    d_a   = c^H D_a c
    a_a   = -c^H G_a c - E_a(t_{n+1}) c^H K c       (Eq. pdm_acceleration without a_Q)
Row layout per step: [t_{n+1}, E_1..E_dim, d_1..d_dim, a_1..a_dim, norm]. Optionally the total dipole
velocity J = c^H Vel c (Sec. "Currents and coherence dynamics") per step; the position-dependent-mass
acceleration term a_Q of Eq. aQ_definition for a given state (1-D).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .assemble import to_band


def observables(mats, c, E_t):
    """[d_1..d_dim, a_1..a_dim, norm] for state c and field vector E_t at the same time."""
    dim = mats["dim"]
    cc = np.conj(c)
    norm = float(np.real(cc @ (mats["S"] @ c)))
    kq = float(np.real(cc @ (mats["K"] @ c)))
    d = [float(np.real(cc @ (mats["D"][a] @ c))) for a in range(dim)]
    acc = [-float(np.real(cc @ (mats["G"][a] @ c))) - float(E_t[a]) * kq for a in range(dim)]
    return d + acc + [norm]


def current(mats, c):
    """Total dipole velocity J_alpha = c^H Vel_alpha c, Vel_alpha = -(i/2) M_alpha (Sec. "Currents and
    coherence dynamics", Eq. velocity_op, Eq. vel_elem)."""
    return [float(np.real(np.conj(c) @ (-0.5j * (M @ c)))) for M in mats["M"]]


def a_quantum(mats, c):
    """The position-dependent-mass term of the dipole acceleration, Eq. aQ_definition, in 1-D:
    (i/4) <[p m^-1 p, p m^-1 + m^-1 p]> = i <[T, v]> with T = 1/2 p m^-1 p and v = 1/2 (p m^-1 + m^-1 p).
    In the Galerkin basis an operator product A B is A S^-1 B, so <[T, v]> = c^H (T S^-1 Vel - Vel S^-1 T) c
    and a_Q = -2 Im[(T c)^H S^-1 (Vel c)]."""
    T, S = mats["T"], mats["S"]
    vel = -0.5j * (mats["M"][0] @ c)
    x = spla.spsolve(S.tocsc(), vel)
    return float(-2.0 * np.imag(np.conj(T @ c) @ x))


def cn_propagate(mats, c0, field, dt, nsteps, step0=0, p=None, record=True, currents=False):
    """Propagate c0 from step index step0 for nsteps Crank-Nicolson steps.

    field: (>= step0+nsteps+1, dim) samples E(t_n) at t_n = n dt. Returns (c, obs) with obs of
    shape (nsteps, 1 + 3 dim + 1). With currents=True also J[nsteps][dim] (current()) after each step,
    returned as a third value."""
    dim = mats["dim"]
    field = np.asarray(field, dtype=np.float64).reshape(len(field), -1)
    tau = 0.5 * dt
    S, H0, D = mats["S"], mats["H0"], mats["D"]
    W = mats.get("W")
    if W is not None and W.count_nonzero() == 0:
        W = None
    c = np.asarray(c0, dtype=np.complex128).copy()
    obs = np.zeros((nsteps, 1 + 3 * dim + 1))
    J = np.zeros((nsteps, dim))
    if dim == 1:
        if p is None:
            p = int(np.max(np.abs(S.tocoo().row - S.tocoo().col)))
        Sb, Hb, Db = to_band(S, p), to_band(H0, p), to_band(D[0], p)
        Wb = to_band(W, p) if W is not None else 0.0
    for k in range(nsteps):
        n = step0 + k
        ebar = 0.5 * (field[n] + field[n + 1])
        if dim == 1:
            Hn = Hb + ebar[0] * Db - 1j * Wb          # H^{n+1/2} - i W (absorbing layer)
            Ab = Sb + 1j * tau * Hn
            Bb = Sb - 1j * tau * Hn
            rhs = _band_matvec(Bb, c, p)
            c = sla.solve_banded((p, p), Ab, rhs)
        else:
            Hn = H0 + sum(ebar[a] * D[a] for a in range(dim))
            if W is not None:
                Hn = Hn - 1j * W
            A = (S + 1j * tau * Hn).tocsc()
            B = (S - 1j * tau * Hn).tocsr()
            c = spla.splu(A).solve(B @ c)
        if record:
            obs[k, 0] = (n + 1) * dt
            obs[k, 1:1 + dim] = field[n + 1]
            obs[k, 1 + dim:] = observables(mats, c, field[n + 1])
        if currents:
            J[k] = current(mats, c)
    if currents:
        return c, obs, J
    return c, obs


def _band_matvec(ab, x, p):
    """y = A x for A in general band storage ab[p + i - j, j]."""
    n = x.shape[0]
    y = np.zeros(n, dtype=np.result_type(ab.dtype, x.dtype))
    for k in range(-p, p + 1):            # diagonal offset j - i = k
        row = p - k
        if k >= 0:
            y[:n - k] += ab[row, k:] * x[k:]
        else:
            y[-k:] += ab[row, :n + k] * x[:n + k]
    return y


def dense_cn_step(S, H, c, dt):
    """One CN step by dense Gaussian elimination (numpy.linalg.solve); brute force for tiny n."""
    S = S.toarray() if hasattr(S, "toarray") else S
    H = H.toarray() if hasattr(H, "toarray") else H
    A = S + 0.5j * dt * H
    B = S - 0.5j * dt * H
    return np.linalg.solve(A, B @ c)
