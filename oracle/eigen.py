"""Ground state (and low spectrum) of the generalised eigenproblem H0 c = eps M c.

TEST INFRASTRUCTURE (oracle). Paper Eq. gen_ev (Sec. "Weak form") and Sec.
"Eigenvalue problem" (shift-and-invert near the expected ground energy). Small
problems use LAPACK's dense generalised symmetric solver; large sparse ones use
ARPACK shift-invert (scipy eigsh with sigma) with the shift placed below min V.

Phase convention (Sec. "Wavefunction realignment"): rotate by
exp(-i arg(c^T M c)/2) so that c is real, renormalise to c^H M c = 1, and fix the
sign so that the largest-magnitude component is positive.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


def realign(c, S):
    c = np.asarray(c, dtype=np.complex128)
    z = c @ (S @ c)                         # <c*|M|c*> = c^T M c (bilinear)
    c = c * np.exp(-0.5j * np.angle(z))
    c = c / np.sqrt(np.real(np.conj(c) @ (S @ c)))
    k = int(np.argmax(np.abs(c)))
    if np.real(c[k]) < 0:
        c = -c
    return c


def lowest_states(mats, k=1, sigma=None, dense_max=2500):
    """(energies[k], vectors[:, k]) of H0 c = eps S c, vectors realigned."""
    S, H0 = mats["S"], mats["H0"]
    n = S.shape[0]
    if n <= dense_max:
        w, v = sla.eigh(H0.toarray(), S.toarray(), subset_by_index=[0, k - 1])
    else:
        if sigma is None:
            raise ValueError("sigma required for sparse shift-invert")
        w, v = spla.eigsh(H0.tocsc(), k=k, M=S.tocsc(), sigma=sigma, which="LM", tol=1e-14)
        order = np.argsort(w)
        w, v = w[order], v[:, order]
    vecs = np.stack([realign(v[:, j], S) for j in range(k)], axis=1)
    return w, vecs


def ground_state(mats, sigma=None, dense_max=2500):
    w, v = lowest_states(mats, 1, sigma=sigma, dense_max=dense_max)
    return float(w[0]), v[:, 0]
