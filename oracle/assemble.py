"""Galerkin matrices by plain element-by-element Gauss quadrature.

TEST INFRASTRUCTURE (oracle). Paper Sec. "Parallel assembly":
    M_ab  = sum_q w_q J_q N_a N_b                                   (Eq. mass_elem; called S here)
    T_ab  = 1/2 sum_q w_q J_q m^-1(r_q) grad N_a . grad N_b         (Eq. bdd_elem)
    V_ab  = sum_q w_q J_q V(r_q) N_a N_b                            (potential element formula)
    D_ab  = sum_q w_q J_q r_{q,alpha} N_a N_b                       (dipole element formula)
and, for the Ehrenfest acceleration of Eq. pdm_acceleration (without a_Q):
    G_ab  = sum_q w_q J_q m^-1(r_q) d_alpha V(r_q) N_a N_b
    K_ab  = sum_q w_q J_q m^-1(r_q) N_a N_b
and the real mask matrix of the complex absorbing potential (CAP matrix, -i W):
    W_ab  = sum_q w_q J_q eta(r_q) N_a N_b
and the BenDaniel-Duke velocity matrix of Eq. vel_elem, kept as its real antisymmetric part M_alpha:
    Vel_alpha = -(i/2) M_alpha,   (M_alpha)_ab = sum_q w_q J_q m^-1(r_q) (N_a d_alpha N_b - d_alpha N_a N_b)
Global matrices are sums of the element matrices; Dirichlet conditions drop the
first and last B-spline along every axis (Sec. "Weak form").

In 2-D and 3-D the basis is the tensor product of Eq. tensor3d and every
integral is taken with the full tensor-product Gauss rule on each element, with
the integrand (mass, potential, its gradient) evaluated pointwise - no
separation or sum factorisation. Linear index of a tensor function: x fastest,
I = i_x + n_x (i_y + n_y i_z).
"""
from __future__ import annotations

from itertools import product

import numpy as np
import scipy.sparse as sp

from .bspline import quadrature_1d


# ------------------------------------------------------------------ media
def _layer_index(bounds, x):
    r = np.searchsorted(np.asarray(bounds, dtype=np.float64), x, side="right") - 1
    return np.clip(r, 0, len(bounds) - 2)


def inv_mass(med, X):
    """m^-1 at points; X is a tuple of coordinate arrays (one per axis)."""
    m = med["mass"]
    k = m["kind"]
    if k == "const":
        return np.full(X[0].shape, 1.0 / m["m"])
    if k == "quesne":                        # m(x) = (1 + x/a)^-1  (Eq. mass)
        return 1.0 + X[0] / m["a"]
    if k == "layers":
        vals = np.asarray(m["m"], dtype=np.float64)
        return 1.0 / vals[_layer_index(m["bounds"], X[0])]
    if k == "ellipse":
        inside = (X[0] / m["a"]) ** 2 + (X[1] / m["b"]) ** 2 < 1.0
        return np.where(inside, 1.0 / m["m_in"], 1.0 / m["m_out"])
    raise ValueError(f"unknown mass kind {k}")


def potential(med, X):
    v = med["potential"]
    k = v["kind"]
    if k == "zero":
        return np.zeros(X[0].shape)
    if k == "softcore":                      # -z / sqrt(|r|^2 + eps)
        r2 = sum(x * x for x in X)
        return -v["z"] / np.sqrt(r2 + v["eps"])
    if k == "ho":                            # 1/2 sum_a w_a^2 x_a^2
        return 0.5 * sum((w * w) * x * x for w, x in zip(v["omega"], X))
    if k == "quesne":                        # V_code = 1/2 * a w^2 x^2 / (4 (x + a))  (Eq. rescaling)
        a, w = v["a"], v["omega"]
        x = X[0]
        return 0.5 * a * w * w * x * x / (4.0 * (x + a))
    if k == "layers":
        vals = np.asarray(v["V"], dtype=np.float64)
        return vals[_layer_index(v["bounds"], X[0])]
    if k == "ellipse":
        inside = (X[0] / v["a"]) ** 2 + (X[1] / v["b"]) ** 2 < 1.0
        return np.where(inside, v["v_in"], v["v_out"])
    if k == "h2p_softcore":                  # two-centre soft-core along x (Sec. Molecular HHG)
        R, eps = v["R"], v["eps"]
        x = X[0]
        return -1.0 / np.sqrt((x + R / 2) ** 2 + eps) - 1.0 / np.sqrt((x - R / 2) ** 2 + eps)
    raise ValueError(f"unknown potential kind {k}")


def grad_potential(med, X, axis):
    """d V / d x_axis at points (piecewise-constant media have zero gradient almost everywhere)."""
    v = med["potential"]
    k = v["kind"]
    if k in ("zero", "layers", "ellipse"):
        return np.zeros(X[0].shape)
    if k == "softcore":
        r2 = sum(x * x for x in X)
        return v["z"] * X[axis] * (r2 + v["eps"]) ** -1.5
    if k == "ho":
        w = v["omega"][axis]
        return w * w * X[axis]
    if k == "quesne":
        a, w = v["a"], v["omega"]
        x = X[0]
        # d/dx [a w^2 x^2 / (8 (x + a))] = a w^2 x (x + 2a) / (8 (x + a)^2)
        return a * w * w * x * (x + 2 * a) / (8.0 * (x + a) ** 2)
    if k == "h2p_softcore":
        R, eps = v["R"], v["eps"]
        x = X[0]
        return (x + R / 2) * ((x + R / 2) ** 2 + eps) ** -1.5 + (x - R / 2) * ((x - R / 2) ** 2 + eps) ** -1.5
    raise ValueError(f"unknown potential kind {k}")


# ------------------------------------------------------------------ absorbing layer (CAP)
# Sec. "Parallel assembly", CAP matrix: W_ab = -i sum_q w_q J_q eta(r_q) N_a N_b with a smooth mask eta >= 0
# that is non-zero only in a boundary layer; the paper implements a Manolopoulos-type mask and prints no
# formula. Readings (medium key "cap"): eta is the sum over the axes of a 1-D mask of |x_a| that starts
# at |x_a| = r0 and ends at |x_a| = R, with s = (|x_a| - r0)/(R - r0) in (0, 1]:
#   "poly":          eta = eta0 s^k                        (closed-form integrals, the pinned case)
#   "manolopoulos":  eta = (1/(2m)) (2 pi/(R - r0))^2 f(c s),  f(y) = a y - b y^3 + 4/(c - y)^2 - 4/(c + y)^2,
#                    a = 1 - 16/c^3,  b = (1 - 17/c^3)/c^2,  c = sqrt(2) K(1/sqrt 2) = 2.62206
# (Manolopoulos' transmission-free absorbing potential, J. Chem. Phys. 117, 9552 (2002): a layer of width
# R - r0 = c/(2 k_min) absorbs with little reflection every wave of energy above E_min = k_min^2/(2m); the
# mask diverges at |x_a| = R, which must be the domain's edge).
MANOLOPOULOS_C = 2.62206


def cap_mask(med, X):
    """eta(r) at points (zero without a "cap" entry in the medium)."""
    cap = med.get("cap")
    out = np.zeros(X[0].shape)
    if not cap:
        return out
    r0, R = float(cap["r0"]), float(cap["R"])
    for x in X:
        s = (np.abs(x) - r0) / (R - r0)
        on = s > 0.0
        sv = np.where(on, s, 0.0)
        if cap["kind"] == "poly":
            f = cap["eta0"] * sv ** cap["k"]
        elif cap["kind"] == "manolopoulos":
            if np.any(sv >= 1.0):
                raise ValueError("Manolopoulos mask evaluated at or beyond its end R")
            c = MANOLOPOULOS_C
            a, b = 1.0 - 16.0 / c ** 3, (1.0 - 17.0 / c ** 3) / c ** 2
            y = c * sv
            scale = (2.0 * np.pi / (R - r0)) ** 2 / (2.0 * cap.get("m", 1.0))
            f = scale * (a * y - b * y ** 3 + 4.0 / (c - y) ** 2 - 4.0 / (c + y) ** 2)
        else:
            raise ValueError(f"unknown CAP kind {cap['kind']}")
        out = out + np.where(on, f, 0.0)
    return out


# ------------------------------------------------------------------ 1-D
def _assemble_pairs(first, Ba, Bb, f, w, n):
    """sum over elements of local matrices loc[e,a,b] = sum_q w f Ba Bb, into an n x n CSR."""
    loc = np.einsum("eq,eqa,eqb->eab", w * f, Ba, Bb)
    E, P1, _ = loc.shape
    rows = first[:, None, None] + np.arange(P1)[None, :, None]
    cols = first[:, None, None] + np.arange(P1)[None, None, :]
    rows = np.broadcast_to(rows, loc.shape)
    cols = np.broadcast_to(cols, loc.shape)
    return sp.coo_matrix((loc.ravel(), (rows.ravel(), cols.ravel())), shape=(n, n)).tocsr()


def _trim(A):
    n = A.shape[0]
    return A[1:n - 1, 1:n - 1].tocsr()


def assemble_1d(knots, p, nq, med, trim=True):
    """1-D matrices {S, T, V, H0, D, G, K} (CSR, Dirichlet-trimmed unless trim=False)."""
    t = np.asarray(knots, dtype=np.float64)
    n = len(t) - p - 1
    q = quadrature_1d(t, p, nq)
    X = (q["x"],)
    w, B, dB, first = q["w"], q["val"], q["der"], q["first"]
    one = np.ones_like(q["x"])
    minv = inv_mass(med, X)
    out = {
        "S": _assemble_pairs(first, B, B, one, w, n),
        "T": _assemble_pairs(first, dB, dB, 0.5 * minv, w, n),
        "V": _assemble_pairs(first, B, B, potential(med, X), w, n),
        "D": [_assemble_pairs(first, B, B, q["x"], w, n)],
        "G": [_assemble_pairs(first, B, B, minv * grad_potential(med, X, 0), w, n)],
        "K": _assemble_pairs(first, B, B, minv, w, n),
        "W": _assemble_pairs(first, B, B, cap_mask(med, X), w, n),
        "M": [(_assemble_pairs(first, B, dB, minv, w, n) - _assemble_pairs(first, dB, B, minv, w, n)).tocsr()],
    }
    if trim:
        out = {k: ([_trim(m) for m in v] if isinstance(v, list) else _trim(v)) for k, v in out.items()}
    out["H0"] = (out["T"] + out["V"]).tocsr()
    out["dim"] = 1
    return out


# ------------------------------------------------------------------ 2-D / 3-D
def assemble_nd(knots_list, p_list, nq_list, med, trim=True, elements=None):
    """Tensor-product matrices by full tensor quadrature on every element (CSR).

    Returns {S, T, V, H0, D[axis], G[axis], K, dim, shape} with shape the per-axis
    number of (trimmed) functions; linear index x fastest. `elements` (optional): the
    tensor elements (tuples of per-axis element indices) to integrate over instead of all;
    the rows of functions whose support lies in them are then complete (assemble_nd_rows)."""
    dim = len(knots_list)
    qs = [quadrature_1d(np.asarray(k, dtype=np.float64), p, nq) for k, p, nq in zip(knots_list, p_list, nq_list)]
    nfun = [len(k) - p - 1 for k, p in zip(knots_list, p_list)]
    N = int(np.prod(nfun))
    acc = {"S": [], "T": [], "V": [], "K": [], "W": []}
    for a in range(dim):
        acc[f"D{a}"] = []
        acc[f"G{a}"] = []
        acc[f"M{a}"] = []
    rows_all, cols_all = [], []
    # loop over tensor elements (one numpy block per element row along the slowest axis)
    E = [len(q["span"]) for q in qs]
    for idx in (product(*[range(e) for e in E]) if elements is None else elements):
        # local points: meshgrid over axes (axis 0 fastest in linear index; here arrays indexed [q0,q1,...])
        pts = np.meshgrid(*[qs[a]["x"][idx[a]] for a in range(dim)], indexing="ij")
        wts = np.ones_like(pts[0])
        for a in range(dim):
            shape = [1] * dim
            shape[a] = -1
            wts = wts * qs[a]["w"][idx[a]].reshape(shape)
        X = tuple(pts)
        minv = inv_mass(med, X)
        Vq = potential(med, X)
        # local tensor basis values: val[a][q, r]
        vals = [qs[a]["val"][idx[a]] for a in range(dim)]
        ders = [qs[a]["der"][idx[a]] for a in range(dim)]
        P1 = [v.shape[1] for v in vals]
        # build full local basis arrays Bl[q..., r0, r1, ...]
        def tensor(fs):
            out = fs[0]
            for a in range(1, dim):
                out = np.multiply.outer(out, fs[a])
            # outer of (Q0,R0),(Q1,R1) -> (Q0,R0,Q1,R1): reorder to (Q0,Q1,...,R0,R1,...)
            order = [2 * a for a in range(dim)] + [2 * a + 1 for a in range(dim)]
            return np.transpose(out, order)
        Bl = tensor(vals)
        nl = int(np.prod(P1))
        Bf = Bl.reshape(wts.size, nl)
        dBf = []
        for a in range(dim):
            fs = [ders[b] if b == a else vals[b] for b in range(dim)]
            dBf.append(tensor(fs).reshape(wts.size, nl))
        wv = wts.reshape(-1)
        def loc(f, L, R):
            return np.einsum("q,qa,qb->ab", wv * f.reshape(-1), L, R)
        acc["S"].append(loc(np.ones_like(wv), Bf, Bf))
        tl = sum(loc(0.5 * minv, dBf[a], dBf[a]) for a in range(dim))
        acc["T"].append(tl)
        acc["V"].append(loc(Vq, Bf, Bf))
        acc["K"].append(loc(minv, Bf, Bf))
        acc["W"].append(loc(cap_mask(med, X), Bf, Bf))
        for a in range(dim):
            acc[f"M{a}"].append(loc(minv, Bf, dBf[a]) - loc(minv, dBf[a], Bf))
            acc[f"D{a}"].append(loc(X[a], Bf, Bf))
            acc[f"G{a}"].append(loc(minv * grad_potential(med, X, a), Bf, Bf))
        # global indices of local functions (x fastest)
        first = [qs[a]["first"][idx[a]] for a in range(dim)]
        gi = np.zeros(P1, dtype=np.int64)
        stride = 1
        for a in range(dim):
            shape = [1] * dim
            shape[a] = -1
            gi = gi + (first[a] + np.arange(P1[a])).reshape(shape) * stride
            stride *= nfun[a]
        gi = gi.reshape(-1)
        rows_all.append(np.repeat(gi, nl))
        cols_all.append(np.tile(gi, nl))
    rows = np.concatenate(rows_all)
    cols = np.concatenate(cols_all)

    def build(key):
        data = np.concatenate([m.reshape(-1) for m in acc[key]])
        return sp.coo_matrix((data, (rows, cols)), shape=(N, N)).tocsr()

    out = {"S": build("S"), "T": build("T"), "V": build("V"), "K": build("K"), "W": build("W"),
           "D": [build(f"D{a}") for a in range(dim)], "G": [build(f"G{a}") for a in range(dim)],
           "M": [build(f"M{a}") for a in range(dim)]}
    shape = list(nfun)
    if trim:
        keep = np.ones(N, dtype=bool)
        grid = np.indices(nfun[::-1]).reshape(dim, -1)[::-1]   # grid[a] = i_a for linear index (x fastest)
        for a in range(dim):
            keep &= (grid[a] > 0) & (grid[a] < nfun[a] - 1)
        sel = np.nonzero(keep)[0]

        def tr(A):
            return A[sel][:, sel].tocsr()
        out = {k: ([tr(m) for m in v] if isinstance(v, list) else tr(v)) for k, v in out.items()}
        shape = [n - 2 for n in nfun]
    out["H0"] = (out["T"] + out["V"]).tocsr()
    out["dim"] = dim
    out["shape"] = shape
    return out


def assemble_nd_rows(knots_list, p_list, nq_list, med, rows):
    """The matrices of assemble_nd (trimmed) with the given rows complete: the same element
    quadrature, restricted to the elements in the support of those rows' functions, so that
    single rows of a system too large to assemble can be checked. rows: trimmed linear indices
    (x fastest). The other rows hold partial sums and must not be used."""
    dim = len(knots_list)
    firsts = [quadrature_1d(np.asarray(k, dtype=np.float64), p, nq)["first"]
              for k, p, nq in zip(knots_list, p_list, nq_list)]
    ntrim = [len(k) - p - 1 - 2 for k, p in zip(knots_list, p_list)]
    elements = set()
    for j in rows:
        per_axis = []
        rest = int(j)
        for a in range(dim):
            i = rest % ntrim[a] + 1            # untrimmed index on axis a
            rest //= ntrim[a]
            f = firsts[a]
            per_axis.append(np.nonzero((f <= i) & (i <= f + p_list[a]))[0].tolist())
        elements.update(product(*per_axis))
    return assemble_nd(knots_list, p_list, nq_list, med, trim=True, elements=sorted(elements))


def to_band(A, p):
    """Dense LAPACK general-band storage ab[p + i - j, j] = A[i, j] (half bandwidth p)."""
    A = A.tocoo()
    n = A.shape[0]
    ab = np.zeros((2 * p + 1, n), dtype=A.dtype)
    keep = np.abs(A.row - A.col) <= p
    if not np.all(keep | (A.data == 0)):
        raise ValueError("matrix has entries outside the band")
    ab[p + A.row[keep] - A.col[keep], A.col[keep]] = A.data[keep]
    return ab
