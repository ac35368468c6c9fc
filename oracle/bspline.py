"""B-spline basis by the Cox-de Boor recursion, and Gauss-Legendre rules.

TEST INFRASTRUCTURE (oracle). Paper: Sec. "Weak form" (open knot vectors with
ends repeated p+1 times, Dirichlet by dropping the first and last function) and
Sec. "Parallel assembly" (Gauss quadrature on knot spans, Jacobian mapping).

The recursion is evaluated literally:
    N_{i,0}(x) = 1 on [t_i, t_{i+1}),   else 0
    N_{i,k}(x) = (x - t_i)/(t_{i+k} - t_i) N_{i,k-1}(x)
               + (t_{i+k+1} - x)/(t_{i+k+1} - t_{i+1}) N_{i+1,k-1}(x)      (0/0 := 0)
    N'_{i,k}(x) = k/(t_{i+k} - t_i) N_{i,k-1}(x) - k/(t_{i+k+1} - t_{i+1}) N_{i+1,k-1}(x)
"""
from __future__ import annotations

import numpy as np


def gauss_legendre(nq: int):
    """nq-point Gauss-Legendre nodes and weights on [-1, 1] (numpy's leggauss)."""
    x, w = np.polynomial.legendre.leggauss(nq)
    return x, w


def _ratio(num, den):
    den = np.asarray(den, dtype=np.float64)
    safe = np.where(den == 0.0, 1.0, den)
    return np.where(den == 0.0, 0.0, num / safe)


def element_spans(knots: np.ndarray, p: int) -> np.ndarray:
    """Indices j of the non-empty knot spans [t_j, t_{j+1}) that carry elements."""
    n = len(knots) - p - 1
    j = np.arange(p, n)
    return j[knots[j + 1] > knots[j]]


def local_basis(knots: np.ndarray, p: int, span: np.ndarray, x: np.ndarray):
    """Values and first derivatives of the p+1 B-splines N_{span-p..span, p} at points x.

    span: (E,) span index per element, x: (E, Q) points inside those spans.
    Returns (val, der), each (E, Q, p+1); column r is function i = span - p + r.
    """
    t = np.asarray(knots, dtype=np.float64)
    E, Q = x.shape
    # degree 0: only N_{span,0} is nonzero inside the span
    prev = np.ones((E, Q, 1))
    for k in range(1, p + 1):
        cur = np.zeros((E, Q, k + 1))
        for r in range(k + 1):
            i = span - k + r                                  # function index at degree k
            left = prev[:, :, r - 1] if r - 1 >= 0 else 0.0    # N_{i,k-1}
            right = prev[:, :, r] if r <= k - 1 else 0.0       # N_{i+1,k-1}
            a = _ratio(x - t[i][:, None], (t[i + k] - t[i])[:, None])
            b = _ratio(t[i + k + 1][:, None] - x, (t[i + k + 1] - t[i + 1])[:, None])
            cur[:, :, r] = a * left + b * right
        if k == p:
            # derivative from the degree p-1 values
            der = np.zeros((E, Q, p + 1))
            for r in range(p + 1):
                i = span - p + r
                left = prev[:, :, r - 1] if r - 1 >= 0 else 0.0
                right = prev[:, :, r] if r <= p - 1 else 0.0
                der[:, :, r] = (_ratio(p, (t[i + p] - t[i])[:, None]) * left
                                - _ratio(p, (t[i + p + 1] - t[i + 1])[:, None]) * right)
        prev = cur
    if p == 0:
        der = np.zeros((E, Q, 1))
    return prev, der


def quadrature_1d(knots: np.ndarray, p: int, nq: int):
    """Per-element physical quadrature points, weights (w_q * J) and local basis tables.

    Returns dict with span (E,), x (E,Q), w (E,Q), val (E,Q,p+1), der (E,Q,p+1), first (E,)
    where first[e] = span[e] - p is the global index of column 0 of the local tables."""
    t = np.asarray(knots, dtype=np.float64)
    span = element_spans(t, p)
    xi, wi = gauss_legendre(nq)
    a, b = t[span], t[span + 1]
    half = 0.5 * (b - a)
    x = 0.5 * (a + b)[:, None] + half[:, None] * xi[None, :]
    w = half[:, None] * wi[None, :]
    val, der = local_basis(t, p, span, x)
    return {"span": span, "x": x, "w": w, "val": val, "der": der, "first": span - p}


def eval_all(knots: np.ndarray, p: int, x: np.ndarray):
    """Dense evaluation of all N_{i,p}(x) (N x len(x)) for small cases (the right end point
    x = t_last is assigned to the last non-empty span)."""
    t = np.asarray(knots, dtype=np.float64)
    n = len(t) - p - 1
    spans = element_spans(t, p)
    x = np.asarray(x, dtype=np.float64)
    idx = np.searchsorted(t[spans], x, side="right") - 1
    idx = np.clip(idx, 0, len(spans) - 1)
    sp = spans[idx]
    val, der = local_basis(t, p, sp, x[:, None])
    out = np.zeros((n, len(x)))
    dout = np.zeros((n, len(x)))
    for r in range(p + 1):
        out[sp - p + r, np.arange(len(x))] = val[:, 0, r]
        dout[sp - p + r, np.arange(len(x))] = der[:, 0, r]
    return out, dout
