"""GPU parity of the 2-D/3-D propagator (Kronecker + Gauss-point operator application,
preconditioned COCG) against the CPU oracle (full tensor quadrature, SuperLU per step).

Cases: separable HO (Kronecker terms only, plus a quadratic V at the Gauss points), the soft-core
atom (non-separable V), the elliptical quantum dot (position-dependent mass and step potential at
the Gauss points), and a 3-D soft-core atom; binary64 (rel-L2 <= 1e-9) and mixed precision (FP32
COCG inside binary64 refinement, rel-L2 <= 1e-8).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import assemble, eigen, propagate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tdz():
    import torch
    assert torch.cuda.is_available()
    import paper_2608_18472_b300 as m
    return m


def _case(name):
    if name == "ho2d":
        t = wl.knots_for_nsplines(-7.0, 7.0, 22, 3)
        return [t, t], 3, wl.ho_medium([1.0, 1.3]), 0.05, 30, 0.2
    if name == "softcore2d":
        t = wl.knots_for_nsplines(-12.0, 12.0, 26, 4)
        return [t, t], 4, wl.softcore_medium(0.5), 0.05, 30, 0.1
    if name == "dot2d":
        t = wl.knots_for_nsplines(-6.0, 6.0, 24, 3)
        med = wl.medium({"kind": "ellipse", "a": 3.0, "b": 2.0, "m_in": 0.5, "m_out": 1.0},
                        {"kind": "ellipse", "a": 3.0, "b": 2.0, "v_in": -1.0, "v_out": 0.0})
        return [t, t], 3, med, 0.1, 25, 0.15
    if name == "softcore3d":
        t = wl.knots_for_nsplines(-8.0, 8.0, 12, 3)
        return [t, t, t], 3, wl.softcore_medium(0.5), 0.05, 12, 0.1
    raise KeyError(name)


@pytest.mark.parametrize("name", ["ho2d", "softcore2d", "dot2d", "softcore3d"])
def test_nd_matches_oracle(tdz, name):
    knots, p, med, dt, nsteps, e0 = _case(name)
    dim = len(knots)
    m = assemble.assemble_nd(knots, [p] * dim, [p + 1] * dim, med)
    _, c0 = eigen.ground_state(m)
    t = wl.time_grid(dt, nsteps)
    field = wl.sin2_pulse(t, e0, 0.5, 1.0, ellipticity=0.3 if dim > 1 else 0.0, dim=dim)
    c, obs = propagate.cn_propagate(m, c0, field, dt, nsteps)
    ops = tdz.Ops([tdz.Basis(k, p, p + 1) for k in knots], med)
    assert ops.n == m["S"].shape[0]
    for prec, tol in ((tdz.FP64, 1e-9), (tdz.MIXED, 1e-8)):
        b = tdz.Batch([ops], [0], prec)
        b.set_state(0, c0)
        b.propagate(field.reshape(1, nsteps + 1, dim), dt, 0, nsteps)
        og, st = b.observe(0)
        cg = b.get_state(0)
        assert st == tdz.TDZ_OK, (prec, st)
        rel = np.linalg.norm(cg - c) / np.linalg.norm(c)
        assert rel < tol, (prec, rel)
        assert np.max(np.abs(og[:, 0] - obs[:, 0])) < 1e-12
        for col in range(1 + dim, 2 + 3 * dim):
            scale = max(1e-3, np.max(np.abs(obs[:, col])))
            assert np.max(np.abs(og[:, col] - obs[:, col])) < 10 * tol * scale, (prec, col)
