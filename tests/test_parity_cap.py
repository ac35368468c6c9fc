"""GPU parity of the absorbing boundary layer (CAP matrix -i W of Sec. "Parallel assembly") against the
CPU oracle, in 1-D: A_n = S + tau W + i tau H_n stays complex symmetric, so the banded LDL^T and the
mixed refinement apply unchanged; the norm decays by the flux the layer absorbs. Both mask readings
(Manolopoulos, polynomial) in both precisions; the norm column must follow the oracle's absorption.
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


def _atom(kind, p=6, nspl=280, L=50.0):
    t = wl.knots_for_nsplines(-L, L, nspl, p)
    base = wl.softcore_medium(2.0)
    if kind == "manolopoulos":
        med = wl.with_cap(base, "manolopoulos", 0.5 * L, L, m=1.0)
    else:
        med = wl.with_cap(base, "poly", 0.5 * L, L, eta0=0.2, k=3.0)
    return t, med


@pytest.mark.parametrize("kind", ["manolopoulos", "poly"])
def test_cap_1d_ionising_pulse_matches_oracle(tdz, kind):
    """A strong 2-cycle pulse (E0 = 0.2, w = 0.25) drives part of the soft-core ground state into the layer
    (|x| > 25 on [-50, 50]): final state, norm
    (absorbed fraction), dipole and acceleration against the oracle (1e-9 binary64, 1e-8 mixed)."""
    p, dt, nsteps = 6, 0.05, 1200
    t, med = _atom(kind, p)
    m = assemble.assemble_1d(t, p, p + 1, med)
    assert abs(m["W"]).max() > 0
    _, c0 = eigen.ground_state(assemble.assemble_1d(t, p, p + 1, wl.softcore_medium(2.0)))
    field = wl.sin2_pulse(wl.time_grid(dt, nsteps), 0.2, 0.25, 2.0)
    c, obs = propagate.cn_propagate(m, c0, field, dt, nsteps)
    assert obs[-1, 4] < 0.99 * obs[0, 4]            # the layer has absorbed 1.7 % (poly) to 5 % of the norm
    ops = tdz.assemble_1d(t, p, med, p + 1)
    assert np.max(np.abs(ops.band("W") - np.stack([np.concatenate([np.zeros(d), m["W"].diagonal(-d)])
                                                    for d in range(p + 1)], axis=1))) < 1e-12 * abs(m["W"]).max()
    for prec, tol in ((tdz.FP64, 1e-9), (tdz.MIXED, 1e-8)):
        b = tdz.Batch([ops], [0], prec)
        b.set_state(0, c0)
        b.propagate(field.reshape(1, nsteps + 1, 1), dt, 0, nsteps)
        og, st = b.observe(0)
        assert st == tdz.TDZ_OK, (prec, st)
        cg = b.get_state(0)
        assert np.linalg.norm(cg - c) / np.linalg.norm(c) < tol, prec
        assert np.max(np.abs(og[:, 4] - obs[:, 4])) < tol, prec
        for col in (2, 3):
            assert np.max(np.abs(og[:, col] - obs[:, col])) < 10 * tol * max(1.0, np.max(np.abs(obs[:, col]))), (prec, col)
        del b


def test_cap_and_plain_geometries_in_one_batch(tdz):
    """A batch mixing a geometry with a layer and one without (same degree): every run follows its own
    oracle trajectory (the plain run keeps its norm to 1e-10 / 1e-8)."""
    p, dt, nsteps = 6, 0.05, 300
    t, med = _atom("manolopoulos", p, nspl=300, L=50.0)
    t2 = wl.knots_for_nsplines(-50.0, 50.0, 250, p)
    plain = wl.softcore_medium(2.0)
    mats = [assemble.assemble_1d(t, p, p + 1, med), assemble.assemble_1d(t2, p, p + 1, plain)]
    c0s = [eigen.ground_state(assemble.assemble_1d(t, p, p + 1, plain))[1], eigen.ground_state(mats[1])[1]]
    fields = [wl.sin2_pulse(wl.time_grid(dt, nsteps), e0, 0.25, 1.0) for e0 in (0.2, 0.15)]
    ops = [tdz.assemble_1d(t, p, med, p + 1), tdz.assemble_1d(t2, p, plain, p + 1)]
    order = [0, 1, 1, 0]
    for prec, tol, drift in ((tdz.FP64, 1e-9, 1e-10), (tdz.MIXED, 1e-8, 1e-8)):
        b = tdz.Batch(ops, order, prec)
        for i, g in enumerate(order):
            b.set_state(i, c0s[g])
        b.propagate(np.stack([fields[i % 2] for i in range(4)]), dt, 0, nsteps)
        for i, g in enumerate(order):
            c, obs = propagate.cn_propagate(mats[g], c0s[g], fields[i % 2], dt, nsteps)
            og, st = b.observe(i)
            assert st == tdz.TDZ_OK
            assert np.linalg.norm(b.get_state(i) - c) / np.linalg.norm(c) < tol, (prec, i)
            assert np.max(np.abs(og[:, 4] - obs[:, 4])) < tol, (prec, i)
            if g == 1:
                assert np.max(np.abs(og[:, 4] - og[0, 4])) < drift, (prec, i)
        del b


def test_cap_parameters_are_validated(tdz):
    t = wl.knots_for_nsplines(-20.0, 20.0, 60, 4)
    for cap in ({"kind": "manolopoulos", "r0": 10.0, "R": 15.0, "m": 1.0},     # ends inside the domain
                {"kind": "poly", "r0": 10.0, "R": 5.0, "eta0": 1.0, "k": 2.0},  # R < r0
                {"kind": "poly", "r0": 10.0, "R": 20.0, "eta0": -1.0, "k": 2.0}):
        med = dict(wl.softcore_medium(2.0))
        med["cap"] = cap
        with pytest.raises(tdz.TDZError) as ei:
            tdz.assemble_1d(t, 4, med, 5)
        assert ei.value.code == tdz.TDZ_EINVAL


def _nd_case(dim, kind):
    if dim == 2:
        p, L, nspl = 4, 12.0, 28
    else:
        p, L, nspl = 3, 9.0, 13
    t = wl.knots_for_nsplines(-L, L, nspl, p)
    base = wl.softcore_medium(0.5)
    if kind == "manolopoulos":
        med = wl.with_cap(base, "manolopoulos", 0.55 * L, L, m=1.0)
    else:
        med = wl.with_cap(base, "poly", 0.55 * L, L, eta0=0.3, k=2.0)
    return [t] * dim, p, base, med


@pytest.mark.parametrize("dim,kind", [(2, "manolopoulos"), (2, "poly"), (3, "manolopoulos")])
def test_cap_nd_matches_oracle(tdz, dim, kind):
    """2-D/3-D soft core with an absorbing layer on every axis (eta = sum of the axes' masks, so W = sum_a
    W_a (x) S (x) S, the separable term tau W_a beside i tau K_a in the Kronecker pass): a strong pulse
    drives part of the ground state into the layer; final state, norm and dipoles against the oracle for
    every operator form and preconditioner, both precisions."""
    knots, p, base, med = _nd_case(dim, kind)
    dt, nsteps = 0.05, 60 if dim == 2 else 30
    m = assemble.assemble_nd(knots, [p] * dim, [p + 1] * dim, med)
    assert abs(m["W"]).max() > 0
    _, c0 = eigen.ground_state(assemble.assemble_nd(knots, [p] * dim, [p + 1] * dim, base))
    field = wl.sin2_pulse(wl.time_grid(dt, nsteps), 0.3, 0.6, 1.0, ellipticity=0.3, dim=dim)
    c, obs = propagate.cn_propagate(m, c0, field, dt, nsteps)
    assert obs[-1, -1] < obs[0, -1] - 1e-6                      # absorption is visible
    ops = tdz.Ops([tdz.Basis(k, p, p + 1) for k in knots], med)
    assert np.max(np.abs(ops.band("W", 0))) > 0
    combos = [("auto", "auto"), ("quadrature", "lines")] + ([("stencil", "fd")] if dim == 2 else [])
    for prec, tol in ((tdz.FP64, 1e-9), (tdz.MIXED, 1e-8)):
        for op, pc in combos:
            b = tdz.Batch([ops], [0], prec)
            b.set_option(tdz.OPT_OPERATOR, {"auto": tdz.OPERATOR_AUTO, "quadrature": tdz.OPERATOR_QUADRATURE,
                                            "stencil": tdz.OPERATOR_STENCIL}[op])
            b.set_option(tdz.OPT_PRECOND, {"auto": tdz.PRECOND_AUTO, "lines": tdz.PRECOND_LINES, "fd": tdz.PRECOND_FD}[pc])
            b.set_state(0, c0)
            b.propagate(field.reshape(1, nsteps + 1, dim), dt, 0, nsteps)
            og, st = b.observe(0)
            assert st == tdz.TDZ_OK, (prec, op, pc, st)
            cg = b.get_state(0)
            assert np.linalg.norm(cg - c) / np.linalg.norm(c) < tol, (prec, op, pc)
            assert np.max(np.abs(og[:, -1] - obs[:, -1])) < tol, (prec, op, pc)
            for col in range(1 + dim, 1 + 2 * dim):
                assert np.max(np.abs(og[:, col] - obs[:, col])) < 10 * tol * max(1.0, np.max(np.abs(obs[:, col])))
            del b
