"""GPU parity of the batched 1-D Crank-Nicolson propagator against the CPU oracle.

Both sides take the same seeded inputs from workloads.py (knots, media, fields) and the
oracle's ground state as initial condition. Tolerances:
  * binary64 path: relative L2 of the final coefficients <= 1e-9, norm drift <= 1e-10,
    observables within 1e-9 relative to their scale;
  * mixed path (FP32 factors + double-float refinement): per-step refinement to 1e-11,
    norm drift <= 1e-8 and harmonic-yield error <= 1e-3 up to the cutoff (HHG metric).
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import assemble, eigen, hhg, propagate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tdz():
    import torch
    assert torch.cuda.is_available()
    import paper_2608_18472_b300 as m
    return m


def _case(nspl, p, L=40.0, eps=2.0, e0=0.05, omega=0.3, dt=0.05, nsteps=200):
    knots = wl.knots_for_nsplines(-L, L, nspl, p)
    med = wl.softcore_medium(eps)
    field = wl.sin2_pulse(wl.time_grid(dt, nsteps), e0, omega, 2.0)
    return knots, med, field


def _oracle_run(knots, p, nq, med, field, dt, nsteps, c0=None):
    m = assemble.assemble_1d(knots, p, nq, med)
    if c0 is None:
        _, c0 = eigen.ground_state(m, sigma=-2.0, dense_max=3000)
    c, obs = propagate.cn_propagate(m, c0, field, dt, nsteps)
    return m, c0, c, obs


def _gpu_run(tdz, knots, p, nq, med, field, dt, nsteps, c0, precision, tol=None):
    ops = tdz.assemble_1d(knots, p, med, nq)
    b = tdz.Batch([ops], [0], precision)
    if tol is not None:
        b.set_refinement(tol)
    b.set_state(0, c0)
    b.propagate(field.reshape(1, nsteps + 1, 1), dt, 0, nsteps)
    obs, st = b.observe(0)
    return b.get_state(0), obs, st, b


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("nspl,p", [(10, 3), (24, 3), (60, 4), (151, 5), (333, 6), (1000, 7), (1100, 6)])
def test_fp64_matches_oracle_chunkings(tdz, nspl, p):
    """K = 1 (tiny), 2, several and 32 chunks, ragged last chunk (n not a multiple of K)."""
    dt, nsteps = 0.05, 120
    knots, med, field = _case(nspl, p, L=max(8.0, nspl * 0.08), dt=dt, nsteps=nsteps)
    m, c0, c, obs = _oracle_run(knots, p, p + 1, med, field, dt, nsteps)
    cg, og, st, _ = _gpu_run(tdz, knots, p, p + 1, med, field, dt, nsteps, c0, tdz.FP64)
    assert st == tdz.TDZ_OK
    assert _rel(cg, c) < 1e-9
    assert np.max(np.abs(og[:, 0] - obs[:, 0])) < 1e-12
    assert np.max(np.abs(og[:, 1] - obs[:, 1])) == 0.0
    for col in (2, 3, 4):
        scale = max(1e-3, np.max(np.abs(obs[:, col])))
        assert np.max(np.abs(og[:, col] - obs[:, col])) < 1e-9 * scale, col


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8])
def test_every_degree_both_precisions(tdz, p):
    dt, nsteps = 0.05, 60
    knots, med, field = _case(40 * p + 30, p, L=30.0, dt=dt, nsteps=nsteps)
    m, c0, c, obs = _oracle_run(knots, p, p + 1, med, field, dt, nsteps)
    cg, og, st, _ = _gpu_run(tdz, knots, p, p + 1, med, field, dt, nsteps, c0, tdz.FP64)
    assert st == tdz.TDZ_OK and _rel(cg, c) < 1e-9
    cm, om, stm, bm = _gpu_run(tdz, knots, p, p + 1, med, field, dt, nsteps, c0, tdz.MIXED)
    assert stm == tdz.TDZ_OK
    assert _rel(cm, c) < 1e-8
    assert np.max(np.abs(om[:, 4] - obs[:, 4])) < 1e-9


def test_batch_of_uneven_runs_matches_oracle(tdz):
    """Several DQW geometries of different sizes and fields in one launch (config-2 shape)."""
    wk = wl.dqw_batch(n_geometries=3, fields_per_geometry=2, nsplines_range=(500, 900), nsteps=150, seed=11)
    ops, ms, c0s = [], [], []
    for g in range(3):
        r = wk.runs[2 * g]
        ops.append(tdz.assemble_1d(r.knots, r.degree, r.medium, r.nquad))
        m = assemble.assemble_1d(r.knots, r.degree, r.nquad, r.medium)
        ms.append(m)
        c0s.append(eigen.ground_state(m, sigma=-1e-3, dense_max=0)[1])
    run_ops = [r.geometry for r in wk.runs]
    field = np.stack([r.field for r in wk.runs])
    for prec, tol in ((tdz.FP64, 1e-9), (tdz.MIXED, 1e-8)):
        b = tdz.Batch(ops, run_ops, prec)
        for i, r in enumerate(wk.runs):
            b.set_state(i, c0s[r.geometry])
        b.propagate(field, wk.dt, 0, wk.nsteps)
        for i, r in enumerate(wk.runs):
            c, obs = propagate.cn_propagate(ms[r.geometry], c0s[r.geometry], r.field, wk.dt, wk.nsteps)
            og, st = b.observe(i)
            assert st == tdz.TDZ_OK
            assert _rel(b.get_state(i), c) < tol
            assert np.max(np.abs(og[:, 4] - obs[:, 4])) < 1e-9
            assert np.max(np.abs(og[:, 2] - obs[:, 2])) < tol * max(1.0, np.max(np.abs(obs[:, 2])))


def _config1(nsteps=None):
    wk = wl.softcore_atom_1d(nsteps=nsteps)
    r = wk.runs[0]
    return wk, r


def test_config1_full_fp64_and_mixed(tdz):
    """The 1-D soft-core atom, 1000 order-7 splines, 8819 steps: FP64 rel-L2 <= 1e-9 and norm drift
    <= 1e-10; mixed: norm drift <= 1e-8 and HHG yields within 1e-3 up to the cutoff harmonic."""
    wk, r = _config1()
    m, c0, c, obs = _oracle_run(r.knots, r.degree, r.nquad, r.medium, r.field, wk.dt, wk.nsteps)
    cg, og, st, _ = _gpu_run(tdz, r.knots, r.degree, r.nquad, r.medium, r.field, wk.dt, wk.nsteps, c0, tdz.FP64)
    assert st == tdz.TDZ_OK
    assert _rel(cg, c) < 1e-9
    assert np.max(np.abs(og[:, 4] - 1.0)) < 1e-10
    cm, om, stm, bm = _gpu_run(tdz, r.knots, r.degree, r.nquad, r.medium, r.field, wk.dt, wk.nsteps, c0, tdz.MIXED)
    assert stm == tdz.TDZ_OK
    assert np.max(np.abs(om[:, 4] - 1.0)) < 1e-8
    w0, e0 = wk.notes["omega"], wk.notes["E0"]
    ip = -eigen.ground_state(m, sigma=-2.0, dense_max=3000)[0]
    qcut = int(math.floor(hhg.cutoff_harmonic(ip, e0, w0)))
    om_o, So = hhg.spectrum(obs[:, 3], wk.dt)
    _, Sm = hhg.spectrum(om[:, 3], wk.dt)
    qs, Yo = hhg.harmonic_yields(om_o, So, w0, qcut)
    _, Ym = hhg.harmonic_yields(om_o, Sm, w0, qcut)
    assert np.max(np.abs(Ym / Yo - 1)) < 1e-3


def test_h2p_hydrogenic_grid_both_precisions(tdz):
    """The 1-D H2+ workload (Sec. Molecular HHG) on a reduced hydrogenic grid: 3007 order-7 splines on
    [-400, 400] (spacing 0.2 a.u. inside |x| < 153, growing to 0.52), trapezoidal pulse, 600 steps
    from the ground state: binary64 rel-L2 <= 1e-9 and norm drift <= 1e-10, mixed <= 1e-8 and
    <= 1e-8, dipoles against the oracle's."""
    wk = wl.h2p_1d(nsplines=3007, l_max=400.0, nsteps=600)
    r = wk.runs[0]
    m = assemble.assemble_1d(r.knots, r.degree, r.nquad, r.medium)
    e0, c0 = eigen.ground_state(m, sigma=-1.2, dense_max=0)
    assert abs(e0 + 1.1026) < 5e-5
    c, obs = propagate.cn_propagate(m, c0, r.field, wk.dt, wk.nsteps)
    for prec, tol, drift in ((tdz.FP64, 1e-9, 1e-10), (tdz.MIXED, 1e-8, 1e-8)):
        cg, og, st, _ = _gpu_run(tdz, r.knots, r.degree, r.nquad, r.medium, r.field, wk.dt, wk.nsteps, c0, prec)
        assert st == tdz.TDZ_OK, prec
        assert _rel(cg, c) < tol, (prec, _rel(cg, c))
        assert np.max(np.abs(og[:, 4] - 1.0)) < drift, prec
        assert np.max(np.abs(og[:, 2] - obs[:, 2])) < 10 * tol * np.max(np.abs(obs[:, 2])), prec


def test_restart_and_state_roundtrip(tdz):
    dt, nsteps = 0.05, 80
    knots, med, field = _case(300, 6, L=40.0, dt=dt, nsteps=nsteps)
    m, c0, c, obs = _oracle_run(knots, 6, 7, med, field, dt, nsteps)
    ops = tdz.assemble_1d(knots, 6, med, 7)
    b = tdz.Batch([ops], [0], tdz.FP64)
    b.set_state(0, c0)
    assert np.array_equal(b.get_state(0), c0)
    b.propagate(field[:41].reshape(1, 41, 1), dt, 0, 40)
    o1, _ = b.observe(0)
    b.propagate(field[40:].reshape(1, 41, 1), dt, 40, 40)
    o2, _ = b.observe(0)
    assert _rel(b.get_state(0), c) < 1e-9
    assert np.allclose(np.vstack([o1, o2])[:, 0], obs[:, 0], atol=1e-12, rtol=0)


def test_field_on_device_equals_host(tdz):
    import torch
    dt, nsteps = 0.05, 50
    knots, med, field = _case(200, 5, dt=dt, nsteps=nsteps)
    ops = tdz.assemble_1d(knots, 5, med, 6)
    _, c0 = ops.ground_state()
    outs = []
    for dev in (False, True):
        b = tdz.Batch([ops], [0], tdz.MIXED)
        b.set_state(0, c0)
        f = field.reshape(1, nsteps + 1, 1)
        if dev:
            f = torch.from_numpy(np.ascontiguousarray(f)).cuda()
        b.propagate(f, dt, 0, nsteps)
        outs.append((b.get_state(0), b.observe(0)[0]))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])


def test_field_free_eigenstate_phase(tdz):
    """Field free, an eigenstate acquires exactly the Cayley phase ((1-i tau E)/(1+i tau E))^n."""
    knots = wl.knots_for_nsplines(-40, 40, 300, 6)
    med = wl.softcore_medium(2.0)
    m = assemble.assemble_1d(knots, 6, 7, med)
    e, c0 = eigen.ground_state(m)
    dt, nsteps = 0.05, 400
    field = np.zeros((1, nsteps + 1, 1))
    tau = dt / 2
    g = ((1 - 1j * tau * e) / (1 + 1j * tau * e)) ** nsteps
    for prec, tol in ((tdz.FP64, 1e-10), (tdz.MIXED, 1e-8)):
        ops = tdz.assemble_1d(knots, 6, med, 7)
        b = tdz.Batch([ops], [0], prec)
        b.set_state(0, c0)
        b.propagate(field, dt, 0, nsteps)
        assert np.linalg.norm(b.get_state(0) - g * c0) < tol


def test_invalid_arguments_are_rejected(tdz):
    knots, med, field = _case(100, 4)
    ops = tdz.assemble_1d(knots, 4, med, 5)
    b = tdz.Batch([ops], [0], tdz.FP64)
    bad = np.zeros(ops.n, dtype=complex)
    bad[3] = np.nan
    with pytest.raises(tdz.TDZError) as ei:
        b.set_state(0, bad)
    assert ei.value.code == tdz.TDZ_ENONFINITE
    with pytest.raises(tdz.TDZError) as ei:
        b.set_state(5, np.zeros(ops.n, dtype=complex))
    assert ei.value.code == tdz.TDZ_EINVAL
    with pytest.raises(tdz.TDZError) as ei:
        b.propagate(field[:11].reshape(1, 11, 1), -0.1, 0, 10)
    assert ei.value.code == tdz.TDZ_EINVAL
    with pytest.raises(tdz.TDZError):
        tdz.Batch([ops], [0], 7)


def test_batched_state_upload_and_observables_match_per_run_calls(tdz):
    """tdz_set_state_all / tdz_observe_all against tdz_set_state / tdz_observe on an uneven batch:
    identical states (the device split of a coefficient into hi + lo rounds exactly as the host one)
    and identical observables after propagation, in both precisions."""
    wk = wl.dqw_batch(n_geometries=3, fields_per_geometry=2, nsplines_range=(500, 900), nsteps=20, seed=5)
    ops = [tdz.assemble_1d(wk.runs[2 * g].knots, 6, wk.runs[2 * g].medium, 7) for g in range(3)]
    run_ops = [r.geometry for r in wk.runs]
    rng = np.random.default_rng(3)
    c0 = [rng.standard_normal(ops[g].n) + 1j * rng.standard_normal(ops[g].n) for g in run_ops]
    field = np.stack([r.field for r in wk.runs])
    for prec in (tdz.FP64, tdz.MIXED):
        a, b = tdz.Batch(ops, run_ops, prec), tdz.Batch(ops, run_ops, prec)
        for i, c in enumerate(c0):
            a.set_state(i, c)
        b.set_states(np.concatenate(c0))
        for i in range(len(c0)):
            assert np.array_equal(a.get_state(i), b.get_state(i)), (prec, i)
        a.propagate(field, wk.dt, 0, wk.nsteps)
        b.propagate(field, wk.dt, 0, wk.nsteps)
        obs_all, st_all = b.observe_all()
        for i in range(len(c0)):
            o, st = a.observe(i)
            assert st == st_all[i] == tdz.TDZ_OK
            assert np.array_equal(o, obs_all[i]), (prec, i)
            assert np.array_equal(a.get_state(i), b.get_state(i)), (prec, i)
    bad = np.concatenate(c0)
    bad[7] = np.nan
    with pytest.raises(tdz.TDZError) as ei:
        b.set_states(bad)
    assert ei.value.code == tdz.TDZ_ENONFINITE
