"""GPU parity of the per-step total dipole velocity J = c^H Vel c (Sec. "Currents and coherence dynamics",
Eq. velocity_op, Eq. vel_elem) against the oracle, both precisions: the Appendix A oscillator (closed form
-(E0/2) t sin t as well), the smooth Quesne mass, and a double quantum well (stepped mass) of the headline
batch shape."""
import math

import numpy as np
import pytest

import bench
import workloads as wl
from oracle import assemble, eigen, propagate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tdz():
    import torch
    assert torch.cuda.is_available()
    import paper_2608_18472_b300 as m
    return m


def _cases():
    e0 = 0.2
    wk = wl.driven_ho_1d(e0=e0, dt=0.01, t_end=10.0, L=20.0, nsplines=200, p=5)
    r = wk.runs[0]
    yield "driven_ho", r.knots, r.degree, r.medium, r.field, wk.dt, wk.nsteps, None
    t = wl.open_uniform_knots(-2.0, 30.0, 300, 7)
    yield "quesne", t, 7, wl.quesne_medium(), wl.sin2_pulse(wl.time_grid(0.01, 600), 0.05, 0.5, 1.0), 0.01, 600, None
    wq = wl.dqw_batch(n_geometries=1, fields_per_geometry=4, nsplines_range=(800, 900), nsteps=400)
    r = wq.runs[3]
    yield "dqw", r.knots, r.degree, r.medium, r.field, wq.dt, wq.nsteps, bench.initial_state(r, r.medium)


@pytest.mark.parametrize("case", list(range(3)), ids=["driven_ho", "quesne", "dqw"])
def test_current_matches_oracle(tdz, case):
    name, knots, p, med, field, dt, nsteps, c0 = list(_cases())[case]
    m = assemble.assemble_1d(knots, p, p + 1, med)
    if c0 is None:
        _, c0 = eigen.ground_state(m)
    c, obs, J = propagate.cn_propagate(m, c0, field, dt, nsteps, currents=True)
    if name == "driven_ho":
        assert np.max(np.abs(J[:, 0] + 0.1 * obs[:, 0] * np.sin(obs[:, 0]))) < 3e-4   # O(dt^2) at dt = 0.01
    scale = np.max(np.abs(J))
    assert scale > 0
    ops = tdz.assemble_1d(knots, p, med, p + 1)
    for prec, tol in ((tdz.FP64, 1e-9), (tdz.MIXED, 1e-8)):
        b = tdz.Batch([ops], [0], prec)
        b.set_option(tdz.OPT_CURRENT, 1)
        b.set_state(0, c0)
        b.propagate(field.reshape(1, nsteps + 1, 1), dt, 0, nsteps)
        og, st = b.observe(0)
        assert st == tdz.TDZ_OK
        Jg = b.observe_current(0)
        assert np.max(np.abs(Jg - J[:, 0])) < 10 * tol * scale, (name, prec, np.max(np.abs(Jg - J[:, 0])) / scale)
        assert np.max(np.abs(og[:, 2] - obs[:, 2])) < 10 * tol * max(1.0, np.max(np.abs(obs[:, 2])))
        del b


def test_current_option_errors(tdz):
    t = wl.knots_for_nsplines(-10.0, 10.0, 40, 4)
    ops = tdz.assemble_1d(t, 4, wl.softcore_medium(2.0), 5)
    b = tdz.Batch([ops], [0], tdz.FP64)
    with pytest.raises(tdz.TDZError):
        b.observe_current(0)          # not enabled
    with pytest.raises(tdz.TDZError):
        b.set_option(tdz.OPT_CURRENT, 2)
    ops2 = tdz.Ops([tdz.Basis(t, 4, 5)] * 2, wl.softcore_medium(0.5))
    with pytest.raises(tdz.TDZError) as ei:
        tdz.Batch([ops2], [0], tdz.FP64).set_option(tdz.OPT_CURRENT, 1)
    assert ei.value.code == tdz.TDZ_EUNSUPPORTED
