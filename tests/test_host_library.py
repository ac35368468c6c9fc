"""Host-side parts of the library (no GPU needed): exported C ABI, basis tables, one-pass band
assembly and the host ground state, each compared with the independent CPU oracle."""
import os
import re

import numpy as np
import pytest

import workloads as wl
from oracle import assemble, bspline, eigen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tdz():
    import paper_2608_18472_b300 as m
    return m


def test_library_exports_every_declared_symbol(tdz):
    import ctypes
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(tdz_\w+)\s*\(", txt, flags=re.M))
    assert len(names) >= 15
    lib = ctypes.CDLL(tdz.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("p", [1, 3, 6, 8])
def test_basis_tables_match_oracle(tdz, p):
    rng = np.random.default_rng(7)
    inner = np.sort(rng.uniform(-5, 5, 13))
    knots = np.concatenate([np.full(p + 1, -5.0), inner, np.full(p + 1, 5.0)])
    b = tdz.Basis(knots, p, p + 1)
    x = rng.uniform(-5, 5, 300)
    v, d = b.eval(x)
    vo, do = bspline.eval_all(knots, p, x)
    assert np.max(np.abs(v - vo)) < 1e-13
    assert np.max(np.abs(d - do)) < 1e-10 * max(1, np.max(np.abs(do)))


def _lower_band(A, p):
    A = A.toarray()
    n = A.shape[0]
    out = np.zeros((n, p + 1))
    for d in range(p + 1):
        out[d:, d] = np.diagonal(A, -d)
    return out


MEDIA = [
    ("softcore", lambda: (wl.knots_for_nsplines(-40, 40, 90, 5), 5, 6, wl.softcore_medium(2.0))),
    ("quesne", lambda: (wl.open_uniform_knots(-2.0, 50.0, 120, 7), 7, 10, wl.quesne_medium())),
    ("dqw", lambda: (wl.dqw_knots(wl.dqw_medium(10.0, 3.0, 0.24), 400, 6), 6, 7, wl.dqw_medium(10.0, 3.0, 0.24))),
    ("ho", lambda: (wl.knots_for_nsplines(-10, 10, 60, 4), 4, 5, wl.ho_medium([1.0]))),
    ("h2p", lambda: (wl.knots_for_nsplines(-60, 60, 150, 7), 7, 8,
                     wl.medium({"kind": "const", "m": 1.0}, {"kind": "h2p_softcore", "R": 2.0, "eps": 1.472}))),
    ("cap_manolopoulos", lambda: (wl.knots_for_nsplines(-40, 40, 120, 6), 6, 7,
                                  wl.with_cap(wl.softcore_medium(2.0), "manolopoulos", 22.0, 40.0, m=1.0))),
    ("cap_poly", lambda: (wl.dqw_knots(wl.dqw_medium(10.0, 3.0, 0.24), 400, 6), 6, 7,
                          wl.with_cap(wl.dqw_medium(10.0, 3.0, 0.24), "poly", 300.0, 1000.0, eta0=0.01, k=2.0))),
]


@pytest.mark.parametrize("name,make", MEDIA, ids=[m[0] for m in MEDIA])
def test_band_assembly_matches_oracle(tdz, name, make):
    knots, p, nq, med = make()
    ops = tdz.assemble_1d(knots, p, med, nq)
    ref = assemble.assemble_1d(knots, p, nq, med)
    for key in ("S", "T", "V", "H0", "K", "W"):
        a, b = ops.band(key), _lower_band(ref[key], p)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)) + 1e-300, key
    assert (np.max(np.abs(ops.band("W"))) > 0) == ("cap" in med)
    for key in ("D", "G"):
        a, b = ops.band(key), _lower_band(ref[key][0], p)
        assert np.max(np.abs(a - b)) <= 1e-12 * max(np.max(np.abs(b)), 1e-300) + 1e-300, key


def test_host_ground_state_matches_oracle(tdz):
    knots = wl.knots_for_nsplines(-60, 60, 200, 6)
    med = wl.softcore_medium(2.0)
    e, c = tdz.assemble_1d(knots, 6, med).ground_state()
    m = assemble.assemble_1d(knots, 6, 7, med)
    eo, co = eigen.ground_state(m)
    assert abs(e - eo) < 1e-12
    assert np.linalg.norm(c - co) < 1e-8


def test_errors_are_status_codes(tdz):
    with pytest.raises(tdz.TDZError) as ei:
        tdz.Basis([0.0, 1.0, 0.5, 2.0], 1)
    assert ei.value.code == tdz.TDZ_EINVAL
    with pytest.raises(tdz.TDZError) as ei:
        tdz.Basis(wl.open_uniform_knots(0, 1, 4, 3)[1:], 3)   # not open
    assert ei.value.code == tdz.TDZ_EINVAL
    b = tdz.Basis(wl.open_uniform_knots(0, 1, 6, 3), 3)
    with pytest.raises(tdz.TDZError) as ei:
        tdz.Ops([b, b], wl.dqw_medium(8.0, 4.0, 0.2))      # layered media are 1-D only
    assert ei.value.code == tdz.TDZ_EINVAL
    b2 = tdz.Basis(wl.open_uniform_knots(0, 1, 6, 2), 2)
    with pytest.raises(tdz.TDZError) as ei:
        tdz.Ops([b, b2], wl.ho_medium([1.0, 1.0]))          # mixed degrees across axes
    assert ei.value.code == tdz.TDZ_EUNSUPPORTED


def test_axis_factors_for_tensor_bases_match_oracle(tdz):
    """2-D/3-D assembly keeps the per-axis 1-D factors S, T1 = 1/2 <N'|N'> and D (Eq. tensor3d)."""
    tx = wl.knots_for_nsplines(-5, 5, 20, 4)
    ty = wl.knots_for_nsplines(-3, 4, 14, 4)
    ops = tdz.Ops([tdz.Basis(tx, 4, 5), tdz.Basis(ty, 4, 5)], wl.softcore_medium(0.5))
    assert ops.dim == 2 and ops.shape == [18, 12]
    for a, t in enumerate((tx, ty)):
        ref = assemble.assemble_1d(t, 4, 5, wl.medium({"kind": "const", "m": 1.0}, {"kind": "zero"}))
        assert np.max(np.abs(ops.band("S", a) - _lower_band(ref["S"], 4))) < 1e-13
        assert np.max(np.abs(ops.band("T", a) - _lower_band(ref["T"], 4))) < 1e-12
        assert np.max(np.abs(ops.band("D", a) - _lower_band(ref["D"][0], 4))) < 1e-13


def test_harmonic_yields_match_oracle(tdz):
    """tdz_harmonic_yields (host) against the oracle's trapezoid yields on the oracle's own FFT grid, for a
    record with odd harmonics spanning ten decades (Sec. "Dipoles")."""
    from oracle import hhg
    dt, w0 = 0.05, 0.057
    t = np.arange(9000) * dt
    sig = sum(10.0 ** (-(q - 1) / 2) * np.sin(q * w0 * t + 0.3 * q) for q in range(1, 22, 2))
    om, S = hhg.spectrum(sig, dt, length_form=True)
    qs, Yo = hhg.harmonic_yields(om, S, w0, 21)
    q2, Y = tdz.harmonic_yields(S, 0.0, om[1] - om[0], w0, 21)
    assert np.array_equal(qs, q2)
    assert np.max(np.abs(Y[0] / Yo - 1)) < 1e-12


def test_velocity_band_and_pdm_acceleration_match_oracle(tdz):
    """The velocity matrix's antisymmetric part M (Eq. vel_elem, Vel = -(i/2) M) of a smooth and of a
    stepped position-dependent mass, and a_Q (Eq. aQ_definition) of a few states, against the oracle."""
    from oracle import propagate
    cases = [(wl.open_uniform_knots(-2.0, 30.0, 200, 7), 7, 8, wl.quesne_medium()),
             (wl.dqw_knots(wl.dqw_medium(10.0, 3.0, 0.24), 500, 6), 6, 7, wl.dqw_medium(10.0, 3.0, 0.24))]
    rng = np.random.default_rng(11)
    for knots, p, nq, med in cases:
        ops = tdz.assemble_1d(knots, p, med, nq)
        ref = assemble.assemble_1d(knots, p, nq, med)
        M = ref["M"][0]
        a, b = ops.band("VEL"), _lower_band(M, p)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
        assert np.all(a[:, 0] == 0.0)
        states = [rng.standard_normal(ops.n) + 1j * rng.standard_normal(ops.n) for _ in range(3)]
        aq = ops.pdm_acceleration(np.stack(states))
        for x, v in zip(states, aq):
            r = propagate.a_quantum(ref, x)
            assert abs(v - r) <= 1e-10 * max(1.0, abs(r)), (v, r)


def test_populations_and_current_decomposition(tdz):
    """tdz_populations against the oracle: the driven oscillator of Appendix A populates its levels as a
    coherent state (P_n = e^{-|a|^2} |a|^{2n} / n!), and J_tot = J_intra + J_inter + J_bc with J_intra = 0
    for real eigenstates (Sec. "Currents and coherence dynamics")."""
    import math
    from oracle import propagate
    e0 = 0.1
    wk = wl.driven_ho_1d(e0=e0, dt=0.01, t_end=6.0, L=20.0, nsplines=200, p=5)
    r = wk.runs[0]
    m = assemble.assemble_1d(r.knots, r.degree, r.nquad, r.medium)
    w, v = eigen.lowest_states(m, 6)
    c, obs, J = propagate.cn_propagate(m, v[:, 0], r.field, wk.dt, wk.nsteps, currents=True)
    ops = tdz.assemble_1d(r.knots, r.degree, r.medium, r.nquad)
    pop, jd = ops.populations(v.T, c)
    T = obs[-1, 0]
    a2 = e0 ** 2 / 8 * (T * T + math.sin(T) ** 2 - T * math.sin(2 * T))
    for k in range(4):
        assert abs(pop[0, k] - math.exp(-a2) * a2 ** k / math.factorial(k)) < 2e-4
    ref = np.abs(v.conj().T @ (m["S"] @ c)) ** 2
    assert np.allclose(pop[0], ref, rtol=0, atol=1e-13)
    assert abs(jd[0, 0] - J[-1, 0]) < 1e-12
    assert abs(jd[0, 1]) < 1e-14
    assert abs(jd[0, 0] - jd[0, 1] - jd[0, 2] - jd[0, 3]) < 1e-14
    # almost all of the coherent state lives in the six lowest levels: the remainder current is small
    assert abs(jd[0, 3]) < 1e-3 * abs(jd[0, 0])
