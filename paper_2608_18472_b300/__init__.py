"""Python binding of the TDSE-Z B300 propagator library (libtdz.so, C ABI in include/tdz.h).

Argument marshalling only: every step of the propagation runs in the library's CUDA
kernels. Importing this package loads the in-tree ``libtdz.so``; if it is missing the
import fails loudly (build it with ``python paper_2608_18472_b300/build.py``). There is
no CPU fallback.

Names follow the paper (arXiv 2608.18472): S (overlap, M in the paper), T (BenDaniel-Duke
kinetic), V, D (dipole), G/K (acceleration matrices), Crank-Nicolson propagation.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtdz.so")

TDZ_OK, TDZ_EINVAL, TDZ_ENOMEM, TDZ_ECUDA, TDZ_ENOCONV, TDZ_ENONFINITE, TDZ_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
FP64, MIXED = 0, 1
OPT_PRECOND, OPT_OPERATOR, OPT_APPLY_GROUPS, OPT_WAIT_TEST, OPT_CURRENT = 1, 2, 3, 4, 5
PRECOND_AUTO, PRECOND_LINES, PRECOND_FD = 0, 1, 2
OPERATOR_AUTO, OPERATOR_QUADRATURE, OPERATOR_STENCIL = 0, 1, 2
MAT = {"S": 0, "T": 1, "V": 2, "H0": 3, "D": 4, "G": 5, "K": 6, "W": 7, "VEL": 8}
_CAP = {"poly": 1, "manolopoulos": 2}
_MASS = {"const": 0, "quesne": 1, "layers": 2, "ellipse": 3}
_POT = {"zero": 0, "softcore": 1, "ho": 2, "quesne": 3, "layers": 4, "ellipse": 5, "h2p_softcore": 6}


class TDZError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what} failed with status {code}: {last_error()}")
        self.code = code


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} not found: build the CUDA library with `python paper_2608_18472_b300/build.py`")
_lib = C.CDLL(LIB_PATH)


class _Medium(C.Structure):
    _fields_ = [("mass_kind", C.c_int), ("pot_kind", C.c_int), ("mass_par", C.c_double * 4),
                ("pot_par", C.c_double * 4), ("nlayers", C.c_int), ("layer_bounds", C.POINTER(C.c_double)),
                ("layer_mass", C.POINTER(C.c_double)), ("layer_pot", C.POINTER(C.c_double)),
                ("cap_kind", C.c_int), ("cap_par", C.c_double * 4)]


_dp = C.POINTER(C.c_double)
_vp = C.c_void_p
_sig = {
    "tdz_last_error": (C.c_char_p, []),
    "tdz_basis_create": (C.c_int, [_dp, C.c_int64, C.c_int, C.c_int, C.POINTER(_vp)]),
    "tdz_basis_info": (C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "tdz_basis_eval": (C.c_int, [_vp, _dp, C.c_int64, _dp, _dp]),
    "tdz_basis_destroy": (None, [_vp]),
    "tdz_assemble": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(_Medium), C.POINTER(_vp)]),
    "tdz_ops_info": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "tdz_ops_band": (C.c_int, [_vp, C.c_int, C.c_int, _dp]),
    "tdz_ops_destroy": (None, [_vp]),
    "tdz_ground_state": (C.c_int, [_vp, _dp, _dp]),
    "tdz_batch_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int, _vp, C.POINTER(_vp)]),
    "tdz_batch_set_refinement": (C.c_int, [_vp, C.c_double, C.c_int]),
    "tdz_batch_info": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_size_t)]),
    "tdz_set_state": (C.c_int, [_vp, C.c_int, _vp]),
    "tdz_get_state": (C.c_int, [_vp, C.c_int, _vp]),
    "tdz_propagate": (C.c_int, [_vp, _vp, C.c_double, C.c_int64, C.c_int64]),
    "tdz_observe": (C.c_int, [_vp, C.c_int, _vp, C.POINTER(C.c_int)]),
    "tdz_refine_stats": (C.c_int, [_vp, _dp, _dp]),
    "tdz_batch_set_option": (C.c_int, [_vp, C.c_int, C.c_int]),
    "tdz_set_state_all": (C.c_int, [_vp, _vp]),
    "tdz_observe_all": (C.c_int, [_vp, _vp, C.POINTER(C.c_int)]),
    "tdz_krylov_stats": (C.c_int, [_vp, _dp]),
    "tdz_batch_tuning": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int), _dp]),
    "tdz_batch_precond_tuning": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int), _dp]),
    "tdz_batch_time_operator": (C.c_int, [_vp, C.c_int, C.c_int, _dp]),
    "tdz_batch_ground_state": (C.c_int, [_vp, C.c_int, C.c_double, C.c_double, C.c_int, _dp, C.POINTER(C.c_int), _dp]),
    "tdz_batch_destroy": (None, [_vp]),
    "tdz_observe_current": (C.c_int, [_vp, C.c_int, _vp]),
    "tdz_lowest_states": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, _dp, _dp, _dp, C.POINTER(C.c_int), _vp]),
    "tdz_populations": (C.c_int, [_vp, _dp, C.c_int, _dp, C.c_int64, _dp, _dp]),
    "tdz_device_rates": (C.c_int, [_dp, _dp]),
    "tdz_tc_axis_transform": (C.c_int, [_vp, _vp, C.c_int64, C.c_int, _vp, _vp, C.c_int, C.c_int64, C.c_int64, _vp,
                                        _vp, C.c_int, _vp]),
    "tdz_pdm_acceleration": (C.c_int, [_vp, _dp, C.c_int64, _dp]),
    "tdz_spectrum": (C.c_int, [_vp, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_double, C.c_double, C.c_int,
                               C.c_double, C.c_double, C.c_int64, _vp, _vp]),
    "tdz_harmonic_yields": (C.c_int, [_dp, C.c_int64, C.c_double, C.c_double, C.c_int64, C.c_double, C.c_int, _dp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def last_error() -> str:
    s = _lib.tdz_last_error()
    return s.decode() if s else ""


def _check(code: int, what: str):
    if code != TDZ_OK:
        raise TDZError(code, what)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _ptr(x) -> int:
    """Address of a numpy array (host) or a torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x.data_ptr())


class Basis:
    """B-spline basis on an open knot vector with an nquad-point Gauss rule per span."""

    def __init__(self, knots: Sequence[float], degree: int, nquad: Optional[int] = None):
        k = np.ascontiguousarray(knots, dtype=np.float64)
        h = _vp()
        _check(_lib.tdz_basis_create(_dptr(k), len(k), int(degree), int(nquad or degree + 1), C.byref(h)),
               "tdz_basis_create")
        self._h = h
        nf, ne, p, nq = C.c_int64(), C.c_int64(), C.c_int(), C.c_int()
        _check(_lib.tdz_basis_info(h, C.byref(nf), C.byref(ne), C.byref(p), C.byref(nq)), "tdz_basis_info")
        self.nfun, self.nelem, self.degree, self.nquad = nf.value, ne.value, p.value, nq.value

    def eval(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        val = np.zeros((self.nfun, len(x)))
        der = np.zeros((self.nfun, len(x)))
        _check(_lib.tdz_basis_eval(self._h, _dptr(x), len(x), _dptr(val), _dptr(der)), "tdz_basis_eval")
        return val, der

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.tdz_basis_destroy(self._h)
            self._h = None


def _medium_struct(med: Dict):
    m, v = med["mass"], med["potential"]
    s = _Medium()
    s.mass_kind = _MASS[m["kind"]]
    s.pot_kind = _POT[v["kind"]]
    keep = []
    mk, vk = m["kind"], v["kind"]
    if mk == "const":
        s.mass_par[0] = m["m"]
    elif mk == "quesne":
        s.mass_par[0] = m["a"]
    elif mk == "ellipse":
        for i, key in enumerate(("a", "b", "m_in", "m_out")):
            s.mass_par[i] = m[key]
    if vk == "softcore":
        s.pot_par[0], s.pot_par[1] = v.get("z", 1.0), v["eps"]
    elif vk == "ho":
        for i, w in enumerate(v["omega"]):
            s.pot_par[i] = w
    elif vk == "quesne":
        s.pot_par[0], s.pot_par[1] = v["a"], v["omega"]
    elif vk == "ellipse":
        for i, key in enumerate(("a", "b", "v_in", "v_out")):
            s.pot_par[i] = v[key]
    elif vk == "h2p_softcore":
        s.pot_par[0], s.pot_par[1] = v["R"], v["eps"]
    cap = med.get("cap")
    if cap:
        s.cap_kind = _CAP[cap["kind"]]
        s.cap_par[0], s.cap_par[1] = cap["r0"], cap["R"]
        if cap["kind"] == "poly":
            s.cap_par[2], s.cap_par[3] = cap["eta0"], cap["k"]
        else:
            s.cap_par[2] = cap.get("m", 1.0)
    if mk == "layers" or vk == "layers":
        b = np.ascontiguousarray(m.get("bounds", v.get("bounds")), dtype=np.float64)
        s.nlayers = len(b) - 1
        s.layer_bounds = _dptr(b)
        keep.append(b)
        if mk == "layers":
            lm = np.ascontiguousarray(m["m"], dtype=np.float64)
            s.layer_mass = _dptr(lm)
            keep.append(lm)
        if vk == "layers":
            lv = np.ascontiguousarray(v["V"], dtype=np.float64)
            s.layer_pot = _dptr(lv)
            keep.append(lv)
    return s, keep


class Ops:
    """Assembled Galerkin operators (S, T_BDD, V, H0, D, G, K) of one geometry."""

    def __init__(self, axes: Sequence[Basis], medium: Dict):
        arr = (_vp * len(axes))(*[a._h for a in axes])
        ms, keep = _medium_struct(medium)
        h = _vp()
        _check(_lib.tdz_assemble(arr, len(axes), C.byref(ms), C.byref(h)), "tdz_assemble")
        del keep
        self._h = h
        self._axes = list(axes)
        dim, shape, deg = C.c_int(), (C.c_int64 * 3)(), (C.c_int * 3)()
        _check(_lib.tdz_ops_info(h, C.byref(dim), shape, deg), "tdz_ops_info")
        self.dim = dim.value
        self.shape = [shape[i] for i in range(self.dim)]
        self.degree = [deg[i] for i in range(self.dim)]

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))

    def band(self, which: str, axis: int = 0) -> np.ndarray:
        out = np.zeros((self.shape[axis], self.degree[axis] + 1))
        _check(_lib.tdz_ops_band(self._h, MAT[which], axis, _dptr(out)), "tdz_ops_band")
        return out

    def pdm_acceleration(self, states) -> np.ndarray:
        """a_Q of Eq. aQ_definition for 1-D states (complex array [n] or [nstates, n]) (tdz_pdm_acceleration)."""
        c = np.atleast_2d(np.asarray(states, dtype=np.complex128))
        buf = np.ascontiguousarray(np.stack([c.real, c.imag], axis=2).reshape(-1))
        out = np.zeros(c.shape[0])
        _check(_lib.tdz_pdm_acceleration(self._h, _dptr(buf), c.shape[0], _dptr(out)), "tdz_pdm_acceleration")
        return out

    def populations(self, phi, states):
        """Projections on field-free eigenstates phi [nev, n] of states [nstates, n] (tdz_populations):
        returns (populations [nstates, nev], currents [nstates, 4] = J_tot, J_intra, J_inter, J_bc)."""
        def pack(z):
            z = np.atleast_2d(np.asarray(z, dtype=np.complex128))
            return np.ascontiguousarray(np.stack([z.real, z.imag], axis=2).reshape(-1)), z.shape[0]
        pb, nev = pack(phi)
        cb, ns = pack(states)
        pop = np.zeros((ns, nev))
        jd = np.zeros((ns, 4))
        _check(_lib.tdz_populations(self._h, _dptr(pb), nev, _dptr(cb), ns, _dptr(pop), _dptr(jd)), "tdz_populations")
        return pop, jd

    def ground_state(self):
        e = C.c_double()
        c = np.zeros(2 * self.n)
        _check(_lib.tdz_ground_state(self._h, C.byref(e), _dptr(c)), "tdz_ground_state")
        return e.value, c[0::2] + 1j * c[1::2]

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.tdz_ops_destroy(self._h)
            self._h = None


def device_rates():
    """FP32 and binary64 FMA throughput of the current device in flop/s (tdz_device_rates)."""
    a, b = C.c_double(), C.c_double()
    _check(_lib.tdz_device_rates(C.byref(a), C.byref(b)), "tdz_device_rates")
    return a.value, b.value


def tc_axis_transform(a_hi, a_lo, b, rows: int, k: int, ncols: int, plane_rows: int, plane_stride: int, out_hi,
                      out_lo=None, b_lo=None, tile_n: int = 0, stream: Optional[int] = None):
    """One fast-diagonalisation axis transform on the tensor cores (tdz_tc_axis_transform). The arrays are
    float32 device tensors: a_hi, a_lo [rows, k], b (and b_lo) [ncols, k]; the result goes to out_hi (and
    out_lo). With a_lo None, a_hi is the FP32 data and the kernel splits it in shared memory."""
    _check(_lib.tdz_tc_axis_transform(_vp(_ptr(a_hi)), _vp(_ptr(a_lo)) if a_lo is not None else None, int(rows), int(k), _vp(_ptr(b)),
                                      _vp(_ptr(b_lo)) if b_lo is not None else None, int(ncols), int(plane_rows),
                                      int(plane_stride), _vp(_ptr(out_hi)),
                                      _vp(_ptr(out_lo)) if out_lo is not None else None, int(tile_n),
                                      _vp(stream or 0)),
           "tdz_tc_axis_transform")


def lowest_states(ops: Sequence["Ops"], nstates: int = 1, stream: Optional[int] = None):
    """The nstates lowest eigenpairs of H0 c = eps S c of several 1-D geometries at once on the GPU
    (tdz_lowest_states). Returns (energies [nops, nstates], list of state arrays [nstates, n_g] complex,
    residuals [nops, nstates], iterations [nops])."""
    arr = (_vp * len(ops))(*[o._h for o in ops])
    sizes = [o.n for o in ops]
    en = np.zeros((len(ops), nstates))
    res = np.zeros((len(ops), nstates))
    st = np.zeros(2 * nstates * sum(sizes))
    its = (C.c_int * len(ops))()
    _check(_lib.tdz_lowest_states(arr, len(ops), int(nstates), _dptr(en), _dptr(st), _dptr(res), its, _vp(stream or 0)),
           "tdz_lowest_states")
    out, o = [], 0
    for n in sizes:
        blk = st[o:o + 2 * n * nstates].reshape(nstates, n, 2)
        out.append(blk[:, :, 0] + 1j * blk[:, :, 1])
        o += 2 * n * nstates
    return en, out, res, np.array(list(its))


def assemble_1d(knots, degree: int, medium: Dict, nquad: Optional[int] = None) -> Ops:
    return Ops([Basis(knots, degree, nquad)], medium)


def spectrum(signals, dt: float, w_lo: float, dw: float, nw: int, beta: float = 8.0, length_form: bool = False,
             stream: Optional[int] = None) -> np.ndarray:
    """Kaiser-windowed spectra S(w_j), w_j = w_lo + j dw, of the records in `signals` ([nsig, nt] or [nt],
    float64 numpy array, host) on the GPU (tdz_spectrum). length_form multiplies by w^4."""
    x = np.ascontiguousarray(np.atleast_2d(signals), dtype=np.float64)
    nsig, nt = x.shape
    S = np.zeros((nsig, int(nw)))
    _check(_lib.tdz_spectrum(_vp(_ptr(x)), nsig, nt, nt, 1, float(dt), float(beta), int(bool(length_form)),
                             float(w_lo), float(dw), int(nw), _vp(_ptr(S)), _vp(stream or 0)), "tdz_spectrum")
    return S


def harmonic_yields(S, w_lo: float, dw: float, omega0: float, qmax: int):
    """Yields of the odd harmonics q = 1, 3, ... <= qmax (tdz_harmonic_yields). Returns (q, Y[nsig, nq])."""
    S = np.ascontiguousarray(np.atleast_2d(S), dtype=np.float64)
    nsig, nw = S.shape
    nq = (int(qmax) + 1) // 2
    Y = np.zeros((nsig, nq))
    _check(_lib.tdz_harmonic_yields(_dptr(S), nsig, float(w_lo), float(dw), nw, float(omega0), int(qmax), _dptr(Y)),
           "tdz_harmonic_yields")
    return np.arange(1, 2 * nq, 2), Y


class Batch:
    """Independent runs propagated together on the current CUDA device, one persistent launch
    per propagate() call. `stream` is a raw cudaStream_t handle (int) or None."""

    def __init__(self, ops: Sequence[Ops], run_ops: Sequence[int], precision: int = FP64, stream: Optional[int] = None):
        arr = (_vp * len(ops))(*[o._h for o in ops])
        idx = (C.c_int * len(run_ops))(*[int(i) for i in run_ops])
        h = _vp()
        _check(_lib.tdz_batch_create(arr, len(ops), len(run_ops), idx, int(precision), _vp(stream or 0), C.byref(h)),
               "tdz_batch_create")
        self._h = h
        self._ops = list(ops)
        self.run_ops = list(run_ops)
        self.nruns = len(run_ops)
        self.precision = precision
        self.dim = ops[0].dim
        self._last_nsteps = 0
        n, dof, nb = C.c_int(), C.c_int64(), C.c_size_t()
        _check(_lib.tdz_batch_info(h, C.byref(n), C.byref(dof), C.byref(nb)), "tdz_batch_info")
        self.total_dof, self.device_bytes = dof.value, nb.value

    def set_refinement(self, tol: float, max_solves: int = 6):
        _check(_lib.tdz_batch_set_refinement(self._h, float(tol), int(max_solves)), "tdz_batch_set_refinement")

    def n_of(self, run: int) -> int:
        return self._ops[self.run_ops[run]].n

    def set_state(self, run: int, c):
        """c: complex numpy array (host) or an interleaved float64 torch tensor (host or device)."""
        if isinstance(c, np.ndarray) and np.iscomplexobj(c):
            buf = np.ascontiguousarray(np.stack([c.real, c.imag], axis=1).reshape(-1), dtype=np.float64)
            _check(_lib.tdz_set_state(self._h, run, _vp(_ptr(buf))), "tdz_set_state")
        else:
            _check(_lib.tdz_set_state(self._h, run, _vp(_ptr(c))), "tdz_set_state")

    def set_states(self, c):
        """All runs at once: c = every run's coefficients concatenated in run order, as a complex numpy
        array or an interleaved float64 array/tensor (host or device)."""
        if isinstance(c, np.ndarray) and np.iscomplexobj(c):
            buf = np.ascontiguousarray(np.stack([c.real, c.imag], axis=1).reshape(-1), dtype=np.float64)
            _check(_lib.tdz_set_state_all(self._h, _vp(_ptr(buf))), "tdz_set_state_all")
        else:
            _check(_lib.tdz_set_state_all(self._h, _vp(_ptr(c))), "tdz_set_state_all")

    def observe_all(self, out=None):
        """Observables of all runs [nruns, nsteps, 2+3dim] and their statuses. Returns (array, statuses)."""
        st = (C.c_int * self.nruns)()
        if out is None:
            out = np.zeros((self.nruns, self._last_nsteps, 2 + 3 * self.dim))
        _check(_lib.tdz_observe_all(self._h, _vp(_ptr(out)), st), "tdz_observe_all")
        return out, np.array(list(st))

    def get_state(self, run: int, out=None):
        if out is None:
            buf = np.zeros(2 * self.n_of(run))
            _check(_lib.tdz_get_state(self._h, run, _vp(_ptr(buf))), "tdz_get_state")
            return buf[0::2] + 1j * buf[1::2]
        _check(_lib.tdz_get_state(self._h, run, _vp(_ptr(out))), "tdz_get_state")
        return out

    def propagate(self, field, dt: float, step0: int, nsteps: int):
        """field: float64 [nruns, nsteps+1, dim] (numpy host array or torch tensor, host or device)."""
        if isinstance(field, np.ndarray):
            field = np.ascontiguousarray(field, dtype=np.float64)
            assert field.size == self.nruns * (nsteps + 1) * self.dim
        _check(_lib.tdz_propagate(self._h, _vp(_ptr(field)), float(dt), int(step0), int(nsteps)), "tdz_propagate")
        self._last_nsteps = nsteps

    def observe(self, run: int, out=None):
        """Observables [nsteps, 2+3dim]: t, E, d, a, norm. Returns (array, status)."""
        st = C.c_int()
        if out is None:
            out = np.zeros((self._last_nsteps, 2 + 3 * self.dim))
        _check(_lib.tdz_observe(self._h, run, _vp(_ptr(out)), C.byref(st)), "tdz_observe")
        return out, st.value

    def observe_current(self, run: int, out=None):
        """Total dipole velocity J = c^H Vel c after every step of the last propagate() (1-D, after
        set_option(OPT_CURRENT, 1))."""
        if out is None:
            out = np.zeros(self._last_nsteps)
        _check(_lib.tdz_observe_current(self._h, run, _vp(_ptr(out))), "tdz_observe_current")
        return out

    def refine_stats(self):
        mx, ns = C.c_double(), C.c_double()
        _check(_lib.tdz_refine_stats(self._h, C.byref(mx), C.byref(ns)), "tdz_refine_stats")
        return mx.value, ns.value

    def set_option(self, option: int, value: int):
        """2-D/3-D solver options: OPT_PRECOND (PRECOND_*), OPT_OPERATOR (OPERATOR_*) or
        OPT_APPLY_GROUPS (0 = autotuned, 8 or 16: variant of the fused FP32 2-D apply)."""
        _check(_lib.tdz_batch_set_option(self._h, int(option), int(value)), "tdz_batch_set_option")

    def tuning(self, geometry: int = 0):
        """Autotuner result of a 2-D mixed batch for one geometry: (chosen variant of the fused FP32
        apply, {variant: measured ms per apply}); (0, {}) where no FP32 stencil exists."""
        g = C.c_int()
        ms = np.zeros(2)
        _check(_lib.tdz_batch_tuning(self._h, int(geometry), C.byref(g), ms.ctypes.data_as(_dp)),
               "tdz_batch_tuning")
        return g.value, ({8: float(ms[0]), 16: float(ms[1])} if g.value else {})

    def precond_tuning(self, geometry: int = 0):
        """Autotuner result of the tensor-core fast-diagonalisation preconditioner of a 2-D/3-D mixed batch
        for one geometry: (chosen variant, [ms per preconditioner apply of variants 0..5]); variants 0-3:
        bit 0 = 256-column tiles (else 128), bit 1 = TF32 split in shared memory; variants 4, 5: 64-column
        tiles, split in memory / in shared memory. (-1, []) where it does not apply."""
        v = C.c_int()
        ms = np.zeros(6)
        _check(_lib.tdz_batch_precond_tuning(self._h, int(geometry), C.byref(v), ms.ctypes.data_as(_dp)),
               "tdz_batch_precond_tuning")
        return v.value, ([float(x) for x in ms] if v.value >= 0 else [])

    def time_operator(self, geometry: int = 0, reps: int = 3) -> float:
        """ms of one inner-solve operator apply y = A_n x (FP32 in mixed batches) for a run of the geometry,
        best of `reps` (tdz_batch_time_operator)."""
        ms = C.c_double()
        _check(_lib.tdz_batch_time_operator(self._h, int(geometry), int(reps), C.byref(ms)), "tdz_batch_time_operator")
        return ms.value

    def ground_state(self, run: int, sigma: float, tol: float = 1e-10, max_outer: int = 200):
        """Ground state of a 2-D/3-D run by shifted inverse iteration on the GPU (tdz_batch_ground_state;
        binary64 in a binary64 batch, FP32 accuracy in a mixed one), started from the run's current state,
        which it replaces (S-normalised). Returns (energy, outer iterations, relative eigen-residual)."""
        e, it, res = C.c_double(), C.c_int(), C.c_double()
        _check(_lib.tdz_batch_ground_state(self._h, int(run), float(sigma), float(tol), int(max_outer), C.byref(e),
                                           C.byref(it), C.byref(res)), "tdz_batch_ground_state")
        return e.value, it.value, res.value

    def krylov_stats(self) -> float:
        """Total Krylov iterations of all runs since creation (0 for 1-D batches)."""
        it = C.c_double()
        _check(_lib.tdz_krylov_stats(self._h, C.byref(it)), "tdz_krylov_stats")
        return it.value

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.tdz_batch_destroy(self._h)
            self._h = None
