"""Seeded synthetic inputs for the TDSE-Z Crank-Nicolson propagator.

This module defines *inputs only*: knot vectors, media (mass / potential
descriptions by kind and parameters), time grids and laser-field samples. It
holds none of the method's arithmetic (no basis functions, no quadrature, no
matrices, no propagation), so that the CPU oracle and the CUDA library can
both be fed from it without sharing any computation.

Workload shapes follow the paper (arXiv 2608.18472):
  * atomic soft-core models and HHG drivers (Sec. "Molecular HHG"),
  * the GaAs/Al0.3Ga0.7As double quantum well (Sec. "Double quantum well
    structure"), with knots placed on every material interface,
  * mid-infrared Keldysh-regime fields (Sec. "Conclusion": lambda = 10 um,
    E_g = 1.42 eV, gamma from 2.3 to 0.5),
  * the resonantly driven harmonic oscillator of Appendix A.
All random choices draw from numpy.random.default_rng(seed).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

# ---------------------------------------------------------------- units (a.u.)
HARTREE_EV = 27.211386245988
BOHR_NM = 0.052917721090          # 1 bohr in nm  (1 nm = 18.8973 bohr)
NM = 1.0 / BOHR_NM                # bohr per nm
I_AU_WCM2 = 3.50944758e16         # intensity of E = 1 a.u. in W/cm^2
SEED = 20261202


def omega_from_nm(lam_nm: float) -> float:
    """Photon energy in Hartree for a wavelength in nm (hbar*omega = 45.5634/lambda[nm])."""
    return 45.56335252907954 / lam_nm


def e0_from_intensity(i_wcm2: float) -> float:
    """Peak field in a.u. for an intensity in W/cm^2."""
    return math.sqrt(i_wcm2 / I_AU_WCM2)


# ---------------------------------------------------------------- knots
def open_uniform_knots(a: float, b: float, n_elem: int, p: int) -> np.ndarray:
    """Open knot vector on [a, b] with n_elem equal spans (ends repeated p+1 times)."""
    inner = np.linspace(a, b, n_elem + 1)
    return np.concatenate([np.full(p, a), inner, np.full(p, b)])


def open_piecewise_knots(breaks: Sequence[float], counts: Sequence[int], p: int) -> np.ndarray:
    """Open knot vector with uniform spans inside each region [breaks[r], breaks[r+1]].

    Every break point is a knot, so material interfaces coincide with element
    boundaries and no Gauss point ever sits on an interface."""
    assert len(breaks) == len(counts) + 1
    pts: List[float] = [breaks[0]]
    for r, c in enumerate(counts):
        seg = np.linspace(breaks[r], breaks[r + 1], int(c) + 1)[1:]
        pts.extend(seg.tolist())
    inner = np.asarray(pts)
    return np.concatenate([np.full(p, breaks[0]), inner, np.full(p, breaks[-1])])


def knots_for_nsplines(a: float, b: float, nsplines: int, p: int) -> np.ndarray:
    """Uniform open knots giving exactly `nsplines` B-splines (boundary functions included)."""
    return open_uniform_knots(a, b, nsplines - p, p)



def hydrogenic_knots(l_max: float, r1: float, n_lin: int, n_exp: int, p: int) -> np.ndarray:
    """Symmetric open knots on [-l_max, l_max] from the hydrogenic grading (Tab. gradings):
    r_i = i r1 for i <= n_lin, then r_i = r_cross exp((i - n_lin) ln(l_max / r_cross) / n_exp),
    r_cross = n_lin r1, up to i = n_lin + n_exp; mirrored to x < 0 (2 (n_lin + n_exp) elements)."""
    r_cross = n_lin * r1
    lin = r1 * np.arange(1, n_lin + 1, dtype=np.float64)
    i = np.arange(1, n_exp + 1, dtype=np.float64)
    ex = r_cross * np.exp(i * math.log(l_max / r_cross) / n_exp)
    ex[-1] = l_max
    pos = np.concatenate([lin, ex])
    inner = np.concatenate([-pos[::-1], [0.0], pos])
    return np.concatenate([np.full(p, -l_max), inner, np.full(p, l_max)])

# ---------------------------------------------------------------- media
def medium(mass: Dict, potential: Dict) -> Dict:
    return {"mass": dict(mass), "potential": dict(potential)}


def softcore_medium(eps: float, z: float = 1.0) -> Dict:
    """Constant unit mass, V = -z / sqrt(|r|^2 + eps)."""
    return medium({"kind": "const", "m": 1.0}, {"kind": "softcore", "z": z, "eps": eps})


def with_cap(med: Dict, kind: str, r0: float, R: float, **par) -> Dict:
    """A copy of `med` with an absorbing layer (complex absorbing potential -i eta) in r0 < |x_a| < R on
    every axis: kind "poly" (eta0, k) or "manolopoulos" (m, the mass in the layer; R must be the edge)."""
    out = {"mass": dict(med["mass"]), "potential": dict(med["potential"])}
    cap = {"kind": kind, "r0": float(r0), "R": float(R)}
    cap.update({k: float(v) for k, v in par.items()})
    out["cap"] = cap
    return out


def ho_medium(omega: Sequence[float]) -> Dict:
    """Constant unit mass, V = 1/2 sum_a omega_a^2 x_a^2."""
    return medium({"kind": "const", "m": 1.0}, {"kind": "ho", "omega": list(map(float, omega))})


def quesne_medium(a: float = 2.0, omega: float = 1.0) -> Dict:
    """Quesne PDM oscillator: m(x) = (1 + x/a)^-1, V = 1/2 * a w^2 x^2 / (4 (x + a))."""
    return medium({"kind": "quesne", "a": a}, {"kind": "quesne", "a": a, "omega": omega})


def dqw_medium(lw_nm: float, wb_nm: float, v0_ev: float, m_w: float = 0.067, m_b: float = 0.092,
               outer_nm: float = 30.0) -> Dict:
    """Symmetric double quantum well, piecewise constant mass and band edge.

    Regions (nm): outer barrier | well | central barrier | well | outer barrier,
    centred on x = 0; returned with the break points in bohr."""
    half_b = 0.5 * wb_nm
    b_nm = [-(half_b + lw_nm + outer_nm), -(half_b + lw_nm), -half_b, half_b, half_b + lw_nm,
            half_b + lw_nm + outer_nm]
    bounds = [x * NM for x in b_nm]
    v0 = v0_ev / HARTREE_EV
    return medium({"kind": "layers", "bounds": bounds, "m": [m_b, m_w, m_b, m_w, m_b]},
                  {"kind": "layers", "bounds": bounds, "V": [v0, 0.0, v0, 0.0, v0]})


def ellipse_dot_medium(a_nm: float, b_nm: float, m_in: float = 0.067, m_out: float = 0.092,
                       dv_ev: float = 0.24) -> Dict:
    """2-D quantum dot: inside x^2/a^2 + y^2/b^2 < 1 (GaAs), outside the barrier material."""
    return medium({"kind": "ellipse", "a": a_nm * NM, "b": b_nm * NM, "m_in": m_in, "m_out": m_out},
                  {"kind": "ellipse", "a": a_nm * NM, "b": b_nm * NM, "v_in": 0.0, "v_out": dv_ev / HARTREE_EV})


# ---------------------------------------------------------------- fields
def sin2_pulse(t: np.ndarray, e0: float, omega: float, ncycles: float, cep: float = 0.0,
               ellipticity: float = 0.0, dim: int = 1) -> np.ndarray:
    """E(t) = E0 sin^2(pi t/T) [sin(w t + cep) x + eps cos(w t + cep) y] / sqrt(1 + eps^2), 0 after T.

    Returns shape (len(t), dim)."""
    T = ncycles * 2.0 * math.pi / omega
    env = np.where((t >= 0) & (t <= T), np.sin(math.pi * t / T) ** 2, 0.0)
    scale = e0 / math.sqrt(1.0 + ellipticity ** 2)
    out = np.zeros((t.shape[0], dim))
    out[:, 0] = scale * env * np.sin(omega * t + cep)
    if dim > 1:
        out[:, 1] = scale * ellipticity * env * np.cos(omega * t + cep)
    return out


def trapezoid_pulse(t: np.ndarray, e0: float, omega: float, ramp_cycles: float, flat_cycles: float,
                    dim: int = 1) -> np.ndarray:
    """Linear ramp up / flat top / linear ramp down, carrier sin(w t); along x."""
    Tc = 2.0 * math.pi / omega
    r, f = ramp_cycles * Tc, flat_cycles * Tc
    env = np.clip(np.minimum(t / r, (2 * r + f - t) / r), 0.0, 1.0)
    out = np.zeros((t.shape[0], dim))
    out[:, 0] = e0 * env * np.sin(omega * t)
    return out


def resonant_sine(t: np.ndarray, e0: float, dim: int = 1) -> np.ndarray:
    """Appendix A drive: E(t) = E0 sin(t) along x."""
    out = np.zeros((t.shape[0], dim))
    out[:, 0] = e0 * np.sin(t)
    return out


def time_grid(dt: float, nsteps: int) -> np.ndarray:
    """Sample times t_n = n dt, n = 0..nsteps (nsteps+1 samples)."""
    return dt * np.arange(nsteps + 1, dtype=np.float64)


def keldysh_e0(gamma: float, omega: float, m_eff: float = 0.067, e_gap_ev: float = 1.42) -> float:
    """Field amplitude for a Keldysh parameter gamma = omega sqrt(m* E_g) / E0."""
    return omega * math.sqrt(m_eff * e_gap_ev / HARTREE_EV) / gamma


# ---------------------------------------------------------------- runs / configs
@dataclass
class Run1D:
    knots: np.ndarray
    degree: int
    nquad: int
    medium: Dict
    field: np.ndarray          # (nsteps+1, 1)
    dt: float
    geometry: int = 0          # runs with equal geometry share knots and medium


@dataclass
class Workload:
    name: str
    runs: List[Run1D]
    nsteps: int
    dt: float
    notes: Dict = field(default_factory=dict)


def softcore_atom_1d(nsplines: int = 1000, p: int = 7, L: float = 200.0, eps: float = 2.0,
                     e0: float = 0.0534, omega: float = 0.057, ncycles: float = 4.0, dt: float = 0.05,
                     nsteps: Optional[int] = None, nquad: Optional[int] = None) -> Workload:
    """1-D soft-core atom V = -1/sqrt(x^2+eps) on [-L, L], sin^2 pulse; the single-run HHG case."""
    T = ncycles * 2 * math.pi / omega
    if nsteps is None:
        nsteps = int(math.ceil(T / dt - 1e-9))
    t = time_grid(dt, nsteps)
    run = Run1D(knots_for_nsplines(-L, L, nsplines, p), p, nquad or p + 1, softcore_medium(eps),
                sin2_pulse(t, e0, omega, ncycles), dt)
    return Workload("softcore_atom_1d", [run], nsteps, dt,
                    {"nsplines": nsplines, "p": p, "L": L, "eps": eps, "E0": e0, "omega": omega,
                     "ncycles": ncycles, "T": T})



def h2p_medium(R: float = 2.0, eps: float = 1.472) -> Dict:
    """1-D H2+ model: two soft-core centres at +-R/2 (Sec. Molecular HHG)."""
    return medium({"kind": "const", "m": 1.0}, {"kind": "h2p_softcore", "R": R, "eps": eps})


def hydrogenic_split(l_max: float, r1: float, n_side: int) -> int:
    """Number of linear intervals n_lin (of n_side on one side) for which the hydrogenic grading has
    no jump in spacing: the first exponential interval r_cross (exp(ln(l_max/r_cross)/n_exp) - 1)
    equals r1 (bisection; that interval grows with n_lin)."""
    def first_exp_step(n_lin):
        rc = n_lin * r1
        return rc * math.expm1(math.log(l_max / rc) / (n_side - n_lin))
    lo, hi = 1, n_side - 1
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if mid * r1 < l_max and first_exp_step(mid) < r1:
            lo = mid
        else:
            hi = mid
    return lo


def h2p_1d(nsplines: int = 30007, p: int = 7, l_max: float = 4000.0, r1: float = 0.2,
           e0: Optional[float] = None, omega: float = 0.057, ramp_cycles: float = 1.0, flat_cycles: float = 4.0,
           dt: float = 0.05, nsteps: Optional[int] = None) -> Workload:
    """1-D H2+ (R = 2, eps = 1.472) on [-l_max, l_max] with hydrogenic knots, 6-cycle trapezoidal
    pulse at w0 = 0.057 and 1e14 W/cm^2 (Sec. Molecular HHG). nsplines - p elements, split evenly
    between the two sides; on each side the linear part (step r1) is as long as keeps the spacing
    continuous into the exponential part (hydrogenic_split)."""
    n_side = (nsplines - p) // 2
    if 2 * n_side != nsplines - p:
        raise ValueError("nsplines - p must be even (symmetric grid)")
    n_lin = hydrogenic_split(l_max, r1, n_side)
    knots = hydrogenic_knots(l_max, r1, n_lin, n_side - n_lin, p)
    if e0 is None:
        e0 = e0_from_intensity(1e14)
    T = (2 * ramp_cycles + flat_cycles) * 2 * math.pi / omega
    if nsteps is None:
        nsteps = int(math.ceil(T / dt - 1e-9))
    t = time_grid(dt, nsteps)
    run = Run1D(knots, p, p + 1, h2p_medium(), trapezoid_pulse(t, e0, omega, ramp_cycles, flat_cycles), dt)
    return Workload("h2p_1d", [run], nsteps, dt,
                    {"nsplines": nsplines, "p": p, "l_max": l_max, "r1": r1, "n_lin": n_lin,
                     "n_exp": n_side - n_lin, "E0": e0, "omega": omega, "T": T})

def dqw_knots(med: Dict, nsplines: int, p: int, well_weight: float = 2.0) -> np.ndarray:
    """Piecewise-uniform knots with all interfaces as knots; wells and the central barrier are
    meshed `well_weight` times denser than the outer barriers (knots clustered near interfaces)."""
    bounds = med["mass"]["bounds"]
    n_elem = nsplines - p
    lengths = np.diff(bounds)
    weights = np.array([1.0, well_weight, well_weight, well_weight, 1.0]) * lengths
    raw = weights / weights.sum() * n_elem
    counts = np.maximum(np.floor(raw).astype(int), 2)
    # distribute the remainder to the regions with the largest fractional parts
    rem = n_elem - counts.sum()
    order = np.argsort(-(raw - np.floor(raw)))
    i = 0
    while rem != 0:
        r = order[i % len(order)]
        if rem > 0:
            counts[r] += 1
            rem -= 1
        elif counts[r] > 2:
            counts[r] -= 1
            rem += 1
        i += 1
    return open_piecewise_knots(bounds, counts.tolist(), p)


def dqw_batch(n_geometries: int = 256, fields_per_geometry: int = 4, p: int = 6, nsplines_range=(800, 3000),
              wb_range_nm=(1.0, 6.0), lw_nm: float = 10.0, v0_ev: float = 0.24, lam_nm: float = 10000.0,
              ncycles: float = 4.0, dt: float = 0.5, nsteps: Optional[int] = None,
              gammas: Sequence[float] = (2.3, 1.5, 1.0, 0.5), seed: int = SEED,
              nquad: Optional[int] = None) -> Workload:
    """Batched 1-D PDM double-quantum-well runs: random barrier widths and basis sizes, each geometry
    driven by `fields_per_geometry` mid-IR intensities (Keldysh gamma values)."""
    rng = np.random.default_rng(seed)
    omega = omega_from_nm(lam_nm)
    T = ncycles * 2 * math.pi / omega
    if nsteps is None:
        nsteps = int(math.ceil(T / dt - 1e-9))
    t = time_grid(dt, nsteps)
    runs: List[Run1D] = []
    wbs = rng.uniform(wb_range_nm[0], wb_range_nm[1], size=n_geometries)
    ns = rng.integers(nsplines_range[0], nsplines_range[1] + 1, size=n_geometries)
    for g in range(n_geometries):
        med = dqw_medium(lw_nm, float(wbs[g]), v0_ev)
        kn = dqw_knots(med, int(ns[g]), p)
        for f in range(fields_per_geometry):
            e0 = keldysh_e0(gammas[f % len(gammas)], omega)
            runs.append(Run1D(kn, p, nquad or p + 1, med, sin2_pulse(t, e0, omega, ncycles), dt, geometry=g))
    return Workload("dqw_batch_1d", runs, nsteps, dt,
                    {"n_geometries": n_geometries, "fields_per_geometry": fields_per_geometry, "p": p,
                     "omega": omega, "T": T, "wb_nm": wbs.tolist(), "nsplines": ns.tolist()})


@dataclass
class RunND:
    knots: List[np.ndarray]    # per axis
    degree: int
    nquad: int
    medium: Dict
    field: np.ndarray          # (nsteps+1, dim)
    dt: float


def dot_batch(n_dots: int = 64, p: int = 6, nsplines_range=(256, 768), semi_axes_nm=(5.0, 20.0),
              margin_nm: float = 20.0, lam_nm: float = 10000.0, ncycles: float = 4.0, dt: float = 0.5,
              nsteps: Optional[int] = None, gammas: Optional[Sequence[float]] = None, n_cep: int = 8,
              seed: int = SEED) -> Workload:
    """Batch of 2-D elliptical quantum dots (position-dependent mass 0.067/0.092, 0.24 eV step):
    N/axis ~ U{nsplines_range}, semi-axes ~ U[semi_axes_nm], square domain of half-width
    max(a, b) + margin; run k is driven by intensity k // n_cep (Keldysh gamma, log-spaced 2.3 .. 0.5)
    and carrier-envelope phase 2 pi (k % n_cep) / n_cep, 10 um, sin^2, polarised along x."""
    rng = np.random.default_rng(seed)
    omega = omega_from_nm(lam_nm)
    T = ncycles * 2 * math.pi / omega
    if nsteps is None:
        nsteps = int(math.ceil(T / dt - 1e-9))
    t = time_grid(dt, nsteps)
    n_int = max(1, n_dots // n_cep)
    if gammas is None:
        gammas = np.geomspace(2.3, 0.5, n_int)
    ab = rng.uniform(semi_axes_nm[0], semi_axes_nm[1], size=(n_dots, 2))
    ns = rng.integers(nsplines_range[0], nsplines_range[1] + 1, size=n_dots)
    runs: List[RunND] = []
    for k in range(n_dots):
        a, b = float(ab[k, 0]), float(ab[k, 1])
        half = (max(a, b) + margin_nm) * NM
        kn = knots_for_nsplines(-half, half, int(ns[k]), p)
        e0 = keldysh_e0(float(gammas[(k // n_cep) % len(gammas)]), omega)
        cep = 2 * math.pi * (k % n_cep) / n_cep
        runs.append(RunND([kn, kn], p, p + 1, ellipse_dot_medium(a, b), sin2_pulse(t, e0, omega, ncycles, cep=cep,
                                                                                     dim=2), dt))
    return Workload("dot_batch_2d", runs, nsteps, dt,
                    {"n_dots": n_dots, "p": p, "omega": omega, "T": T, "semi_axes_nm": ab.tolist(),
                     "nsplines": ns.tolist()})


def driven_ho_1d(e0: float = 0.1, dt: float = 0.01, t_end: float = 10.0, L: float = 20.0,
                 nsplines: int = 200, p: int = 5) -> Workload:
    """1-D analogue of Appendix A: HO (omega=1) driven by E0 sin t."""
    nsteps = int(round(t_end / dt))
    t = time_grid(dt, nsteps)
    run = Run1D(knots_for_nsplines(-L, L, nsplines, p), p, p + 1, ho_medium([1.0]), resonant_sine(t, e0), dt)
    return Workload("driven_ho_1d", [run], nsteps, dt, {"E0": e0})


# ---------------------------------------------------------------- initial states (no method arithmetic)
def greville(knots: np.ndarray, p: int) -> np.ndarray:
    """Greville abscissae (knot averages) of the interior B-splines (Dirichlet ends dropped)."""
    n = len(knots) - p - 1
    g = np.array([knots[i + 1:i + p + 1].mean() for i in range(n)])
    return g[1:-1]


def gaussian_coeffs(knots: np.ndarray, p: int, x0: float, sigma: float, k0: float = 0.0) -> np.ndarray:
    """Coefficients sampled from a Gaussian wavepacket at the Greville points (a synthetic state)."""
    g = greville(knots, p)
    return np.exp(-0.5 * ((g - x0) / sigma) ** 2 + 1j * k0 * g)


def random_coeffs(n: int, seed: int = SEED) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)
