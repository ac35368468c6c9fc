"""Writes softcore3d_p6.npz: the oracle's trajectory for the 3-D soft-core parity case at the degree of
the 3-D workload (p = 6), which the oracle's full tensor quadrature takes minutes to assemble.

Calls only oracle/ and the input generators in workloads.py (no library code):
  12 order-6 splines per axis on [-8, 8]^3 (10 coefficients per axis, 1000 in all), V = -1/sqrt(r^2 + 0.5),
  ground state of Eq. gen_ev, then 10 Crank-Nicolson steps (Eq. cn_system) of an elliptically
  polarised (0.3) sin^2 pulse, E0 = 0.1, w = 0.5, one cycle, dt = 0.05, with the per-step observables
  of Sec. "Dipoles".
Run: python tests/golden/make_softcore3d_p6.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as wl  # noqa: E402
from oracle import assemble, eigen, propagate  # noqa: E402

PARAMS = {"nsplines": 12, "p": 6, "L": 8.0, "eps": 0.5, "dt": 0.05, "nsteps": 10, "e0": 0.1, "omega": 0.5,
          "ncycles": 1.0, "ellipticity": 0.3}


def inputs():
    P = PARAMS
    t = wl.knots_for_nsplines(-P["L"], P["L"], P["nsplines"], P["p"])
    field = wl.sin2_pulse(wl.time_grid(P["dt"], P["nsteps"]), P["e0"], P["omega"], P["ncycles"],
                          ellipticity=P["ellipticity"], dim=3)
    return [t, t, t], wl.softcore_medium(P["eps"]), field


def main():
    P = PARAMS
    knots, med, field = inputs()
    m = assemble.assemble_nd(knots, [P["p"]] * 3, [P["p"] + 1] * 3, med)
    e, c0 = eigen.ground_state(m)
    c, obs = propagate.cn_propagate(m, c0, field, P["dt"], P["nsteps"])
    np.savez_compressed(os.path.join(HERE, "softcore3d_p6.npz"), c0=c0, c=c, obs=obs, energy=e,
                        params=np.array([P[k] for k in sorted(P)]), param_names=np.array(sorted(P)))


if __name__ == "__main__":
    main()
