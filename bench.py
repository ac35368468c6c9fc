"""Benchmark: TDSE coefficient-updates/s of the batched Crank-Nicolson propagator on B300.

Workload (N=1): the batched 1-D position-dependent-mass double-quantum-well scan -
256 GaAs/Al0.3Ga0.7As geometries (barrier 1-6 nm, wells 10 nm, 0.24 eV offset,
m* 0.067/0.092, 800-3000 order-6 B-splines with knots on every interface) x 4 mid-IR
intensities (lambda = 10 um, Keldysh gamma 2.3/1.5/1.0/0.5) = 1024 uneven runs in one
persistent launch, dt = 0.5 a.u., mixed precision (FP32 factors + double-float
refinement). A step = one CN step of every run incl. the per-step observables.

Beside the headline line: the paper's 1-D H2+ run (30 007 order-7 splines, hydrogenic knots;
config_h2p_1d) and the 2-D/3-D workloads (config_2d, config_dots_2d, config_3d), each in both
precisions.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--h2p-steps S]
                  [--nd-legs 2d,dots,3d] [--nd-steps S]

Prints one JSON line. With torchrun (N > 1) the batch grows to N x 256 geometries and is split over
the ranks by the longest-processing-time rule on coefficients x steps (weak scaling: each rank holds
about the one-GPU batch; no collective inside the time loop); rank 0 prints the line with the max time
over ranks and gathers every run's status on the host.

The CPU baseline is the oracle on the host cores (one run per spawned process); the same runs, whole
pulse, also check the mixed path's harmonic yields against the oracle's.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

# the CPU-baseline leg times the oracle single-threaded: pin BLAS/OpenMP pools before numpy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

# DRAM bytes (read + write) per coefficient-step of the mixed 1-D kernel, from one ncu capture of the
# current kernel (lane-packed, residual on packed f32x2 pairs, separator chains spread over the warps)
# on the DQW batch: 3.3143 GB read + 0.9234 GB written in the 3-step warm-up launch of 1 873 260
# coefficients; the traffic of a timed launch is this times its coefficient-steps.
NCU_DRAM_BYTES_PER_COEFF_STEP = 754.0
METRIC = "TDSE coefficient-updates/s: batched mixed vs plain FP64 at stated HHG/norm error"
UNIT = "coefficient-updates/s"


def flops_per_dof_step(p: int) -> int:
    """Algorithmic flops of one CN step per coefficient (complex MAC = 8 flops): band LDL^T
    (p(p+1)/2 MACs + p scalings + reciprocal), rhs (2p+1 MACs), forward/back substitution
    (2p MACs + D^-1), and the four quadratic forms S, D, G, K of the observables."""
    factor = 8 * p * (p + 1) // 2 + 6 * p + 10
    rhs = 8 * (2 * p + 1)
    subst = 16 * p + 6
    obs = 3 * (p + 1) + 8 * (p + 1)
    return factor + rhs + subst + obs


def build_batch_inputs(n_geom, fields_per_geom, nsteps, seed=wl.SEED):
    wk = wl.dqw_batch(n_geometries=n_geom, fields_per_geometry=fields_per_geom, nsteps=nsteps, seed=seed)
    return wk


def initial_state(run: wl.Run1D, med) -> np.ndarray:
    """Synthetic initial state: Gaussian wavepacket centred in the left well (Greville samples)."""
    b = med["mass"]["bounds"]
    x0 = 0.5 * (b[1] + b[2])
    sigma = 0.25 * (b[2] - b[1])
    c = wl.gaussian_coeffs(run.knots, run.degree, x0, sigma)
    return c / np.sqrt(np.sum(np.abs(c) ** 2))


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


# ----------------------------------------------------------------------------- CPU baseline (oracle)
def _oracle_worker(job):
    """One run through the CPU oracle, as it stands, in a spawned worker process (one BLAS thread):
    assembly, `warm` untimed and then `steps` timed Crank-Nicolson steps. Returns (job index, final
    state, observables of the timed steps, timed seconds, coefficients)."""
    idx, run, c0, dt, warm, steps = job
    from oracle import assemble, propagate
    m = assemble.assemble_1d(run.knots, run.degree, run.nquad, run.medium)
    c = np.asarray(c0, dtype=np.complex128)
    if warm:
        c, _ = propagate.cn_propagate(m, c, run.field, dt, warm)
    t0 = time.perf_counter()
    c, obs = propagate.cn_propagate(m, c, run.field, dt, steps, step0=warm)
    return idx, c, obs, time.perf_counter() - t0, len(c)


def oracle_pool_leg(runs, c0s, dt, warm, steps):
    """The CPU oracle on the host cores: one independent run per spawned process, all concurrently.
    Throughput = coefficient-steps of all runs / the longest run's timed seconds. Returns (value,
    details, per-run results in input order)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    jobs = [(i, runs[i], c0s[i], dt, warm, steps) for i in range(len(runs))]
    t0 = time.perf_counter()
    with ctx.Pool(len(jobs)) as pool:
        out = sorted(pool.map(_oracle_worker, jobs, chunksize=1), key=lambda x: x[0])
    wall = time.perf_counter() - t0
    secs = [o[3] for o in out]
    dof = [o[4] for o in out]
    longest = max(secs)
    single = sum(d * steps / t for d, t in zip(dof, secs)) / len(out)
    return sum(dof) * steps / longest, {"seconds": longest, "wall_s": wall, "dof": sum(dof), "single_core": single}, out


def cpu_workers(args) -> int:
    return max(1, min(os.cpu_count() or 1, args.cpu_workers))


def reference_arm(args):
    """--impl reference: the CPU oracle (the stated reference for this build) on the host cores, one
    run of the batch per process, W warm-up and K timed steps each."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    nw = cpu_workers(args)
    wk = build_batch_inputs(args.n_geom, 4, args.warmup + args.steps + 1)
    runs = wk.runs[:nw]
    c0s = [initial_state(r, r.medium) for r in runs]
    value, det, _ = oracle_pool_leg(runs, c0s, wk.dt, args.warmup, args.steps)
    sample = (f"first {nw} runs of the batch ({det['dof']} coefficients), one per process, concurrently; "
              f"{args.warmup} warm-up + {args.steps} timed steps each")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * det["seconds"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "dqw_batch_1d", "runs": len(wk.runs), "sample_runs": nw, "degree": 6},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nw, "nproc": os.cpu_count(), "kind": "oracle",
                             "sample": sample, "single_core": {"value": det["single_core"], "unit": UNIT}},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_leg(tdz, args):
    """CPU baseline and the accuracy of the mixed path on whole pulses. The first `cpu_workers` runs of
    the batch (their whole 4-cycle pulse) go through the oracle, one run per host core, and through the
    GPU mixed path; compared are the final states (rel-L2), the dipoles, the norm drift and every
    odd-harmonic yield up to the run's cutoff I_p + 3.17 U_p (length form w^4 |d~|^2, Sec. "Dipoles";
    I_p = barrier top minus the ground level, U_p with the well mass)."""
    from oracle import assemble, eigen, hhg
    nw = cpu_workers(args)
    wk = build_batch_inputs(args.n_geom, 4, None)
    runs = wk.runs[:nw]
    c0s = [initial_state(r, r.medium) for r in runs]
    value, det, out = oracle_pool_leg(runs, c0s, wk.dt, 0, wk.nsteps)
    geoms = sorted({r.geometry for r in runs})
    ops, ip = [], {}
    for g in geoms:
        r = next(x for x in runs if x.geometry == g)
        ops.append(tdz.assemble_1d(r.knots, r.degree, r.medium, r.nquad))
        m = assemble.assemble_1d(r.knots, r.degree, r.nquad, r.medium)
        ip[g] = max(r.medium["potential"]["V"]) - eigen.ground_state(m, sigma=-1e-3, dense_max=0)[0]
    b = tdz.Batch(ops, [geoms.index(r.geometry) for r in runs], tdz.MIXED)
    for i, c in enumerate(c0s):
        b.set_state(i, c)
    b.propagate(np.ascontiguousarray(np.stack([r.field for r in runs])), wk.dt, 0, wk.nsteps)
    w0 = wk.notes["omega"]
    rel = dmax = herr = drift = 0.0
    nharm = 0
    for i, r in enumerate(runs):
        _, c_o, obs_o, _, _ = out[i]
        og, st = b.observe(i)
        if st != 0:
            raise RuntimeError(f"GPU run {i} status {st}")
        rel = max(rel, float(np.linalg.norm(b.get_state(i) - c_o) / np.linalg.norm(c_o)))
        dmax = max(dmax, float(np.max(np.abs(og[:, 2] - obs_o[:, 2])) / max(1e-30, np.max(np.abs(obs_o[:, 2])))))
        drift = max(drift, float(np.max(np.abs(og[:, 4] - og[0, 4]))))
        qcut = max(3, int(math.floor(hhg.cutoff_harmonic(ip[r.geometry], float(np.max(np.abs(r.field))), w0,
                                                          m_eff=0.067))))
        om, So = hhg.spectrum(obs_o[:, 2], wk.dt, length_form=True)
        _, Sg = hhg.spectrum(og[:, 2], wk.dt, length_form=True)
        _, Yo = hhg.harmonic_yields(om, So, w0, qcut)
        _, Yg = hhg.harmonic_yields(om, Sg, w0, qcut)
        herr = max(herr, float(np.max(np.abs(Yg / Yo - 1))))
        nharm += len(Yo)
    del b
    cpu = {"value": value, "unit": UNIT, "cores": nw, "nproc": os.cpu_count(), "kind": "oracle",
           "sample": (f"first {nw} runs of the batch, whole 4-cycle pulse ({wk.nsteps} steps, {det['dof']} "
                      f"coefficients), one run per process, concurrently; value = coefficient-steps / the "
                      f"longest run's {det['seconds']:.1f} s"),
           "single_core": {"value": det["single_core"], "unit": UNIT, "cores": 1,
                           "sample": "mean over the same runs of each run's own throughput"}}
    acc = {"runs": nw, "steps": wk.nsteps, "max_rel_l2": rel, "max_dipole_rel_err": dmax, "max_norm_drift": drift,
           "max_hhg_yield_rel_err": herr, "harmonics_compared": nharm,
           "hhg": "odd q up to I_p + 3.17 U_p per run, w^4 |d~|^2 with a Kaiser (beta 8) window"}
    return cpu, acc


def _nd_time(tdz, name, ops, run_ops, c0s, fields, dt, nsteps, extra, fp64_steps=None):
    """Time `nsteps` steps of a 2-D/3-D batch in mixed precision and `fp64_steps` (default: the same) in
    binary64, each after one warm-up step; the rel-L2 comparison of the two is taken after the binary64
    window (the mixed run is repeated to that length first when the windows differ)."""
    import torch
    fp64_steps = nsteps if fp64_steps is None else fp64_steps
    res = {"workload": name, "runs": len(run_ops), "coefficients": int(sum(ops[g].n for g in run_ops)),
           "steps": {"mixed": nsteps, "fp64": fp64_steps}}
    res.update(extra)
    dim = fields.shape[2]
    states = {}
    for label, prec in (("mixed", tdz.MIXED), ("fp64", tdz.FP64)):
        k = nsteps if label == "mixed" else fp64_steps
        t0 = time.perf_counter()
        b = tdz.Batch(ops, run_ops, prec)
        t_create = time.perf_counter() - t0
        for i, c in enumerate(c0s):
            b.set_state(i, c)
        b.propagate(np.ascontiguousarray(fields[:, :2]), dt, 0, 1)   # warm-up step
        for i, c in enumerate(c0s):
            b.set_state(i, c)
        _, solves0 = b.refine_stats()
        it0 = b.krylov_stats()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.propagate(np.ascontiguousarray(fields[:, :k + 1]), dt, 0, k)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
        drift, st_bad = 0.0, 0
        for i in range(len(run_ops)):
            o, st = b.observe(i)
            drift = max(drift, float(np.max(np.abs(o[:, -1] - o[0, -1]))))
            st_bad += int(st != 0)
        _, solves = b.refine_stats()
        nsteps_runs = k * len(run_ops)
        res[label] = {"value": res["coefficients"] / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                      "runs_not_ok": st_bad, "norm_drift": drift,
                      "krylov_iterations_per_run_step": (b.krylov_stats() - it0) / nsteps_runs,
                      "solves_per_run_step": (solves - solves0) / nsteps_runs, "device_gb": b.device_bytes / 1e9,
                      "create_s": t_create}
        if label == "mixed" and k != fp64_steps:  # the state after the binary64 window, for the comparison
            for i, c in enumerate(c0s):
                b.set_state(i, c)
            b.propagate(np.ascontiguousarray(fields[:, :fp64_steps + 1]), dt, 0, fp64_steps)
        states[label] = [b.get_state(i) for i in range(len(run_ops))]
        if label == "mixed" and dim == 2:
            res["fused_apply"] = _apply_roofline(tdz, b, ops, run_ops)
            res["operator_choice"] = _operator_choice(tdz, b, ops, run_ops)
        if label == "mixed":
            res["preconditioner_apply"] = _precond_roofline(tdz, b, ops, run_ops)
            if dim == 3:
                res["operator_apply"] = _quad_roofline(tdz, b, ops, run_ops)
        del b
    num = sum(np.linalg.norm(x - y) ** 2 for x, y in zip(states["mixed"], states["fp64"]))
    den = sum(np.linalg.norm(y) ** 2 for y in states["fp64"])
    res["mixed_vs_fp64_rel_l2"] = float(np.sqrt(num / den))
    res["speedup_mixed"] = res["fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"]
    return res


def _apply_roofline(tdz, b, ops, run_ops):
    """HBM roofline of the fused FP32 2-D apply for the largest geometry of the batch, from the
    autotuner's CUDA-event timing (best of three, batch creation). Algorithmic bytes per apply: the
    (2p+1)^2-point FP32 stencil (4 B per entry) plus x read and y written (8 B each per coefficient)."""
    peaks = _measured_peaks()
    g = max(set(run_ops), key=lambda k: ops[k].n)
    groups, ms = b.tuning(g)
    if not groups:
        return None
    p = ops[g].degree[0]
    n = ops[g].n
    nbytes = n * ((2 * p + 1) ** 2 * 4 + 16)
    t = ms[groups] * 1e-3
    ach = nbytes / t / 1e9
    fpd = quad_flops_per_dof(ops[g].shape, p, p + 1)
    alu = fpd * n / t / 1e12
    return {"kernel": f"k_apply2d_tma<{p},{groups}>", "coefficients": n, "bound": "hbm",
            "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
            "peak_source": peaks["source"], "algorithmic_bytes": nbytes, "ms_per_apply": ms[groups],
            "variants_ms": {str(k): v for k, v in ms.items()},
            "state_only_bytes": n * 16, "state_only_frac": n * 16 / t / 1e9 / peaks["hbm_gbs"],
            "quadrature_view": {"flops_per_coefficient": fpd, "achieved_tflops": alu, "peak_tflops": PEAK_FP32_TFLOPS,
                                "frac": alu / PEAK_FP32_TFLOPS,
                                "note": "the same operator's on-the-fly Gauss-point flops over this kernel's time"}}


def quad_flops_per_dof(shape, p, nq):
    """Algorithmic FP32 flops of one Gauss-point sum-factorised apply of the non-separable term, per
    coefficient: interpolation passes over the first dim-1 axes (4(p+1) flops per output: a real basis
    value times a complex coefficient, fused multiply-add on both parts), the fused last-axis pass
    (interpolate, scale by the complex point factor, project back: 8(p+1) + 6 per Gauss point) and the
    projection passes (the same count as the interpolations)."""
    E = [n - p for n in shape]
    Q = [nq * e for e in E]
    total = 0.0
    for a in range(len(shape) - 1):
        pts = float(np.prod(Q[:a + 1])) * float(np.prod(shape[a + 1:]))
        total += 2 * 4 * (p + 1) * pts
    total += float(np.prod(Q)) * (8 * (p + 1) + 6)
    return total / float(np.prod(shape))


def _quad_roofline(tdz, b, ops, run_ops):
    """FP32-ALU roofline of the 3-D inner-solve operator apply (Kronecker passes plus the Gauss-point sum
    factorisation of the soft-core V) for the largest geometry: one apply timed by the library with CUDA
    events (tdz_batch_time_operator, best of 3); algorithmic flops: quad_flops_per_dof (the Kronecker
    passes, about 60 flops per coefficient each, are left out)."""
    g = max(set(run_ops), key=lambda k: ops[k].n)
    ms = b.time_operator(g, 3)
    p = ops[g].degree[0]
    fpd = quad_flops_per_dof(ops[g].shape, p, p + 1)
    ach = fpd * ops[g].n / (ms * 1e-3) / 1e12
    return {"kernels": "k_interp, k_fused_last, k_project (FP32) + Kronecker axis passes", "coefficients": ops[g].n,
            "bound": "alu", "flops_per_coefficient": fpd, "ms_per_apply": ms, "achieved": ach, "peak": PEAK_FP32_TFLOPS,
            "unit": "TFLOP/s", "frac": ach / PEAK_FP32_TFLOPS,
            "peak_source": "148 SM x 128 FP32 lanes x 2 flop x 2.032 GHz (unit counts and max clock)"}


def _operator_choice(tdz, b, ops, run_ops):
    """The two ways the library applies the 2-D operator in the FP32 inner solve, timed on the same
    batch (tdz_batch_time_operator, best of 3): the fused kernel over the assembled (2p+1)^2 stencil
    (HBM-bound), and the Gauss-point sum factorisation with V evaluated at the points (FP32-ALU-bound).
    The library's default is the stencil where it is assembled."""
    g = max(set(run_ops), key=lambda k: ops[k].n)
    p = ops[g].degree[0]
    n = ops[g].n
    ms_stencil = b.time_operator(g, 3)
    b.set_option(tdz.OPT_OPERATOR, tdz.OPERATOR_QUADRATURE)
    ms_quad = b.time_operator(g, 3)
    b.set_option(tdz.OPT_OPERATOR, tdz.OPERATOR_AUTO)
    fpd = quad_flops_per_dof(ops[g].shape, p, p + 1)
    return {"stencil_ms": ms_stencil, "quadrature_ms": ms_quad,
            "quadrature_tflops": fpd * n / (ms_quad * 1e-3) / 1e12,
            "quadrature_frac_fp32_peak": fpd * n / (ms_quad * 1e-3) / 1e12 / PEAK_FP32_TFLOPS,
            "faster": "stencil" if ms_stencil <= ms_quad else "quadrature"}


def _measured_peaks():
    """HBM copy bandwidth and dense BF16 tensor rate (burst) measured on this machine, else the fallback figures."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "source": "fallback"}


# FP32 ALU peak: 148 SM x 128 FP32 lanes x 2 flop x 2.032 GHz (unit counts and max clock), TFLOP/s
PEAK_FP32_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12

# dense TF32 : BF16 tensor rate of B300 (nominal 1.1 : 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25


def _precond_roofline(tdz, b, ops, run_ops):
    """Tensor roofline of the mixed fast-diagonalisation preconditioner for the largest geometry, from the
    autotuner's CUDA-event timing of one whole apply (split, 2 dim tcgen05 axis transforms, scaling, merge;
    batch creation, best of three, six variants). Tensor work per apply: for each axis a and each of the
    two passes, 2 TF32 products x 2 flops x (2 Np / np_a rows) x np_a columns x np_a (k) = 8 Np np_a, i.e.
    16 Np sum_a np_a; the algorithmic (one FP32 product) flops are half of that. Peak: the measured BF16
    rate x the nominal TF32/BF16 ratio."""
    peaks = _measured_peaks()
    g = max(set(run_ops), key=lambda k: ops[k].n)
    v, ms = b.precond_tuning(g)
    if v < 0:
        return None
    npad = [(n + 7) // 8 * 8 for n in ops[g].shape]
    Np = int(np.prod(npad))
    tflop = 16.0 * Np * sum(npad) / 1e12
    t = ms[v] * 1e-3
    peak = peaks["bf16_tflops"] * TF32_PER_BF16
    names = [f"{128 << (c & 1)}-column tiles, " + ("split in shared memory" if c & 2 else "TF32 pairs in memory")
             for c in range(4)] + ["64-column tiles, TF32 pairs in memory", "64-column tiles, split in shared memory"]
    return {"kernel": f"k_tc_axis<{128 << (v & 1)}, false, {'true' if v & 2 else 'false'}> x {2 * len(npad)}"
                      " + split/scale/merge", "padded_shape": npad, "variant": names[v],
            "bound": "tensor", "achieved": tflop / t, "peak": peak, "unit": "TFLOP/s", "frac": tflop / t / peak,
            "peak_source": peaks["source"] + " bf16 x nominal tf32/bf16", "tensor_tflop_per_apply": tflop,
            "algorithmic_fp32_tflop_per_apply": tflop / 2, "ms_per_apply": ms[v],
            "variants_ms": {names[c]: ms[c] for c in range(len(ms))}}


def _gauss_state(knots, p, dim):
    g = wl.greville(knots, p)
    psi = np.exp(-0.5 * (g / (0.05 * (g[-1] - g[0]))) ** 2)
    c = psi
    for _ in range(dim - 1):
        c = np.kron(psi, c)
    return (c / np.linalg.norm(c)).astype(complex)


def _nd_ground_state(tdz, ops, c_starts, v_mins, prec, tol):
    """The library's own ground states of 2-D/3-D geometries (tdz_batch_ground_state; one batch of all
    `ops`, run i from c_starts[i]): a coarse pass with the shift just below the potential's minimum v_min
    (residual 1e-3), then the shift min(0.05, a tenth of the coarse level's height above that shift) below
    the coarse level, to the eigen-residual `tol`. Returns the states and a summary."""
    t0 = time.perf_counter()
    b = tdz.Batch(ops, list(range(len(ops))), prec)
    energies, outer, res = [], 0, 0.0
    for i, (c, vm) in enumerate(zip(c_starts, v_mins)):
        b.set_state(i, c)
        s1 = vm - 0.01 * max(1e-3, abs(vm))
        e1, o1, _ = b.ground_state(i, s1, tol=1e-3, max_outer=200)
        e, o2, r = b.ground_state(i, e1 - min(0.05, 0.1 * (e1 - s1)), tol=tol, max_outer=200)
        energies.append(e)
        outer += o1 + o2
        res = max(res, r)
    c0s = [b.get_state(i) for i in range(len(ops))]
    info = {"precision": "binary64" if prec == tdz.FP64 else "mixed (FP32 solves)", "eigen_residual_max": res,
            "energy_min": min(energies), "energy_max": max(energies), "outer_iterations": outer,
            "krylov_iterations": b.krylov_stats(), "seconds": time.perf_counter() - t0}
    del b
    return c0s, info


def _v_min(medium):
    """The potential's minimum (a lower bound of every level)."""
    v = medium["potential"]
    if v["kind"] == "softcore":
        return -v["z"] / np.sqrt(v["eps"])
    if v["kind"] == "ellipse":
        return min(v["v_in"], v["v_out"])
    raise KeyError(v["kind"])


# timed steps (mixed, binary64) of the 2-D/3-D legs by default
ND_WINDOWS = {"2d": (200, 20), "dots": (20, 4), "3d": (20, 3)}


def nd_legs(tdz, nsteps, which, n2d=1024, n3d=256):
    """2-D/3-D workloads beside the 1-D batch, timed over ND_WINDOWS (mixed, binary64) steps unless
    `nsteps` (> 0) sets both windows:
    softcore_atom_2d: V = -1/sqrt(r^2+0.5) on [-150,150]^2, 1024 order-7 splines per axis (1.04 M
      coefficients), 800 nm 1e14 W/cm^2 sin^2 pulse, dt = 0.05, from the library's ground state (binary64,
      eigen-residual 1e-10; the dots and the 3-D atom from ground states of the mixed batches' FP32 solves,
      eigen-residual 1e-5: a binary64 solve of 64 dots or of the 3-D grid takes minutes);
    dot_batch_2d: 64 elliptical GaAs dots (16 M coefficients), 10 um, 8 intensities x 8 CEPs, dt = 0.5;
    softcore_atom_3d: [-100,100]^3, 256 order-6 splines per axis (16.4 M coefficients), elliptical
      (0.3) 800 nm pulse, dt = 0.05."""
    def win(leg):
        return (nsteps, nsteps) if nsteps else ND_WINDOWS[leg]

    out = {}
    if "2d" in which:
        km, kd = win("2d")
        p, t = 7, wl.knots_for_nsplines(-150.0, 150.0, n2d, 7)
        ops = tdz.Ops([tdz.Basis(t, p, p + 1) for _ in range(2)], wl.softcore_medium(0.5))
        dt = 0.05
        f = wl.sin2_pulse(wl.time_grid(dt, max(km, kd) + 1), wl.e0_from_intensity(1e14), wl.omega_from_nm(800.0), 4.0,
                          dim=2)
        med = wl.softcore_medium(0.5)
        c0s, gs = _nd_ground_state(tdz, [ops], [_gauss_state(t, p, 2)], [_v_min(med)], tdz.FP64, 1e-10)
        out["config_2d"] = _nd_time(tdz, "softcore_atom_2d", [ops], [0], c0s, f[None], dt, km,
                                    {"operator": "assembled (2p+1)^2 stencil",
                                     "preconditioner": "fast diagonalisation (tcgen05 TF32 axis transforms)",
                                     "initial_state": "ground state (tdz_batch_ground_state)", "ground_state": gs}, kd)
    if "dots" in which:
        km, kd = win("dots")
        wk = wl.dot_batch(nsteps=max(km, kd) + 1)
        ops = [tdz.Ops([tdz.Basis(k, r.degree, r.nquad) for k in r.knots], r.medium) for r in wk.runs]
        c0s, gs = _nd_ground_state(tdz, ops, [_gauss_state(r.knots[0], r.degree, 2) for r in wk.runs],
                                   [_v_min(r.medium) for r in wk.runs], tdz.MIXED, 1e-5)
        fields = np.stack([r.field for r in wk.runs])
        out["config_dots_2d"] = _nd_time(tdz, "dot_batch_2d", ops, list(range(len(ops))), c0s, fields, wk.dt, km,
                                         {"operator": "assembled stencil (variable mass + step potential)",
                                          "preconditioner": "fast diagonalisation, mean 1/m",
                                          "initial_state": "ground states (tdz_batch_ground_state)",
                                          "ground_state": gs}, kd)
    if "3d" in which:
        km, kd = win("3d")
        p, t = 6, wl.knots_for_nsplines(-100.0, 100.0, n3d, 6)
        ops = tdz.Ops([tdz.Basis(t, p, p + 1) for _ in range(3)], wl.softcore_medium(0.5))
        dt = 0.05
        f = wl.sin2_pulse(wl.time_grid(dt, max(km, kd) + 1), 0.05, wl.omega_from_nm(800.0), 4.0, ellipticity=0.3,
                          dim=3)
        med = wl.softcore_medium(0.5)
        c0s, gs = _nd_ground_state(tdz, [ops], [_gauss_state(t, p, 3)], [_v_min(med)], tdz.MIXED, 1e-5)
        out["config_3d"] = _nd_time(tdz, "softcore_atom_3d", [ops], [0], c0s, f[None], dt, km,
                                    {"operator": "Gauss-point sum factorisation",
                                     "preconditioner": "fast diagonalisation (tcgen05 TF32 axis transforms)",
                                     "initial_state": "ground state (tdz_batch_ground_state)", "ground_state": gs},
                                    kd)
    return out


def h2p_leg(tdz, nsteps):
    """The paper's 1-D H2+ run (Sec. Molecular HHG): one run of 30 007 order-7 splines on [-4000, 4000]
    with hydrogenic knots, 6-cycle trapezoidal pulse (w0 = 0.057, 1e14 W/cm^2), dt = 0.05, from the
    library's own ground state; `nsteps` timed steps of the ramp in each precision (CUDA events)."""
    import torch
    wk = wl.h2p_1d(nsteps=nsteps + 2)
    r = wk.runs[0]
    ops = tdz.assemble_1d(r.knots, r.degree, r.medium, r.nquad)
    e_ground, c0 = ops.ground_state()
    field = np.ascontiguousarray(r.field.reshape(1, -1, 1))
    res = {"workload": "h2p_1d", "runs": 1, "coefficients": ops.n, "degree": r.degree, "dt": wk.dt, "steps": nsteps,
           "ground_energy": e_ground, "grid": {k: wk.notes[k] for k in ("l_max", "r1", "n_lin", "n_exp")}}
    states = {}
    for label, prec in (("mixed", tdz.MIXED), ("fp64", tdz.FP64)):
        b = tdz.Batch([ops], [0], prec)
        b.set_state(0, c0)
        b.propagate(np.ascontiguousarray(field[:, :3]), wk.dt, 0, 2)  # warm-up
        b.set_state(0, c0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.propagate(np.ascontiguousarray(field[:, :nsteps + 1]), wk.dt, 0, nsteps)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / nsteps
        o, st = b.observe(0)
        res[label] = {"value": ops.n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "status": st,
                      "norm_drift": float(np.max(np.abs(o[:, 4] - 1.0)))}
        states[label] = b.get_state(0)
        del b
    res["mixed_vs_fp64_rel_l2"] = float(np.linalg.norm(states["mixed"] - states["fp64"]) /
                                        np.linalg.norm(states["fp64"]))
    res["speedup_mixed"] = res["fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"]
    # the same grid as a scan: 148 independent runs (one per SM) of 37 intensities (0.5-2.0e14 W/cm^2,
    # log-spaced) x 4 carrier-envelope phases, sharing one geometry, in one persistent launch
    nscan, nsteps_scan = 148, max(10, nsteps // 4)
    t = wl.time_grid(wk.dt, nsteps_scan + 2)
    fields = []
    for k in range(nscan):
        e0 = wl.e0_from_intensity(1e14 * 10 ** (math.log10(0.5) + (math.log10(2.0) - math.log10(0.5)) * (k // 4) / 36))
        cep = 0.5 * math.pi * (k % 4)
        Tc = 2 * math.pi / 0.057
        env = np.clip(np.minimum(t / Tc, (6 * Tc - t) / Tc), 0.0, 1.0)
        fields.append(e0 * env * np.sin(0.057 * t + cep))
    fields = np.ascontiguousarray(np.stack(fields)[:, :, None])
    scan = {"runs": nscan, "coefficients": nscan * ops.n, "steps": nsteps_scan,
            "scan": "37 intensities 0.5-2e14 W/cm^2 (log) x 4 CEPs, trapezoidal 1+4+1 cycles"}
    for label, prec in (("mixed", tdz.MIXED), ("fp64", tdz.FP64)):
        b = tdz.Batch([ops], [0] * nscan, prec)
        c_all = np.concatenate([c0] * nscan)
        b.set_states(c_all)
        b.propagate(np.ascontiguousarray(fields[:, :3]), wk.dt, 0, 2)  # warm-up
        b.set_states(c_all)
        torch.cuda.synchronize()
        e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0_.record()
        b.propagate(np.ascontiguousarray(fields[:, :nsteps_scan + 1]), wk.dt, 0, nsteps_scan)
        e1_.record()
        torch.cuda.synchronize()
        ms = e0_.elapsed_time(e1_) / nsteps_scan
        obs, sts = b.observe_all()
        scan[label] = {"value": nscan * ops.n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                       "runs_not_ok": int(sum(int(x) != 0 for x in sts)),
                       "norm_drift": float(np.max(np.abs(obs[:, :, 4] - 1.0)))}
        del b
    scan["speedup_mixed"] = scan["fp64"]["ms_per_step"] / scan["mixed"]["ms_per_step"]
    res["scan"] = scan
    return res


# ----------------------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-geom", type=int, default=256)
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--cpu-workers", type=int, default=16, help="oracle processes (one run each), <= nproc")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--nd-steps", type=int, default=0,
                    help="timed steps of each 2-D/3-D leg in both precisions (0: the per-leg windows ND_WINDOWS)")
    ap.add_argument("--nd-legs", default="2d,dots,3d", help="comma list of 2d, dots, 3d (empty: none)")
    ap.add_argument("--nd-2d-splines", type=int, default=1024, help="splines per axis of the 2-D atom")
    ap.add_argument("--nd-3d-splines", type=int, default=256, help="splines per axis of the 3-D atom")
    ap.add_argument("--h2p-steps", type=int, default=200, help="timed steps of the 1-D H2+ run (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2608_18472_b300 as tdz

    nsteps_total = args.warmup + args.steps
    # one global batch of world x n_geom geometries x 4 intensities (seeded), split over the ranks by the
    # longest-processing-time rule on coefficients x steps: every rank propagates only its own runs, about
    # the work of the one-GPU batch (weak scaling), with no collective inside the time loop
    from paper_2608_18472_b300 import shard
    wk = build_batch_inputs(args.n_geom * world, 4, max(nsteps_total, args.fp64_steps) + 1)
    run_dof = [len(r.knots) - r.degree - 3 for r in wk.runs]
    dof_all = sum(run_dof)
    mine = shard.lpt_partition([d * nsteps_total for d in run_dof], world)[rank]
    runs = [wk.runs[i] for i in mine]
    geoms = {}
    for r in runs:
        if r.geometry not in geoms:
            geoms[r.geometry] = tdz.assemble_1d(r.knots, r.degree, r.medium, r.nquad)
    gids = sorted(geoms)
    ops = [geoms[g] for g in gids]
    run_ops = [gids.index(r.geometry) for r in runs]
    c0 = [initial_state(r, r.medium) for r in runs]
    p = runs[0].degree
    field_all = np.ascontiguousarray(np.stack([r.field for r in runs]))  # [runs, steps+1, 1]
    nruns = len(runs)
    dof = sum(ops[g].n for g in run_ops)
    assert dof == sum(run_dof[i] for i in mine)
    stream = torch.cuda.current_stream()

    def make_batch(prec):
        b = tdz.Batch(ops, run_ops, prec, stream=stream.cuda_stream)
        for i in range(nruns):
            b.set_state(i, c0[i])
        return b

    def dev_field(k0, k):
        return torch.from_numpy(np.ascontiguousarray(field_all[:, k0:k0 + k + 1, :])).cuda()

    # ---------------- mixed (headline): warm-up then K timed steps, inputs resident on device
    bm = make_batch(tdz.MIXED)
    fw, ft = dev_field(0, args.warmup), dev_field(args.warmup, args.steps)
    bm.propagate(fw, wk.dt, 0, args.warmup)
    norm0 = np.array([bm.observe(i)[0][-1, 4] for i in range(nruns)])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        bm.propagate(ft, wk.dt, args.warmup, args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    local = {}
    for i in range(nruns):
        o, st = bm.observe(i)
        local[mine[i]] = (int(st), float(np.max(np.abs(o[:, 4] - norm0[i]) / norm0[i])))
    max_rel, nsolve = bm.refine_stats()
    solves_per_step = nsolve / (nruns * (args.warmup + args.steps))
    summary = shard.gather_runs(local, len(wk.runs))       # host-side gather of every run's status and drift
    if dist:
        t = torch.tensor([max_rel, solves_per_step], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        max_rel, solves_per_step = float(t[0]), float(t[1])
    statuses = [x[0] for x in summary] if summary else []
    drift = max(x[1] for x in summary) if summary else 0.0

    # ---------------- plain FP64 on the same batch (comparison leg)
    bf = make_batch(tdz.FP64)
    ff = dev_field(0, args.fp64_steps)
    bf.propagate(dev_field(0, 2), wk.dt, 0, 2)  # warm-up
    for i in range(nruns):
        bf.set_state(i, c0[i])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bf.propagate(ff, wk.dt, 0, args.fp64_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    del bf

    # ---------------- end to end through the public API with host buffers: upload every run's state,
    # propagate with the field in pinned host memory, read every run's observables
    pinned_field = torch.from_numpy(np.ascontiguousarray(field_all[:, args.warmup:args.warmup + args.steps + 1, :])).pin_memory()
    c_all = np.concatenate(c0)
    pinned_state = torch.from_numpy(np.ascontiguousarray(np.stack([c_all.real, c_all.imag], axis=1).reshape(-1))).pin_memory()
    obs_host = torch.empty((nruns, args.steps, 5), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bm.set_states(pinned_state)
    bm.propagate(pinned_field, wk.dt, args.warmup, args.steps)
    bm.observe_all(out=obs_host)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = (pinned_field.numel() * 8 + pinned_state.numel() * 8) / args.steps
    d2h = obs_host.numel() * 8 / args.steps

    value = dof_all * args.steps / (ms * 1e-3)
    value64 = dof * args.fp64_steps / (ms64 * 1e-3)
    flops = flops_per_dof_step(p) * dof * args.steps
    peak_fp32 = PEAK_FP32_TFLOPS
    achieved = flops / (ms * 1e-3) / 1e12

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+ff", "data": "synthetic",
            "config": {"workload": "dqw_batch_1d", "runs": len(wk.runs), "geometries": args.n_geom * world,
                       "coefficients": dof_all, "runs_per_gpu": nruns, "coefficients_per_gpu": dof,
                       "degree": p, "dt": wk.dt, "precision": "mixed", "l2": "working set > L2 (126 MB): no flush",
                       "parallelism": f"dp{world}: LPT shards of one batch" if world > 1 else "dp1"},
            "gpu_launches": 1,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                         "frac": achieved / peak_fp32,
                         "traffic": (NCU_DRAM_BYTES_PER_COEFF_STEP * dof * args.steps
                                     if NCU_DRAM_BYTES_PER_COEFF_STEP else None),
                         "note": ("achieved: algorithmic flops per coefficient-step x coefficient-steps of the timed "
                                  "launch / its event time; peak: 148 SM x 128 FP32 lanes x 2 flop x 2.032 GHz (unit "
                                  "counts and max clock); traffic: DRAM bytes of the timed launch (ncu bytes per "
                                  "coefficient-step x coefficient-steps)")},
            "plain_fp64": {"value": value64, "unit": UNIT, "ms_per_step": ms64 / args.fp64_steps, "steps": args.fp64_steps,
                           "speedup_mixed": dof * args.steps / (ms * 1e-3) / value64},
            "accuracy": {"norm_drift_max": drift, "refine_max_rel_residual": max_rel,
                         "solves_per_step": solves_per_step, "runs_not_ok": int(sum(s != 0 for s in statuses))},
            "e2e": {"value": dof_all * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "clocks": clk.summary()}
    r32, r64 = tdz.device_rates()
    line["device_rates"] = {"fp32_fma_tflops": r32 / 1e12, "fp64_fma_tflops": r64 / 1e12, "ratio": r32 / r64,
                            "how": "tdz_device_rates: 8 independent FMA chains per thread, 8 x 256 threads per SM"}
    # ---------------- 2-D leg: the soft-core atom of the 2-D configuration (1024 x 1024 order-7 splines),
    # a few steps in both precisions (Kronecker + Gauss-point operator, preconditioned COCG)
    if rank == 0 and args.h2p_steps > 0:
        line["config_h2p_1d"] = h2p_leg(tdz, args.h2p_steps)
    if rank == 0 and args.nd_steps >= 0 and args.nd_legs:
        line.update(nd_legs(tdz, args.nd_steps, args.nd_legs.split(","), args.nd_2d_splines, args.nd_3d_splines))
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"], line["accuracy"]["sample_vs_oracle"] = cpu_leg(tdz, args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
