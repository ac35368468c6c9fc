"""Sharding of one batch of uneven runs over two ranks (gloo on CPU, world size 2): LPT partition on
coefficients x steps, each rank propagating only its shard, and the host-side gather of observables
and final states on rank 0, which must equal a single-process run of the whole batch exactly.

The propagation inside the ranks is the CPU oracle (this machine has no GPU); what is under test is
the product's host logic in paper_2608_18472_b300/shard.py, which bench.py uses between GPU ranks.
"""
import os
import pickle
import socket

import numpy as np
import pytest

import workloads as wl

SHARD_PATH = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2608_18472_b300",
                          "shard.py")


def _shard_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("tdz_shard", SHARD_PATH)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _batch():
    """Five uneven double-quantum-well runs (two geometries, different fields), short window."""
    wk = wl.dqw_batch(n_geometries=3, fields_per_geometry=2, nsplines_range=(120, 400), nsteps=25, seed=17)
    return wk, wk.runs[:5]


def _propagate(runs, dt, nsteps, ids):
    from oracle import assemble, propagate
    out = {}
    for i in ids:
        r = runs[i]
        m = assemble.assemble_1d(r.knots, r.degree, r.nquad, r.medium)
        c0 = wl.gaussian_coeffs(r.knots, r.degree, 0.0, 50.0)
        c, obs = propagate.cn_propagate(m, c0, r.field, dt, nsteps)
        out[i] = (c, obs)
    return out


def _rank_main(rank, world, port, path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shard = _shard_module()
        wk, runs = _batch()
        costs = [(len(r.knots) - r.degree - 3) * wk.nsteps for r in runs]
        mine = shard.lpt_partition(costs, world)[rank]
        local = _propagate(runs, wk.dt, wk.nsteps, mine)
        merged = shard.gather_runs(local, len(runs), dst=0)
        if rank == 0:
            with open(path, "wb") as f:
                pickle.dump({"merged": merged, "shards": shard.lpt_partition(costs, world)}, f)
        else:
            assert merged is None
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_lpt_partition_properties():
    shard = _shard_module()
    costs = [7, 5, 4, 4, 3, 3, 3, 1]
    parts = shard.lpt_partition(costs, 3)
    assert sorted(i for p in parts for i in p) == list(range(len(costs)))
    # by hand: 7->r0, 5->r1, 4->r2, 4->r2 (load 4 < 5), 3->r1 (5), 3->r0 (7), 3->r1 (8, tie with r2 goes
    # to the lower rank), 1->r2 (8): loads 10, 11, 9
    assert parts == [[0, 5], [1, 4, 6], [2, 3, 7]]
    assert shard.shard_loads(costs, parts) == [10.0, 11.0, 9.0]
    assert shard.lpt_partition([3.0], 4) == [[0], [], [], []]
    with pytest.raises(ValueError):
        shard.lpt_partition(costs, 0)
    # makespan within Graham's 4/3 bound of the best possible (the total / ranks lower bound, here)
    rng = np.random.default_rng(wl.SEED)
    c = rng.integers(800, 3001, 1024) * 1.0
    loads = shard.shard_loads(c, shard.lpt_partition(c, 8))
    assert max(loads) <= (4.0 / 3.0) * max(c.sum() / 8, c.max())
    assert max(loads) - min(loads) <= c.max()


def test_two_rank_shard_and_gather_equals_single_process(tmp_path):
    import torch.multiprocessing as tmp
    path = str(tmp_path / "gather.pkl")
    world = 2
    tmp.spawn(_rank_main, args=(world, _free_port(), path), nprocs=world, join=True)
    with open(path, "rb") as f:
        got = pickle.load(f)
    wk, runs = _batch()
    ref = _propagate(runs, wk.dt, wk.nsteps, range(len(runs)))
    assert all(len(s) > 0 for s in got["shards"])
    assert len(got["merged"]) == len(runs)
    for i, (c, obs) in enumerate(got["merged"]):
        assert np.array_equal(c, ref[i][0]), i
        assert np.array_equal(obs, ref[i][1]), i


def test_gather_single_process_passthrough():
    shard = _shard_module()
    assert shard.gather_runs({1: "b", 0: "a"}, 2) == ["a", "b"]
    with pytest.raises(RuntimeError):
        shard.gather_runs({0: "a"}, 2)
