"""The multi-process path of bench.py on CPU: two gloo ranks (spawned, on
127.0.0.1) reduce their timed seconds to the slowest one, the job value
counts every rank's replica, and only rank 0 runs the reference arm."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench._dist()
        t = bench._max_over_ranks(1.5 + rank, w, torch.device("cpu"))
        v = bench._job_value(1000, 10, w, t)
        q.put((r, w, t, v))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got)
    assert all(g[2] == 2.5 for g in got)                       # max(1.5, 2.5)
    assert all(g[3] == pytest.approx(1000 * 10 * 2 / 2.5) for g in got)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.main() == 0
    assert capsys.readouterr().out == ""


def _shard_rank_main(rank, world, port, q):
    """One rank of the scene split: step its share of 12 small scenes (the
    oracle stands in for the GPU library on CPU) and gather every rank's
    results."""
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2311_15088_gb300 import shard

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        scs = _small_scenes()
        parts = shard.assign([shard.scene_weight(sc) for sc in scs], world)
        local = {}
        for k in parts[rank]:
            sc = scs[k]
            o = oracle.step(sc["params"], sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
            local[k] = (rank, o["new_fluid_pos"], o["new_boid_vel"])
        out, owner = shard.gather(local, len(scs), world)
        q.put((rank, parts, [(r, fp.tobytes(), bv.tobytes()) for r, fp, bv in out], owner))
    finally:
        dist.destroy_process_group()


def _small_scenes():
    from paper_2311_15088_gb300 import scenes

    rng = np.random.default_rng(4)
    out = []
    for k in range(12):
        n = int(rng.integers(150, 1200))
        sc = scenes.scaled_block(n, int(rng.integers(0, 12)), (0.4, 0.4, 0.4), (0.4, 0.25, 0.4), seed=50 + k)
        out.append(sc)
    return out


def test_two_gloo_ranks_split_the_scenes():
    """Every scene is stepped by exactly one rank (the one the bin-pack gave
    it), every rank ends with all results in scene order, and each result
    is bit for bit the scene stepped alone."""
    import oracle

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    # read the results before joining: a child holding a large queued item
    # cannot exit until it has been read
    got = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    scs = _small_scenes()
    parts = got[0][1]
    assert got[1][1] == parts and sorted(parts[0] + parts[1]) == list(range(len(scs)))
    assert got[0][2] == got[1][2] and got[0][3] == got[1][3]
    for k, (r, fp, bv) in enumerate(got[0][2]):
        assert k in parts[r] and got[0][3][k] == r
        sc = scs[k]
        o = oracle.step(sc["params"], sc["fluid_pos"], sc["fluid_vel"], sc["boid_pos"], sc["boid_vel"])
        assert fp == o["new_fluid_pos"].tobytes() and bv == o["new_boid_vel"].tobytes()
