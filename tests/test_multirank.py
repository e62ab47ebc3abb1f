"""The multi-process path of bench.py on CPU: two ranks over gloo (127.0.0.1).

Under torchrun every rank runs an independent replica of the workload (its own
seed, no data-path collective); rank 0 reports the maximum of the ranks' timed
seconds and the sum of their particle-steps.  These tests run those reductions
and the replica seeding with world_size 2, and check that the reference arm
does its work on rank 0 only."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from oracle import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        # timing reduction: the job time is the slowest rank's
        t = bench.max_over_ranks(1.0 + rank, w, "cpu")
        units = bench.sum_over_ranks(1000.0 * (rank + 1), w, "cpu")
        # replicas: each rank steps its own seeded problem with the oracle
        prob = bench.workload(4096, seed=rank)
        s = prob.species[0]
        cfg = O.ES1DConfig(nc=prob.nc, L=prob.L, order=prob.order, dt=prob.dt, scheme=2)
        sp = [O.Species(s.q, s.m, s.x.copy(), s.v.copy(), None, s.w0)]
        E = O.poisson_e0_1d(cfg, sp)
        O.es1d_step(cfg, sp, E)
        total_steps = bench.sum_over_ranks(float(len(s.x)), w, "cpu")
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.array([t, units, total_steps, s.x[0], sp[0].x[0]]))
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_ranks(tmp_path_factory):
    out = tmp_path_factory.mktemp("ranks")
    mp.spawn(_worker, args=(2, _free_port(), str(out)), nprocs=2, join=True)
    return [np.load(out / f"rank{r}.npy") for r in range(2)]


def test_max_and_sum_over_ranks(two_ranks):
    for r in two_ranks:
        assert r[0] == 2.0          # max of 1.0 and 2.0
        assert r[1] == 3000.0       # 1000 + 2000
        assert r[2] == 2 * 4096.0   # particle-steps of both replicas


def test_replicas_have_their_own_seed(two_ranks):
    assert two_ranks[0][3] != two_ranks[1][3]   # different initial markers
    assert two_ranks[0][4] != two_ranks[1][4]   # and different stepped states


def test_reference_arm_runs_on_rank0_only(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    ns = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    assert bench.run_reference(ns) is None
    assert capsys.readouterr().out == ""
