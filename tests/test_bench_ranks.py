"""Host logic of the bench's multi-process launch (replicas), on CPU with two gloo ranks.

Every rank times its own instance; the job's step time is the maximum over ranks and the
value counts all ranks' pair-modes over that time.  The reference arm runs on rank 0 only.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    step = bench.job_step_ms(10.0 + 5.0 * rank, world, dist, device="cpu")
    out[rank] = (step, bench.job_value(3.1e9, world, step))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    import torch.multiprocessing as mp

    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        step, value = res[rank]
        assert step == 15.0
        assert value == pytest.approx(world * 3.1e9 / 15e-3 / 1e9)


def test_rank_forces_are_distinct_and_reproducible():
    import bench
    from paper_2105_08798_gb300 import inputs

    w = inputs.WORKLOADS["ring200x300_L16_iso"]
    f0, f1 = bench.rank_forces(w, 0), bench.rank_forces(w, 1)
    assert f0.shape == f1.shape == (w.n_rhs, w.n_i, w.L, 3)
    assert not np.array_equal(f0, f1)
    np.testing.assert_array_equal(f0, bench.rank_forces(w, 0))


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.job_step_ms(12.5, 1) == 12.5
    assert bench.job_value(1e9, 1, 1.0) == pytest.approx(1000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out == ""
