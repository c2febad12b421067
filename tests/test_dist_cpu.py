"""The bench's N > 1 host logic on CPU ranks (gloo, world size 2, 127.0.0.1).

bench.py runs one process per GPU; the problem does not shard, so every rank
runs its own replica (Philox instance = rank) and the only cross-rank steps are
the barrier and the max-over-ranks of the timed durations.  Here two spawned
processes run those steps over gloo:
  * dist_env reads (world, rank, local rank) from the torchrun variables;
  * max_over_ranks returns the slowest rank's time on every rank;
  * job_rate counts the units of all ranks over that time (weak scaling);
  * the reference arm's other ranks exit without work;
  * different instances draw different noise (independent replicas), the same
    instance the same noise.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.dist_env()
    dist.barrier()
    t = bench.max_over_ranks(0.25 * (rank + 1), dist, "cpu")
    rate = bench.job_rate(w, 6553600 * 5, t)
    q.put((rank, w, r, lr, t, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_time_and_rate():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    for rank, w, r, lr, t, rate in res:
        assert (w, r, lr) == (2, rank, rank)
        assert t == 0.5                                 # the slower rank's time on both
        assert rate == pytest.approx(2 * 6553600 * 5 / 0.5, rel=1e-15)


def test_single_process_defaults(monkeypatch):
    import bench
    for v in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(v, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.max_over_ranks(0.75, None, "cpu") == 0.75
    assert bench.job_rate(1, 100, 0.5) == 200.0


def test_reference_arm_other_ranks_exit(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    calls = []
    monkeypatch.setattr(bench, "oracle_updates", lambda *a, **k: calls.append(a) or (1, [1.0]))

    class Args:
        warmup, steps, gpus = 3, 5, 2
    assert bench.run_reference(Args()) == 0 and not calls


def test_replicas_draw_independent_noise(orc):
    from paper_2302_11719_gb300 import inputs as I
    pr = I.single_problem(K=8, T=10)
    m = orc.Model(pr.params, pr.track)
    a0 = orc.noise_block(m, 0, 0, range(8), 10)
    a0b = orc.noise_block(m, 0, 0, range(8), 10)
    a1 = orc.noise_block(m, 0, 1, range(8), 10)
    assert np.array_equal(a0, a0b)
    assert not np.any(a0 == a1)
