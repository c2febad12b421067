"""The bench's N > 1 host logic on CPU ranks (gloo, world size 2, 127.0.0.1).

bench.py runs one process per GPU.  By default every rank runs its own replica
(Philox instance = rank) and the only cross-rank steps are the barrier and the
max-over-ranks of the timed durations; with --shard-rollouts the ranks split
the K rollouts of one problem and exchange their slice partials by an
all-gather before the merge.  Here two spawned processes run those steps over
gloo:
  * the sharded update: each rank's slice partial, the all-gather and the
    merge give every rank the unsharded update's V+ (oracle arithmetic on the
    CPU ranks; the CUDA partial and merge are checked on the GPU);
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


def _shard_rank_main(rank, world, port, q):
    """One rank of the sharded update: its slice of the K rollouts (the
    binding's shard_range), the slice partial (m_g, eta_g, A_g) of Eq. 10-11,
    an all-gather of the partials over gloo and the merge."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import oracle as orc
    from paper_2302_11719_gb300 import inputs as I
    from paper_2302_11719_gb300.smppi import shard_range
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pr = I.single_problem(K=200, T=16)
    m = orc.Model(pr.params, pr.track)
    k_lo, k_hi = shard_range(m.K, world, rank)
    S = np.array([orc.rollout(m, pr.x0, pr.V, k, 4, 2)[0] for k in range(k_lo, k_hi)])
    mine = torch.from_numpy(orc.partial(m, S, k_lo, 4, 2))
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine)
    Vm = orc.merge(m, np.stack([p.numpy() for p in parts]), pr.V)
    q.put((rank, k_lo, k_hi, Vm))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_rollouts(orc):
    """Two ranks each run half of the K rollouts of one iteration; after the
    all-gather and the merge both hold the unsharded iteration's V+."""
    from paper_2302_11719_gb300 import inputs as I
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    assert [(r[1], r[2]) for r in res] == [(0, 100), (100, 200)]
    assert np.array_equal(res[0][3], res[1][3])          # every rank merges the same V+
    pr = I.single_problem(K=200, T=16)
    _, Vp = orc.mppi_step(orc.Model(pr.params, pr.track), pr.x0, pr.V, 4, 2)
    assert np.max(np.abs(res[0][3] - Vp)) < 1e-13


def test_shard_range_partitions():
    from paper_2302_11719_gb300.smppi import shard_range
    for K, world in ((65536, 8), (1000, 3), (7, 7), (10, 4)):
        sl = [shard_range(K, world, r) for r in range(world)]
        assert sl[0][0] == 0 and sl[-1][1] == K
        assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
        sizes = [b - a for a, b in sl]
        assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        shard_range(3, 4, 0)


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
