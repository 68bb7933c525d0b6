"""The multi-GPU host logic on CPU with two gloo ranks: whole meshes of a batch
are sharded without overlap and balanced by cells, the timed duration is the
slowest rank's, the job's units are summed, and the per-rank oracle residuals
of a sharded batch are those of the whole batch (no data crosses ranks)."""
import os
import socket

import numpy as np
import pytest

from paper_1602_02694_gb300.replicas import shard_meshes


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shards_cover_every_mesh_once_and_balance_cells():
    rng = np.random.default_rng(5)
    sizes = [2 * int(n) ** 2 for n in rng.choice(np.arange(16, 257, 8), size=48)]
    for world in (1, 2, 3, 4, 8):
        parts = shard_meshes(sizes, world)
        assert len(parts) == world
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[k] for k in p) for p in parts]
        # greedy largest-first: the spread is at most the largest mesh
        assert max(loads) - min(loads) <= max(sizes)
        assert all(p == sorted(p) for p in parts)
    assert shard_meshes([5, 5], 4)[2:] == [[], []]
    with pytest.raises(ValueError):
        shard_meshes([1], 0)


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from oracle import wlseno_oracle as O
    from paper_1602_02694_gb300 import synth
    from paper_1602_02694_gb300.replicas import max_over_ranks, shard_meshes, sum_over_ranks, whole_job_rate

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        meshes = [synth.tri_mesh(n, seed=60 + n) for n in (4, 5, 6)]
        parts = shard_meshes([m.n_cells for m in meshes], world)
        mine = parts[rank]
        res = {}
        for k in mine:
            m = meshes[k]
            prob = O.Problem(m.vertices, m.cells, m.period, p=3, ring=1.0, pde=O.BURGERS)
            res[k] = O.residual(prob, synth.burgers_2d_initial(m))
        cells = sum(meshes[k].n_cells for k in mine)
        ms = 10.0 + 5.0 * rank  # a rank-dependent duration
        slowest = max_over_ranks(ms, dist)
        total = sum_over_ranks(cells, dist)
        rate, slow2 = whole_job_rate(cells, ms, dist)
        out.put((rank, mine, {k: v.tolist() for k, v in res.items()}, slowest, total, rate, slow2))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_time_and_sum():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    import queue
    import time

    got = []
    deadline = time.time() + 300
    while len(got) < len(procs):
        try:
            got.append(q.get(timeout=2))
        except queue.Empty:
            failed = [p.exitcode for p in procs if p.exitcode not in (None, 0)]
            if failed or time.time() > deadline:
                for p in procs:
                    p.kill()
                pytest.fail(f"a rank failed (exit codes {[p.exitcode for p in procs]})")
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    from oracle import wlseno_oracle as O
    from paper_1602_02694_gb300 import synth

    meshes = [synth.tri_mesh(n, seed=60 + n) for n in (4, 5, 6)]
    owned = sorted(k for g in got for k in g[1])
    assert owned == [0, 1, 2]
    total_cells = sum(m.n_cells for m in meshes)
    for rank, mine, res, slowest, total, rate, slow2 in got:
        assert slowest == 15.0 and slow2 == 15.0  # the slower rank's time on both
        assert total == total_cells
        assert abs(rate - total_cells / 15e-3) <= 1e-9 * rate
        for k, L in res.items():
            m = meshes[int(k)]
            prob = O.Problem(m.vertices, m.cells, m.period, p=3, ring=1.0, pde=O.BURGERS)
            assert np.array_equal(np.asarray(L), O.residual(prob, synth.burgers_2d_initial(m)))
