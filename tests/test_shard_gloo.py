"""Multi-rank particle sharding on CPU: 2 gloo ranks, each sums its particle range with the FP64
oracle, one all-reduce; the result equals the oracle on the whole ensemble. Trajectories shard the
same way: with global particle ids each particle keeps its random stream, so the sharded records
equal the single-process ones bit for bit. A rank that leaves is detected by the next
collective."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1910_10391_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle as O
    from paper_1910_10391_gb300 import inputs as I
    from paper_1910_10391_gb300 import shard as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tr = I.channeling(7, 10e9, +1, 300, 5e-9, seed=21)
    tr.weight = np.full(7, 1.0 / 7)
    grid = I._ensemble_grid(10e9, 20.0, 6, 4)
    p0, p1 = S.particle_range(tr.n_particles, world, rank)
    part = O.spectrum_cube(tr.subset(range(p0, p1)), grid, O.CLASSICAL) if p1 > p0 else np.zeros((6, 16))
    t = torch.from_numpy(part.copy())
    S.allreduce_sum(t)
    if rank == 0:
        out.put(t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_particle_shards_sum_to_ensemble():
    import oracle as O
    from paper_1910_10391_gb300 import inputs as I
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    tr = I.channeling(7, 10e9, +1, 300, 5e-9, seed=21)
    tr.weight = np.full(7, 1.0 / 7)
    ref = O.spectrum_cube(tr, I._ensemble_grid(10e9, 20.0, 6, 4), O.CLASSICAL)
    np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_partition_and_batches():
    for n, w in [(7, 2), (1024, 8), (3, 4)]:
        ranges = [shard.particle_range(n, w, r) for r in range(w)]
        assert ranges[0][0] == 0 and ranges[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
        assert max(b - a for a, b in ranges) - min(b - a for a, b in ranges) <= 1
    seen = set()
    for r in range(4):
        p0, p1 = shard.step_batch(3, r, 4, 32, 1024)
        assert p1 - p0 == 32 and p0 not in seen
        seen.add(p0)
    with pytest.raises(ValueError):
        shard.particle_range(5, 2, 2)


def _worker_leaves(rank, world, port, out):
    """Rank 1 leaves after the rendezvous, between steps; rank 0's next collective must fail with
    an error within the process group's timeout instead of hanging."""
    import datetime
    import time
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(0)  # leaves without joining the reduction of the next step
    t0 = time.perf_counter()
    try:
        shard.allreduce_sum(torch.zeros(4, dtype=torch.float64))
        out.put(("no error", time.perf_counter() - t0))
    except Exception as e:  # the failure is detected on the host
        out.put((type(e).__name__, time.perf_counter() - t0))


def test_rank_that_leaves_is_detected_by_the_next_collective():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_leaves, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    kind, dt = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    assert kind != "no error", "the all-reduce with a departed rank returned normally"
    assert dt < 60.0


def _worker_traj(rank, world, port, out):
    """Each rank integrates its particle range with the global particle ids (so every particle
    keeps its own random stream) and one all-reduce of the zero-padded records assembles the
    ensemble."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import traj as T
    from paper_1910_10391_gb300 import inputs as I
    from paper_1910_10391_gb300 import shard as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, L = 7, 400
    rng = np.random.default_rng(5)
    x0, th = rng.uniform(0, I.SI110_DP, n), rng.normal(0, 2e-5, n)
    pot = T.PlanarPotential(I.SYNTH_DT_A, I.SYNTH_DT_B, I.SI_N, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX,
                            I.SI_I_EV)
    p0, p1 = S.particle_range(n, world, rank)
    full = np.zeros((n, L, 10))
    if p1 > p0:
        full[p0:p1] = T.trajectories(x0[p0:p1], th[p0:p1], 0.0, 20e9, L, 5e-9, 17, charge=-1, pot=pot, ms_el=True,
                                     ll=True, ms_loss=True, particle_ids=np.arange(p0, p1))
    t = torch.from_numpy(full)
    S.allreduce_sum(t)
    if rank == 0:
        out.put(t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_trajectories_keep_their_random_streams():
    from oracle import traj as T
    from paper_1910_10391_gb300 import inputs as I
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_traj, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=180)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    n, L = 7, 400
    rng = np.random.default_rng(5)
    x0, th = rng.uniform(0, I.SI110_DP, n), rng.normal(0, 2e-5, n)
    pot = T.PlanarPotential(I.SYNTH_DT_A, I.SYNTH_DT_B, I.SI_N, I.SYNTH_DT_AX, I.SYNTH_DT_BX, I.SYNTH_DT_CX,
                            I.SI_I_EV)
    ref = T.trajectories(x0, th, 0.0, 20e9, L, 5e-9, 17, charge=-1, pot=pot, ms_el=True, ll=True, ms_loss=True)
    assert np.array_equal(got, ref)
    # and the streams differ between particles: no two particles received the same kicks
    kicks = np.diff(ref[:, :, 4], axis=1)
    assert len({float(k) for k in kicks[:, 10]}) == n
