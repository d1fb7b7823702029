"""The exchange step of data parallelism over walkers, on host processes.

Two gloo ranks on 127.0.0.1 each hold half of every geometry's walkers.  Their
local sums and gradient shares come from the oracle (FP64), and
paper_2011_07125_gb300.replicas adds them over the ranks.  The result must be
the oracle's gradient of the whole batch (Eq. 2), and a reduction that skipped
the first exchange (per-rank mean energies) must not be.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2011_07125_gb300 import synth

WORLD = 2


def _case():
    """Two geometries of a two-centre, four-electron system; 12 + 8 walkers."""
    net = synth.Net(2, 16, 8, 2, 2, 2, 2)
    geoms = [synth.Geometry(np.array([[0.0, 0.0, -0.7], [0.0, 0.0, 0.7]]), np.array([2.0, 1.0])),
             synth.Geometry(np.array([[0.0, 0.0, -1.1], [0.0, 0.0, 1.1]]), np.array([2.0, 1.0]))]
    counts = [12, 8]
    wl = synth.Workload("two-centre", net, geoms, counts, 1.0, 1, 0.02, "fp32", True)
    P = synth.init_params(oracle.layout(net), seed=5)
    x = synth.init_walkers(wl, seed=6).astype(np.float64)
    geo = synth.geometry_of_walkers(counts)
    eloc = oracle.local_energy(net, P, geoms, x, geo=geo)["eloc"]
    return net, geoms, counts, P, x, geo, eloc


def _shard(counts, rank, world):
    """Indices of this rank's walkers: a contiguous share of every geometry."""
    idx, off = [], 0
    for c in counts:
        per = c // world
        lo = off + rank * per
        hi = off + (c if rank == world - 1 else (rank + 1) * per)
        idx.extend(range(lo, hi))
        off += c
    return np.array(idx, np.int64)


def _local(net, geoms, P, x, geo, eloc, G):
    import torch
    sums = torch.tensor([eloc[geo == g].sum() for g in range(G)], dtype=torch.float64)
    cnts = torch.tensor([float((geo == g).sum()) for g in range(G)], dtype=torch.float64)

    def partial(esum, cnt):
        esum, cnt = esum.numpy(), cnt.numpy()
        em = esum / cnt
        seeds = 2.0 * (eloc - em[geo]) / cnt[geo]
        return torch.from_numpy(em), torch.from_numpy(oracle.logpsi_vjp(net, P, geoms, x, seeds, geo=geo))

    return sums, cnts, partial


def _worker(rank, world, port, q):
    import datetime

    import torch.distributed as dist

    from paper_2011_07125_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
        net, geoms, counts, P, x, geo, eloc = _case()
        idx = _shard(counts, rank, world)
        sums, cnts, partial = _local(net, geoms, P, x[idx], geo[idx], eloc[idx], len(geoms))
        em, grad = replicas.reduce_energy_grad(sums, cnts, partial)
        # the same shares with each rank's own mean energy (no first exchange)
        em_l = sums / cnts
        g_l = partial(em_l * cnts * world, cnts * world)[1].clone()
        dist.all_reduce(g_l)
        q.put((rank, em.numpy(), grad.numpy(), g_l.numpy(), None))
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent
        q.put((rank, None, None, None, repr(e)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shards_partition_the_batch():
    counts = [12, 8, 5]
    idx = np.concatenate([_shard(counts, r, 3) for r in range(3)])
    assert np.array_equal(np.sort(idx), np.arange(sum(counts)))


def test_single_process_reduction_is_the_plain_gradient():
    """Without a process group the reduction is the single-batch estimator."""
    from paper_2011_07125_gb300 import replicas
    net, geoms, counts, P, x, geo, eloc = _case()
    sums, cnts, partial = _local(net, geoms, P, x, geo, eloc, len(geoms))
    em, grad = replicas.reduce_energy_grad(sums, cnts, partial)
    em_o, g_o = oracle.energy_grad(net, P, geoms, x, eloc, geo=geo)
    np.testing.assert_allclose(em.numpy(), em_o, rtol=1e-14, atol=0)
    np.testing.assert_allclose(grad.numpy(), g_o, rtol=1e-10, atol=1e-12 * np.abs(g_o).max())


def test_two_rank_gloo_reduction_matches_whole_batch():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    res = {}
    try:
        for _ in range(WORLD):
            rank, em, grad, g_l, err = q.get(timeout=300)
            assert err is None, f"rank {rank}: {err}"
            res[rank] = (em, grad, g_l)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    net, geoms, counts, P, x, geo, eloc = _case()
    em_o, g_o = oracle.energy_grad(net, P, geoms, x, eloc, geo=geo)
    scale = np.abs(g_o).max()
    for r in range(WORLD):
        em, grad, g_l = res[r]
        np.testing.assert_allclose(em, em_o, rtol=1e-13, atol=0)
        np.testing.assert_allclose(grad, g_o, rtol=1e-9, atol=1e-11 * scale)
        # every rank ends with the same gradient
        assert np.array_equal(grad, res[0][1])
        # per-rank means differ from the batch mean, and so does that gradient
        assert np.abs(g_l - g_o).max() > 1e-6 * scale
