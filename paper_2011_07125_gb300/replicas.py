"""Data parallelism over walkers: the exchange step of a VMC gradient whose
batch is split over several processes.

The expectation of Eq. 2 and the mean energy in its gradient run over every
walker of the batch, and each walker's weight is E_L minus that mean, so the
gradient takes two exchanges (all-reduces over torch.distributed: NCCL between
GPUs, gloo between host processes):

1. each geometry's FP64 energy sum and walker count, added over the processes,
   give the batch mean E_mean,g;
2. each process weights its own walkers by 2 (E_L,w - E_mean,g) / count_g and
   runs its adjoint, and the FP64 gradient shares are added.

Everything else in a VMC step (Metropolis moves, the local energy) is per
walker and needs no exchange.
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple


def _world(group) -> int:
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 1
    return dist.get_world_size(group)


def reduce_energy_grad(local_sums, local_counts, partial_grad: Callable, group=None) -> Tuple[object, object]:
    """Two-phase reduction of the VMC energy gradient.

    local_sums, local_counts: float64 tensors [G] (this process's energy sum
    and walker count per geometry).  partial_grad(sums, counts), given the
    batch-wide sums and counts, returns (emean [G], this process's float64
    gradient share [P]); the division happens behind the C ABI.
    Returns (emean [G], grad [P]), float64 and identical on every process.
    """
    import torch
    import torch.distributed as dist
    G = local_sums.numel()
    buf = torch.cat([local_sums.reshape(-1), local_counts.reshape(-1)]).to(torch.float64)
    if _world(group) > 1:
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    sums, counts = buf[:G].contiguous(), buf[G:].contiguous()
    emean, grad = partial_grad(sums, counts)
    grad = grad.to(torch.float64)
    if _world(group) > 1:
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return emean, grad


def energy_grad(fn, x, eloc, group=None):
    """VMC energy gradient over the batch split across the processes of
    `group`, each holding its walkers x and local energies eloc on its GPU
    (fn: a binding.FermiNet).  Returns (emean [G], grad [P]) as float64."""
    B = x.shape[0]
    return reduce_energy_grad(fn.energy_sums(eloc), fn.walker_counts(B),
                              lambda sums, cnt: fn.energy_grad_partial(x, eloc, sums, cnt), group)
