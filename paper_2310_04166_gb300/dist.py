"""Data-parallel VMC step over ranks, one process per GPU.

The sampling tree splits into independent subtrees (Sec. II.C): every rank
walks the first ``split_level`` slots of the same pass (same seed and
counter), keeps its round-robin share of that frontier and samples on from
there, so the ranks' unique sets are disjoint and together are the one-GPU
sample set with the same counts.  E_loc of a sample needs nothing from other
ranks.  The one exchange of the step is the energy estimate (Eq. energy_est)
and the gradient (Eq. grad_def), both sums over all samples: the ranks
gather their four statistics, combine them on the device
(``stats_combine``), take the gradient of their samples against the
combined statistics, and sum the gradients.  The gathers and sums go through
``torch.distributed`` (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import math

import torch
import torch.distributed as dist

from . import (Hamiltonian, Model, grad, grad_workspace_bytes, local_energy, local_energy_workspace_bytes,
               sample_shard_into, sample_workspace_bytes, stats_combine)


def default_split_level(n_orb: int, world: int) -> int:
    """First slot level whose frontier can hold 4 nodes per rank (4^p >= 4 world)."""
    if world <= 1:
        return 0
    return min(n_orb, 1 + math.ceil(math.log(world, 4)))


def exchange_stats(stats: torch.Tensor, group=None) -> torch.Tensor:
    """Every rank's [4] statistics, gathered into [world, 4] on every rank."""
    world = dist.get_world_size(group)
    parts = [torch.empty_like(stats) for _ in range(world)]
    dist.all_gather(parts, stats.contiguous(), group=group)
    return torch.stack(parts)


def reduce_grad(g: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of the ranks' gradient contributions, in place."""
    dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return g


class ShardedStep:
    """One rank's buffers for repeated sharded VMC passes of a fixed size."""

    def __init__(self, model: Model, ham: Hamiltonian, n_samples: int, seed: int, split_level: int | None = None,
                 group=None):
        self.model, self.ham, self.n_samples, self.seed, self.group = model, ham, int(n_samples), int(seed), group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.split_level = default_split_level(model.n_orb, self.world) if split_level is None else split_level
        dev = model.params.device
        cap = min(self.n_samples, ham.sector_dim)
        i64, f64 = dict(dtype=torch.int64, device=dev), dict(dtype=torch.float64, device=dev)
        self.x, self.n = torch.empty(cap, **i64), torch.empty(cap, **i64)
        self.n_unique = torch.zeros(1, **i64)
        self.ere, self.eim, self.stats = torch.empty(cap, **f64), torch.empty(cap, **f64), torch.empty(4, **f64)
        self.stats_global = torch.empty(4, **f64)
        self.g = torch.empty(model.n_params, dtype=torch.float32, device=dev)
        u8 = dict(dtype=torch.uint8, device=dev)
        self.ws_s = torch.empty(sample_workspace_bytes(model, ham, self.n_samples), **u8)
        self.ws_e = torch.empty(local_energy_workspace_bytes(model, ham, cap), **u8)
        self.ws_g = torch.empty(grad_workspace_bytes(model, ham, cap), **u8)

    def __call__(self, counter: int = 0, counter_dev: torch.Tensor | None = None):
        """(global stats f64[4], summed gradient f32[n_params]) of one pass."""
        sample_shard_into(self.model, self.ham, self.n_samples, self.seed, counter, self.rank, self.world,
                          self.split_level, self.x, self.n, self.n_unique, self.ws_s, counter_dev=counter_dev)
        local_energy(self.model, self.ham, self.x, self.n, self.ws_e, n_dev=self.n_unique,
                     out=(self.ere, self.eim, self.stats))
        st = exchange_stats(self.stats, self.group) if self.world > 1 else self.stats.reshape(1, 4)
        stats_combine(st, out=self.stats_global)
        grad(self.model, self.ham, self.x, self.n, self.ere, self.eim, self.stats_global, self.ws_g,
             n_dev=self.n_unique, out=self.g)
        if self.world > 1:
            reduce_grad(self.g, self.group)
        return self.stats_global, self.g
