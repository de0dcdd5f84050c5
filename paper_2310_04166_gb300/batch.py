"""Many independent problems (Hamiltonian + ansatz) stepped together.

Each problem's VMC pass (sampling, local energies with their statistics,
gradient) runs on its own CUDA stream; the passes of all problems are
captured into one CUDA graph (fork from the capturing stream, join back), so
one replay launches every problem's kernels and the GPU runs problems of
different sizes side by side.  With `persistent=True` the local energies of
all problems come from one anqs_batched_local_energy call between the
samplers and the gradients: the 16-bit MLP problems' amplitude stage then
runs as one persistent launch over every (problem, slot, tile), with the
schedule the handle's autotuner picked.  All sizes stay on the device
(unique counts, Philox counters), as for a single problem.  Argument
marshalling only: every step runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import _lib
from . import (EnergyBatch, Hamiltonian, Model, grad, grad_workspace_bytes, local_energy,
               local_energy_workspace_bytes, sample_into, sample_workspace_bytes, _ws)


class Problem:
    """Buffers of one problem's pass (N_s samples, at most min(N_s, sector) unique)."""

    def __init__(self, ham: Hamiltonian, model: Model, n_samples: int, seed: int):
        self.ham, self.model, self.n_samples, self.seed = ham, model, int(n_samples), int(seed)
        dev = model.params.device
        cap = min(self.n_samples, ham.sector_dim)
        i64, f64 = dict(dtype=torch.int64, device=dev), dict(dtype=torch.float64, device=dev)
        self.x, self.cnt = torch.empty(cap, **i64), torch.empty(cap, **i64)
        self.nu, self.ctr = torch.zeros(1, **i64), torch.zeros(1, **i64)
        self.ere, self.eim, self.stats = torch.zeros(cap, **f64), torch.zeros(cap, **f64), torch.zeros(4, **f64)
        self.g = torch.zeros(model.n_params, dtype=torch.float32, device=dev)
        self.ws_s = _ws(sample_workspace_bytes(model, ham, self.n_samples), dev)
        self.ws_e = _ws(local_energy_workspace_bytes(model, ham, cap), dev)
        self.ws_g = _ws(grad_workspace_bytes(model, ham, cap), dev)

    def sample(self, stream=None):
        m = self.model
        if m.desc.form == _lib.ANQS_FORM_BF16:
            m.sync(stream)
        sample_into(m, self.ham, self.n_samples, self.seed, 0, self.x, self.cnt, self.nu, self.ws_s, stream,
                    counter_dev=self.ctr)

    def energy_item(self) -> dict:
        """This problem's arguments of a batched local-energy call."""
        return dict(model=self.model, ham=self.ham, x=self.x, counts=self.cnt, n_dev=self.nu, workspace=self.ws_e,
                    out=(self.ere, self.eim, self.stats))

    def gradient(self, stream=None):
        grad(self.model, self.ham, self.x, self.cnt, self.ere, self.eim, self.stats, workspace=self.ws_g,
             stream=stream, n_dev=self.nu, out=self.g)
        s = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(s):
            self.ctr.add_(1)

    def step(self, stream=None):
        """One pass on the current (or given) stream; the counter advances on the device."""
        self.sample(stream)
        local_energy(self.model, self.ham, self.x, self.cnt, workspace=self.ws_e, stream=stream, n_dev=self.nu,
                     out=(self.ere, self.eim, self.stats))
        self.gradient(stream)


class BatchedStep:
    """All problems' passes in one CUDA graph (one stream per problem; with
    persistent=True the local energies in one batched call)."""

    def __init__(self, problems: list[Problem], persistent: bool = False):
        self.problems = problems
        self.streams = [torch.cuda.Stream() for _ in problems]
        self.graph = None
        self.energy = EnergyBatch(len(problems)) if persistent else None

    def _each(self, fn):
        main = torch.cuda.current_stream()
        for p, s in zip(self.problems, self.streams):
            s.wait_stream(main)
            with torch.cuda.stream(s):
                fn(p, s)
        for s in self.streams:
            main.wait_stream(s)

    def _fork_join(self):
        if self.energy is None:
            self._each(lambda p, s: p.step(s))
            return
        self._each(lambda p, s: p.sample(s))
        self.energy.local_energy([p.energy_item() for p in self.problems])
        self._each(lambda p, s: p.gradient(s))

    def autotune(self):
        """Pick the persistent launch's schedule on the current sample sets
        (run one eager pass first so that they exist)."""
        return self.energy.autotune([p.energy_item() for p in self.problems])

    def eager(self):
        self._fork_join()

    def capture(self):
        self._fork_join()  # allocate lazily-created resources outside the capture
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._fork_join()
        return self

    def replay(self):
        self.graph.replay()

    def n_unique(self) -> int:
        return int(torch.stack([p.nu for p in self.problems]).sum().item())
