"""Variational Monte Carlo optimisation of the ansatz on the GPU.

One iteration is the paper's training step (Sec. II.A-C): statistics
sampling of N_s samples from |psi|^2, the local energies of the unique
samples and the count-weighted energy estimate (Eq. energy_est), the
gradient of Eq. grad_def from the library's adjoint, and an Adam update of
the flat parameters (the paper trains with Adam).  Every step of the VMC
pass runs in the library's kernels; the parameter update is a PyTorch
optimizer on the parameter tensor the model reads.
"""
from __future__ import annotations

import torch

from . import _lib
from . import Hamiltonian, Model, grad, grad_workspace_bytes, local_energy, local_energy_workspace_bytes
from . import sample_into, sample_workspace_bytes, _ws


class VMC:
    """Optimiser state and preallocated buffers for repeated VMC iterations."""

    def __init__(self, model: Model, ham: Hamiltonian, n_samples: int, lr: float = 1e-2, seed: int = 0,
                 binomial: bool = False, betas=(0.9, 0.999)):
        self.model, self.ham, self.n_samples, self.seed, self.binomial = model, ham, int(n_samples), int(seed), binomial
        self.params = model.params
        dev = self.params.device
        cap = min(self.n_samples, ham.sector_dim)
        i64, f64 = dict(dtype=torch.int64, device=dev), dict(dtype=torch.float64, device=dev)
        self.x, self.cnt = torch.empty(cap, **i64), torch.empty(cap, **i64)
        self.nu, self.ctr = torch.zeros(1, **i64), torch.zeros(1, **i64)
        self.ere, self.eim, self.stats = torch.zeros(cap, **f64), torch.zeros(cap, **f64), torch.zeros(4, **f64)
        self.g = torch.zeros(model.n_params, dtype=torch.float32, device=dev)
        self.ws_s = _ws(sample_workspace_bytes(model, ham, self.n_samples), dev)
        self.ws_e = _ws(local_energy_workspace_bytes(model, ham, cap), dev)
        self.ws_g = _ws(grad_workspace_bytes(model, ham, cap), dev)
        self.opt = torch.optim.Adam([self.params], lr=lr, betas=betas)

    def step(self) -> torch.Tensor:
        """One iteration; returns the statistics (Re E, Im E, Var, sum n) of
        the samples it drew (before the update)."""
        m = self.model
        if m.desc.form == _lib.ANQS_FORM_BF16:
            m.sync()
        sample_into(m, self.ham, self.n_samples, self.seed, 0, self.x, self.cnt, self.nu, self.ws_s,
                    counter_dev=self.ctr, binomial=self.binomial)
        local_energy(m, self.ham, self.x, self.cnt, workspace=self.ws_e, n_dev=self.nu,
                     out=(self.ere, self.eim, self.stats))
        grad(m, self.ham, self.x, self.cnt, self.ere, self.eim, self.stats, workspace=self.ws_g, n_dev=self.nu,
             out=self.g)
        self.ctr.add_(1)
        self.params.grad = self.g
        self.opt.step()
        return self.stats.clone()
