"""Symmetry-masked autoregressive VMC hot path on one GB300 (libanqs).

Thin Python binding over the C ABI of ``include/anqs.h``: argument
marshalling only.  PyTorch provides device memory and streams; every step of
the computation runs in the library's CUDA kernels.  If ``lib/libanqs.so``
has not been built, every call raises.

    ham   = Hamiltonian(h, g, e_nuc, n_alpha, n_beta)
    model = Model.mlp(n_orb, width, n_hidden, params_cuda_f32, form="bf16")
    x, n  = sample(model, ham, n_samples, seed)
    eloc_re, eloc_im, stats = local_energy(model, ham, x, n)
    g     = grad(model, ham, x, n, eloc_re, eloc_im, stats)
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import AnqsError, ModelDesc, check

__all__ = ["Hamiltonian", "Model", "EnergyBatch", "connected", "logpsi", "logpsi_vjp", "sample", "sample_into",
           "local_energy", "grad", "LogPsi", "AnqsError", "library_path"]


def library_path() -> str:
    return _lib.LIB_PATH


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _u64(t: torch.Tensor) -> torch.Tensor:
    if t.dtype not in (torch.int64, torch.uint64):
        raise TypeError("determinants and counts are 64-bit integer tensors")
    return t.contiguous()


class Hamiltonian:
    """Integrals and (N_alpha, N_beta) sector on the current CUDA device."""

    def __init__(self, h, g, e_nuc: float, n_alpha: int, n_beta: int):
        lib = _lib.load()
        h = np.ascontiguousarray(h, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        n = h.shape[0]
        if h.shape != (n, n) or g.shape != (n, n, n, n):
            raise ValueError("h must be n x n and g n x n x n x n")
        self.n, self.n_alpha, self.n_beta, self.nz = n, n_alpha, n_beta, 0
        self.device = torch.cuda.current_device()
        hp = C.c_void_p()
        check(lib.anqs_hamiltonian_create(C.byref(hp), n, n_alpha, n_beta, h.ctypes.data, g.ctypes.data,
                                          float(e_nuc)))
        self._h = hp
        k, d = C.c_uint64(), C.c_uint64()
        check(lib.anqs_hamiltonian_info(hp, C.byref(k), C.byref(d)))
        self.n_connected, self.sector_dim = k.value, d.value

    @property
    def handle(self):
        return self._h

    def status(self, clear: bool = False) -> int:
        """Sampler event bits recorded on the device (anqs_hamiltonian_status)."""
        v = C.c_int()
        check(_lib.load().anqs_hamiltonian_status(self._h, C.byref(v), int(bool(clear))))
        return v.value

    def set_pruning(self, du_levels: int) -> "Hamiltonian":
        """MU-d (Sec. III.C): MU on the first n_orb - du_levels slots, DU on the rest."""
        check(_lib.load().anqs_hamiltonian_set_pruning(self._h, int(du_levels)))
        return self

    def set_z2(self, qubit_masks) -> "Hamiltonian":
        """Z2 symmetries (Pauli-Z strings commuting with H), one qubit mask each."""
        m = np.ascontiguousarray(np.asarray(qubit_masks, dtype=np.uint64))
        check(_lib.load().anqs_hamiltonian_set_z2(self._h, len(m), m.ctypes.data if len(m) else None))
        self.nz = len(m)
        info_k, info_d = C.c_uint64(), C.c_uint64()
        check(_lib.load().anqs_hamiltonian_info(self._h, C.byref(info_k), C.byref(info_d)))
        self.sector_dim = info_d.value
        return self

    def slot_masks(self) -> np.ndarray:
        """[n][N_a + 1][N_b + 1] (or [...][2^nz] with Z2 symmetries) outcome bits."""
        shape = (self.n, self.n_alpha + 1, self.n_beta + 1) + ((1 << self.nz,) if self.nz else ())
        out = np.zeros(shape, dtype=np.uint8)
        check(_lib.load().anqs_hamiltonian_slot_masks(self._h, out.ctypes.data, out.nbytes))
        return out

    def __del__(self):
        if getattr(self, "_h", None) and _lib._lib is not None:
            _lib._lib.anqs_hamiltonian_destroy(self._h)
            self._h = None


class Model:
    """Autoregressive ansatz over caller-owned float32 CUDA parameters.

    A model's calls may be queued on any stream, but not from several host
    threads at once: the 16-bit MLP keeps scratch rows and a second stream of
    its own (forked from and joined back into the caller's stream)."""

    def __init__(self, desc: ModelDesc, params: torch.Tensor):
        lib = _lib.load()
        if params.device.type != "cuda" or params.dtype != torch.float32 or not params.is_contiguous():
            raise TypeError("params must be a contiguous float32 CUDA tensor")
        n = C.c_uint64()
        check(lib.anqs_model_param_count(C.byref(desc), C.byref(n)))
        if params.numel() != n.value:
            raise ValueError(f"expected {n.value} parameters, got {params.numel()}")
        self.desc, self.params, self.n_params = desc, params, n.value
        mp = C.c_void_p()
        with torch.cuda.device(params.device):
            check(lib.anqs_model_create(C.byref(mp), C.byref(desc), params.data_ptr()))
        self._m = mp

    @classmethod
    def mlp(cls, n_orb, width, n_hidden, params, form="fp32"):
        d = ModelDesc(_lib.ANQS_MODEL_MLP, _form(form), n_orb, width, n_hidden, 0, 0, 0)
        return cls(d, params)

    @classmethod
    def transformer(cls, n_orb, d_model, n_heads, n_layers, params, form="fp32"):
        d = ModelDesc(_lib.ANQS_MODEL_TF, _form(form), n_orb, 0, 0, d_model, n_heads, n_layers)
        return cls(d, params)

    @classmethod
    def table(cls, n_orb, params):
        d = ModelDesc(_lib.ANQS_MODEL_TABLE, _lib.ANQS_FORM_FP32, n_orb, 0, 0, 0, 0, 0)
        return cls(d, params)

    @classmethod
    def nade(cls, n_orb, width, params):
        """Per-qubit complex NADE of Appendix B.1 (FP32 form)."""
        d = ModelDesc(_lib.ANQS_MODEL_NADE, _lib.ANQS_FORM_FP32, n_orb, width, 0, 0, 0, 0)
        return cls(d, params)

    @property
    def n_orb(self):
        return self.desc.n_orb

    def status(self) -> int:
        """0, or 1 if a bounded wait in a tensor-core kernel gave up (synchronous)."""
        v = C.c_int()
        check(_lib.load().anqs_model_status(self._m, C.byref(v)))
        return v.value

    def sync(self, stream=None):
        """Refresh internal copies after params changed (BF16 packing)."""
        check(_lib.load().anqs_model_sync(self._m, _stream(stream)))

    def __del__(self):
        if getattr(self, "_m", None) and _lib._lib is not None:
            _lib._lib.anqs_model_destroy(self._m)
            self._m = None


def _form(f):
    return {"fp32": _lib.ANQS_FORM_FP32, "bf16": _lib.ANQS_FORM_BF16}[f] if isinstance(f, str) else int(f)


def _ws(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def connected(ham: Hamiltonian, x: torch.Tensor, stream=None):
    """(xp [n_x, K], hval [n_x, K] f64, first_slot [n_x, K] u8, hdiag [n_x] f64)."""
    x = _u64(x)
    n_x, K = x.numel(), ham.n_connected
    xp = torch.empty((n_x, K), dtype=torch.int64, device=x.device)
    hv = torch.empty((n_x, K), dtype=torch.float64, device=x.device)
    js = torch.empty((n_x, K), dtype=torch.uint8, device=x.device)
    hd = torch.empty(n_x, dtype=torch.float64, device=x.device)
    check(_lib.load().anqs_connected(ham.handle, x.data_ptr(), n_x, xp.data_ptr(), hv.data_ptr(), js.data_ptr(),
                                     hd.data_ptr(), _stream(stream)))
    return xp, hv, js, hd


def logpsi(model: Model, ham: Hamiltonian, x: torch.Tensor, stream=None):
    """(log|psi(x)|, arg psi(x)) as float32 tensors."""
    x = _u64(x)
    la = torch.empty(x.numel(), dtype=torch.float32, device=x.device)
    ph = torch.empty_like(la)
    check(_lib.load().anqs_logpsi(model._m, ham.handle, x.data_ptr(), x.numel(), la.data_ptr(), ph.data_ptr(),
                                  _stream(stream)))
    return la, ph


def logpsi_vjp(model: Model, ham: Hamiltonian, x: torch.Tensor, cot_abs: torch.Tensor, cot_phase: torch.Tensor,
               stream=None):
    x = _u64(x)
    g = torch.empty(model.n_params, dtype=torch.float32, device=x.device)
    ca = cot_abs.to(torch.float32).contiguous()
    cp = cot_phase.to(torch.float32).contiguous()
    b = C.c_size_t()
    check(_lib.load().anqs_logpsi_vjp_workspace_size(model._m, ham.handle, x.numel(), C.byref(b)))
    ws = _ws(b.value, x.device) if b.value else None
    check(_lib.load().anqs_logpsi_vjp(model._m, ham.handle, x.data_ptr(), x.numel(), ca.data_ptr(), cp.data_ptr(),
                                      g.data_ptr(), _ptr(ws), b.value, _stream(stream)))
    return g


class LogPsi(torch.autograd.Function):
    """log|psi|, arg psi of determinants as a function of the flat parameters;
    the backward pass is the library's hand-written adjoint."""

    @staticmethod
    def forward(ctx, params, model, ham, x):
        ctx.model, ctx.ham = model, ham
        ctx.save_for_backward(x)
        return logpsi(model, ham, x)

    @staticmethod
    def backward(ctx, g_abs, g_phase):
        (x,) = ctx.saved_tensors
        if g_abs is None:
            g_abs = torch.zeros(x.numel(), device=x.device)
        if g_phase is None:
            g_phase = torch.zeros(x.numel(), device=x.device)
        return logpsi_vjp(ctx.model, ctx.ham, x, g_abs, g_phase), None, None, None


def sample_workspace_bytes(model: Model, ham: Hamiltonian, n_samples: int) -> int:
    b = C.c_size_t()
    check(_lib.load().anqs_sample_workspace_size(model._m, ham.handle, n_samples, C.byref(b)))
    return b.value


def sample_into(model, ham, n_samples, seed, counter, x_out, n_out, n_unique, workspace, stream=None,
                counter_dev=None, binomial=False):
    """Asynchronous sampling into preallocated device buffers (no host sync).
    With counter_dev (a 1-element int64 CUDA tensor) the Philox counter is
    counter + counter_dev[0], read on the device.  binomial=True splits each
    node's samples by chained binomials (cost independent of n_samples)."""
    fn = _lib.load().anqs_sample_binomial if binomial else _lib.load().anqs_sample
    check(fn(model._m, ham.handle, int(n_samples), int(seed) & (2**64 - 1),
                                  int(counter) & (2**64 - 1), _ptr(counter_dev), x_out.data_ptr(), n_out.data_ptr(),
                                  x_out.numel(), n_unique.data_ptr(), workspace.data_ptr(), workspace.numel(),
                                  _stream(stream)))


def sample(model: Model, ham: Hamiltonian, n_samples: int, seed: int, counter: int = 0, stream=None,
           binomial: bool = False):
    """Unique determinants and their counts (trimmed; synchronises once)."""
    dev = model.params.device
    cap = min(int(n_samples), ham.sector_dim)
    x = torch.empty(cap, dtype=torch.int64, device=dev)
    n = torch.empty(cap, dtype=torch.int64, device=dev)
    nu = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = _ws(sample_workspace_bytes(model, ham, n_samples), dev)
    sample_into(model, ham, n_samples, seed, counter, x, n, nu, ws, stream, binomial=binomial)
    k = int(nu.item())
    return x[:k], n[:k]


def sample_shard_into(model, ham, n_samples, seed, counter, rank, world, split_level, x_out, n_out, n_unique,
                      workspace, stream=None, counter_dev=None):
    """This rank's share of sample_into's pass: the level-``split_level``
    frontier is split round-robin over ``world`` ranks (asynchronous)."""
    check(_lib.load().anqs_sample_shard(model._m, ham.handle, int(n_samples), int(seed) & (2**64 - 1),
                                        int(counter) & (2**64 - 1), _ptr(counter_dev), int(rank), int(world),
                                        int(split_level), x_out.data_ptr(), n_out.data_ptr(), x_out.numel(),
                                        n_unique.data_ptr(), workspace.data_ptr(), workspace.numel(),
                                        _stream(stream)))


def sample_shard(model, ham, n_samples, seed, rank, world, split_level, counter=0, stream=None):
    """Unique determinants and counts of this rank's share (synchronises once)."""
    dev = model.params.device
    cap = min(int(n_samples), ham.sector_dim)
    x = torch.empty(cap, dtype=torch.int64, device=dev)
    n = torch.empty(cap, dtype=torch.int64, device=dev)
    nu = torch.zeros(1, dtype=torch.int64, device=dev)
    ws = _ws(sample_workspace_bytes(model, ham, n_samples), dev)
    sample_shard_into(model, ham, n_samples, seed, counter, rank, world, split_level, x, n, nu, ws, stream)
    k = int(nu.item())
    return x[:k], n[:k]


def stats_combine(stats_all: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Statistics of the union of disjoint sample sets; stats_all f64 [world, 4]
    on the device."""
    stats_all = stats_all.contiguous()
    out = out if out is not None else torch.empty(4, dtype=torch.float64, device=stats_all.device)
    check(_lib.load().anqs_stats_combine(stats_all.data_ptr(), stats_all.numel() // 4, out.data_ptr(),
                                         _stream(stream)))
    return out


def local_energy_workspace_bytes(model, ham, n_x) -> int:
    b = C.c_size_t()
    check(_lib.load().anqs_local_energy_workspace_size(model._m, ham.handle, n_x, C.byref(b)))
    return b.value


def local_energy(model: Model, ham: Hamiltonian, x: torch.Tensor, counts: torch.Tensor | None = None,
                 workspace: torch.Tensor | None = None, stream=None, n_dev: torch.Tensor | None = None,
                 out=None):
    """(eloc_re f64, eloc_im f64, stats f64[4] or None).  With n_dev (a
    1-element int64 CUDA tensor) only the first n_dev[0] rows are used."""
    x = _u64(x)
    n_x = x.numel()
    if out is None:
        ere = torch.empty(n_x, dtype=torch.float64, device=x.device)
        eim = torch.empty_like(ere)
        stats = torch.empty(4, dtype=torch.float64, device=x.device) if counts is not None else None
    else:
        ere, eim, stats = out
    if workspace is None:
        workspace = _ws(local_energy_workspace_bytes(model, ham, n_x), x.device)
    cnt = _u64(counts) if counts is not None else None
    check(_lib.load().anqs_local_energy(model._m, ham.handle, x.data_ptr(), _ptr(cnt), n_x, _ptr(n_dev),
                                        ere.data_ptr(), eim.data_ptr(), _ptr(stats), workspace.data_ptr(),
                                        workspace.numel(), _stream(stream)))
    return ere, eim, stats


AUTOTUNE_CANDIDATES = [(_lib.ANQS_BATCH_STATIC, 1)] + \
    [(_lib.ANQS_BATCH_DYNAMIC, c) for c in (8, 16, 32, 64, 128, 256, 512)]


class EnergyBatch:
    """Handle of anqs_batched_local_energy: one stream and one event per
    problem slot (max_problems of them) on the current CUDA device."""

    def __init__(self, max_problems: int):
        h = C.c_void_p()
        check(_lib.load().anqs_batch_create(C.byref(h), int(max_problems)))
        self._h, self.max_problems = h, int(max_problems)

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib._lib is not None:
            _lib._lib.anqs_batch_destroy(self._h)
            self._h = None

    def _problems(self, items):
        probs = (_lib.ElocProblem * max(len(items), 1))()
        keep, results = [], []
        for k, it in enumerate(items):
            model, ham, x = it["model"], it["ham"], _u64(it["x"])
            counts = it.get("counts")
            cnt = _u64(counts) if counts is not None else None
            n_x = x.numel()
            if it.get("out") is None:
                ere = torch.empty(n_x, dtype=torch.float64, device=x.device)
                eim = torch.empty_like(ere)
                stats = torch.empty(4, dtype=torch.float64, device=x.device) if cnt is not None else None
            else:
                ere, eim, stats = it["out"]
            ws = it.get("workspace")
            if ws is None:
                ws = _ws(local_energy_workspace_bytes(model, ham, n_x), x.device)
            probs[k] = _lib.ElocProblem(model._m, ham.handle, x.data_ptr(), _ptr(cnt), n_x, _ptr(it.get("n_dev")),
                                        ere.data_ptr(), eim.data_ptr(), _ptr(stats), ws.data_ptr(), ws.numel())
            keep += [x, cnt, ws]
            results.append((ere, eim, stats))
        return probs, keep, results

    def local_energy(self, items, stream=None):
        """Local energies of several independent problems in one call, side
        by side on the handle's streams, the 16-bit MLP problems' amplitude
        stage in one persistent launch, ordered on `stream` (capturable in a
        CUDA graph).  items: dicts with model, ham, x and optionally counts,
        n_dev, workspace, out=(eloc_re, eloc_im, stats).  Returns the
        (eloc_re, eloc_im, stats) of each problem."""
        probs, keep, results = self._problems(items)
        check(_lib.load().anqs_batched_local_energy(self._h, probs, len(items), _stream(stream)))
        self._keep = keep  # inputs and workspaces stay alive until the next call
        return results

    def set_schedule(self, mode: int, chunk: int = 8):
        """Schedule of the persistent launch: _lib.ANQS_BATCH_STATIC or
        ANQS_BATCH_DYNAMIC with `chunk` tiles per work item, or
        ANQS_BATCH_STREAMS (every problem whole on its own stream)."""
        check(_lib.load().anqs_batch_set_schedule(self._h, int(mode), int(chunk)))

    @property
    def schedule(self):
        mode, chunk = C.c_int(), C.c_int()
        check(_lib.load().anqs_batch_get_schedule(self._h, C.byref(mode), C.byref(chunk)))
        return mode.value, chunk.value

    def autotune(self, items, stream=None):
        """Time every candidate schedule of the persistent launch on these
        problems (outside any capture) and keep the fastest.  Returns the 8
        times in ms of AUTOTUNE_CANDIDATES: STATIC, then DYNAMIC with chunk
        8 .. 512."""
        probs, keep, _ = self._problems(items)
        times = (C.c_float * 8)()
        check(_lib.load().anqs_batch_autotune(self._h, probs, len(items), _stream(stream), times))
        self._keep = keep
        return list(times)


def grad_workspace_bytes(model, ham, n_x, least: bool = False) -> int:
    """Workspace of anqs_grad; with least=True the smallest it accepts (the
    transformer's adjoint then recomputes each block's activations)."""
    b = C.c_size_t()
    fn = _lib.load().anqs_grad_workspace_size_min if least else _lib.load().anqs_grad_workspace_size
    check(fn(model._m, ham.handle, n_x, C.byref(b)))
    return b.value


def grad(model: Model, ham: Hamiltonian, x, counts, eloc_re, eloc_im, stats, workspace=None, stream=None,
         n_dev=None, out=None):
    """VMC gradient (float32, flat parameter layout)."""
    x, counts = _u64(x), _u64(counts)
    g = out if out is not None else torch.empty(model.n_params, dtype=torch.float32, device=x.device)
    if workspace is None:
        b = C.c_size_t()
        check(_lib.load().anqs_grad_workspace_size(model._m, ham.handle, x.numel(), C.byref(b)))
        workspace = _ws(b.value, x.device)
    check(_lib.load().anqs_grad(model._m, ham.handle, x.data_ptr(), counts.data_ptr(), x.numel(), _ptr(n_dev),
                                eloc_re.data_ptr(), eloc_im.data_ptr(), stats.data_ptr(), g.data_ptr(),
                                workspace.data_ptr(), workspace.numel(), _stream(stream)))
    return g
