"""Autoregressive neural quantum state with MU masking, in FP64 (torch CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

psi(x) = prod_p psi_p(v_p | v_<p)  (Eq. anqs_def), with the autoregressive
unit a spatial orbital (slot p, value v_p = x_{2p} + 2 x_{2p+1}).  Each slot
conditional comes from 8 network outputs: modulus logits l_v and phases
phi_v, v = 0..3.  Normalisation is the third activation of Appendix B.1,
f3(z) = z - 1/2 LSE(2 Re z), with z_v = l_v / 2 + i phi_v, so that
|psi_p(v)|^2 = softmax(l)_v.  The MU strategy (Sec. III.C) masks the outcomes
that IsPhys rules out: the softmax runs over the allowed outcomes only and a
masked outcome has amplitude exactly 0.  Reading: masking renormalises the
modulus and keeps the phases of the allowed outcomes (the paper's binary
example fixes the single allowed amplitude to 1; with ``forced_phase_zero`` a
slot with exactly one allowed outcome gets phase 0 instead).

Networks (the paper's own ansatz, the per-qubit complex NADE of Appendix
B.1, and readings):
* per-qubit NADE (NADEAnsatz): see its docstring.
* per-slot MLP: slot p reads the one-hot of v_<p (4p inputs), tanh hidden
  layers, 8 outputs; slot 0 has no input (first layer = bias).
* causal transformer: token t is the start token (t = 0) or v_{t-1}, plus a
  learned position; pre-LayerNorm blocks (eps 1e-5) with causal multi-head
  attention and a ReLU FFN of width 4d, final LayerNorm, head d -> 8.
* tabular: the 8 outputs of slot p are looked up by the prefix v_<p.

Pins: normalisation over the sector by brute force, zero amplitude outside
the sector, the autoregressive property, and scalar-loop evaluations of tiny
networks (tests/test_oracle_anqs.py).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .sector import IsPhys

DT = torch.float64


def slot_values(xs, n: int) -> np.ndarray:
    xs = np.asarray(xs, dtype=np.uint64)
    return np.stack([((xs >> np.uint64(2 * p)) & np.uint64(3)).astype(np.int64) for p in range(n)], axis=1)


def allowed_masks(isphys: IsPhys, xs, n: int) -> np.ndarray:
    """[B, n, 4] bool: outcome v of slot p allowed after the prefix v_<p of x.

    Uses Proposition 1: physicality depends only on the partial eigenvalues,
    so IsPhys is queried with s(x_<i) computed from the prefix bits."""
    xs = np.asarray(xs, dtype=np.uint64)
    syms = isphys.syms
    B = len(xs)
    out = np.zeros((B, n, 4), dtype=bool)
    bits = [((xs >> np.uint64(q)) & np.uint64(1)).astype(np.int64) for q in range(2 * n)]
    s = [np.full(B, sym.identity, dtype=np.int64) for sym in syms]

    def compose(sym, a, b):
        return a + b if sym.op == "add" else a * b

    cache: dict = {}
    for p in range(n):
        for v in range(4):
            s2 = []
            for k, sym in enumerate(syms):
                t = compose(sym, s[k], np.full(B, sym.local(2 * p + 1, v & 1)))
                t = compose(sym, t, np.full(B, sym.local(2 * p + 2, v >> 1)))
                s2.append(t)
            keys = np.stack(s2, axis=1)
            uniq, inv = np.unique(keys, axis=0, return_inverse=True)
            vals = []
            for u in uniq:
                key = (2 * p + 3, tuple(int(t) for t in u))
                if key not in cache:
                    cache[key] = isphys(2 * p + 3, key[1])
                vals.append(cache[key])
            out[:, p, v] = np.asarray(vals, dtype=bool)[inv.reshape(-1)]
        for k, sym in enumerate(syms):
            s[k] = compose(sym, s[k], np.array([sym.local(2 * p + 1, 0), sym.local(2 * p + 1, 1)])[bits[2 * p]])
            s[k] = compose(sym, s[k], np.array([sym.local(2 * p + 2, 0), sym.local(2 * p + 2, 1)])[bits[2 * p + 1]])
    return out


def masked_log_prob(logits: torch.Tensor, mask: torch.Tensor) -> torch.Tensor:
    """log p~(v) = l_v - LSE over allowed outcomes; -inf for masked ones."""
    neg = torch.full_like(logits, -math.inf)
    lm = torch.where(mask, logits, neg)
    lse = torch.logsumexp(lm, dim=-1, keepdim=True)
    # a prefix with no allowed outcome lies outside the sector: every outcome
    # gets log p~ = -inf (amplitude exactly zero) instead of -inf - (-inf)
    lse = torch.where(torch.isfinite(lse), lse, torch.zeros_like(lse))
    return lm - lse


def norm_masks(mask: np.ndarray, du_levels: int = 0) -> np.ndarray:
    """Outcomes over which each slot's conditional is normalised under the
    MU-d strategy (Sec. III.C): the physical ones on the first n - d slots
    (MU), all four on the last d (DU, where samples sent to an unphysical
    child are discarded).  d = 0 is MU, d = n is DU."""
    nm = np.array(mask, dtype=bool, copy=True)
    if du_levels > 0:
        nm[:, nm.shape[1] - du_levels:, :] = True
    return nm


def log_psi_from_logits(out: torch.Tensor, xs, mask: np.ndarray, forced_phase_zero: bool = False,
                        du_levels: int = 0):
    """out: [B, n, 8] network outputs per slot.  Returns (log|psi|, phase)
    as FP64 tensors: log|psi| = sum_p 1/2 log p~_p(v_p), phase = sum_p phi_p(v_p),
    with p~ normalised as norm_masks says and zero for unphysical v_p."""
    n = out.shape[1]
    v = torch.as_tensor(slot_values(xs, n))
    m = torch.as_tensor(mask)
    lp = masked_log_prob(out[..., :4], torch.as_tensor(norm_masks(mask, du_levels)))
    lp = torch.where(m, lp, torch.full_like(lp, -math.inf))
    lp_sel = torch.gather(lp, 2, v[..., None])[..., 0]
    ph_sel = torch.gather(out[..., 4:], 2, v[..., None])[..., 0]
    if forced_phase_zero:
        single = m.sum(-1) == 1
        ph_sel = torch.where(single, torch.zeros_like(ph_sel), ph_sel)
    return 0.5 * lp_sel.sum(1), ph_sel.sum(1)


class MLPAnsatz:
    """Per-slot MLP (one network per spatial orbital, Appendix B.1 layout)."""

    def __init__(self, slots, n: int):
        self.n = n
        self.slots = [[(torch.tensor(W, dtype=DT), torch.tensor(b, dtype=DT)) for W, b in layers]
                      for layers in slots]

    def parameters(self):
        return [t for layers in self.slots for W, b in layers for t in (W, b)]

    def slot_out(self, xs, p: int) -> torch.Tensor:
        """[B, 8] outputs of slot p's network for the prefixes of xs."""
        B = len(xs)
        v = slot_values(xs, self.n)[:, :p] if p > 0 else np.zeros((B, 0), dtype=np.int64)
        u = torch.zeros((B, 4 * p), dtype=DT)
        for q in range(p):
            u[torch.arange(B), 4 * q + torch.as_tensor(v[:, q])] = 1.0
        layers = self.slots[p]
        hcur = u
        for k, (W, b) in enumerate(layers):
            z = (hcur @ W.T if W.shape[1] > 0 else torch.zeros((B, W.shape[0]), dtype=DT)) + b
            hcur = torch.tanh(z) if k < len(layers) - 1 else z
        return hcur

    def outputs(self, xs) -> torch.Tensor:
        return torch.stack([self.slot_out(xs, p) for p in range(self.n)], dim=1)


def _layer_norm(x, g, b, eps=1e-5):
    mu = x.mean(-1, keepdim=True)
    var = ((x - mu) ** 2).mean(-1, keepdim=True)
    return (x - mu) / torch.sqrt(var + eps) * g + b


class TFAnsatz:
    """Causal transformer over the n slots (decoder-only, pre-LayerNorm)."""

    def __init__(self, P, n: int, n_heads: int):
        self.n = n
        self.H = n_heads
        t = lambda a: torch.tensor(np.asarray(a), dtype=DT)
        self.tok = t(P["tok"])
        self.pos = t(P["pos"])
        self.layers = [{k: t(v) for k, v in L.items()} for L in P["layers"]]
        self.lnf_g, self.lnf_b = t(P["lnf_g"]), t(P["lnf_b"])
        self.head_w, self.head_b = t(P["head_w"]), t(P["head_b"])
        self.d = self.tok.shape[1]

    def parameters(self):
        ps = [self.tok, self.pos]
        for L in self.layers:
            ps += list(L.values())
        return ps + [self.lnf_g, self.lnf_b, self.head_w, self.head_b]

    def outputs(self, xs, upto: int | None = None) -> torch.Tensor:
        """[B, T, 8] outputs for positions 0..T-1 (T = upto or n)."""
        n = self.n
        T = n if upto is None else upto
        B = len(xs)
        v = slot_values(xs, n)
        tokens = np.full((B, T), 4, dtype=np.int64)
        if T > 1:
            tokens[:, 1:] = v[:, :T - 1]
        hcur = self.tok[torch.as_tensor(tokens)] + self.pos[:T][None]
        d, H = self.d, self.H
        dh = d // H
        causal = torch.tril(torch.ones(T, T, dtype=torch.bool))
        for L in self.layers:
            a = _layer_norm(hcur, L["ln1_g"], L["ln1_b"])
            q = a @ L["wq"].T + L["bq"]
            k = a @ L["wk"].T + L["bk"]
            vv = a @ L["wv"].T + L["bv"]
            q = q.view(B, T, H, dh).transpose(1, 2)
            k = k.view(B, T, H, dh).transpose(1, 2)
            vv = vv.view(B, T, H, dh).transpose(1, 2)
            s = (q @ k.transpose(-1, -2)) / math.sqrt(dh)
            s = torch.where(causal, s, torch.full_like(s, -math.inf))
            att = torch.softmax(s, dim=-1)
            o = (att @ vv).transpose(1, 2).reshape(B, T, d)
            hcur = hcur + o @ L["wo"].T + L["bo"]
            f = _layer_norm(hcur, L["ln2_g"], L["ln2_b"])
            hcur = hcur + torch.relu(f @ L["w1"].T + L["b1"]) @ L["w2"].T + L["b2"]
        hcur = _layer_norm(hcur, self.lnf_g, self.lnf_b)
        return hcur @ self.head_w.T + self.head_b

    def slot_out(self, xs, p: int) -> torch.Tensor:
        return self.outputs(xs, upto=p + 1)[:, p]


def leaky_relu(x):
    """LeReLU of Appendix B.1, read as the usual leaky ReLU: x for x >= 0,
    0.01 x otherwise (the printed "-0.01 x" would make the function
    non-monotonic; reading)."""
    return torch.where(x >= 0, x, 0.01 * x)


class NADEAnsatz:
    """The paper's own ansatz (Appendix B.1): one complex MLP per qubit
    i = 1..N (here 0-based, i = 0..2n-1) reading the i previous bits, with
    f1 = tanh (complex), f2 = LeReLU(Re z) + i LeReLU(Im z), and f3(z) =
    z - 1/2 LSE(2 Re z) over its two outputs, so that
    log psi_i(x_i | x_<i) = f3(z)_{x_i}.

    The slot formulation used here groups qubits 2p (alpha) and 2p + 1
    (beta): the slot conditional of v = a + 2b is psi_{2p}(a) psi_{2p+1}(b | a).
    MU masking acts on each qubit's binary conditional (Sec. III.C): the
    allowed values of qubit 2p are those a with some allowed (a, b) in the
    slot, those of qubit 2p+1 the b with (a, b) allowed; the modulus is
    renormalised over them and the phases kept (reading 4).  On the DU slots
    of an MU-d strategy no value is masked.  slot_out returns the 8 slot
    values l_v = log |psi_slot(v)|^2 and phi_v = arg psi_slot(v) (-inf for
    masked v), which are already normalised, so the slot-level machinery
    (masked log-softmax, sampler) reproduces them.
    """

    def __init__(self, qubits, n: int, isphys: IsPhys, du_levels: int = 0):
        self.n, self.isphys, self.du_levels = n, isphys, du_levels
        self.q = [[(torch.tensor(a.real, dtype=DT), torch.tensor(a.imag, dtype=DT)) for a in arrs] for arrs in qubits]

    def parameters(self):
        return [t for arrs in self.q for pair in arrs for t in pair]

    def _qubit(self, i: int, bits: torch.Tensor) -> torch.Tensor:
        """log psi_i(0), log psi_i(1) (complex, unmasked) for bits [B, i]."""
        (W1r, W1i), (b1r, b1i), (W2r, W2i), (b2r, b2i), (W3r, W3i), (b3r, b3i) = self.q[i]
        W1, b1 = torch.complex(W1r, W1i), torch.complex(b1r, b1i)
        W2, b2 = torch.complex(W2r, W2i), torch.complex(b2r, b2i)
        W3, b3 = torch.complex(W3r, W3i), torch.complex(b3r, b3i)
        B = bits.shape[0]
        z = b1.expand(B, -1) + (bits.to(torch.complex128) @ W1.T if i > 0 else 0)
        h = torch.tanh(z)
        z = h @ W2.T + b2
        h = torch.complex(leaky_relu(z.real), leaky_relu(z.imag))
        z = h @ W3.T + b3
        return z - 0.5 * torch.logsumexp(2 * z.real, dim=-1, keepdim=True)

    @staticmethod
    def _mask(lq: torch.Tensor, allowed: torch.Tensor) -> torch.Tensor:
        """Renormalise the modulus over the allowed values, keep the phases."""
        neg = torch.full_like(lq.real, -math.inf)
        re = torch.where(allowed, lq.real, neg)
        lse = 0.5 * torch.logsumexp(2 * re, dim=-1, keepdim=True)
        lse = torch.where(torch.isfinite(lse), lse, torch.zeros_like(lse))
        return torch.complex(re - lse, lq.imag)

    def slot_out(self, xs, p: int) -> torch.Tensor:
        xs = np.asarray(xs, dtype=np.uint64)
        B = len(xs)
        bits = torch.tensor(np.stack([((xs >> np.uint64(q)) & np.uint64(1)).astype(np.float64)
                                      for q in range(2 * p)], axis=1) if p > 0 else np.zeros((B, 0)), dtype=DT)
        lq0 = self._qubit(2 * p, bits)
        lq1 = [self._qubit(2 * p + 1, torch.cat([bits, torch.full((B, 1), float(a), dtype=DT)], 1)) for a in (0, 1)]
        if p < self.n - self.du_levels:
            m = torch.as_tensor(allowed_masks(self.isphys, xs, self.n)[:, p])  # [B, 4], v = a + 2b
            lq0 = self._mask(lq0, torch.stack([m[:, 0] | m[:, 2], m[:, 1] | m[:, 3]], 1))
            lq1 = [self._mask(lq1[a], torch.stack([m[:, a], m[:, a + 2]], 1)) for a in (0, 1)]
        out = torch.zeros((B, 8), dtype=DT)
        for v in range(4):
            a, b = v & 1, v >> 1
            lv = lq0[:, a] + lq1[a][:, b]
            out[:, v] = 2 * lv.real
            out[:, 4 + v] = lv.imag
        return out

    def outputs(self, xs) -> torch.Tensor:
        return torch.stack([self.slot_out(xs, p) for p in range(self.n)], dim=1)


class TableAnsatz:
    """Slot outputs looked up by prefix: table[p] has shape [4^p, 8] and row
    r = sum_{q<p} v_q 4^q (the prefix bits of x read as an integer)."""

    def __init__(self, tables, n: int):
        self.n = n
        self.tables = [torch.tensor(np.asarray(t), dtype=DT) for t in tables]

    def slot_out(self, xs, p: int) -> torch.Tensor:
        xs = np.asarray(xs, dtype=np.uint64)
        r = (xs & np.uint64((1 << (2 * p)) - 1)).astype(np.int64)
        return self.tables[p][torch.as_tensor(r)]

    def outputs(self, xs) -> torch.Tensor:
        return torch.stack([self.slot_out(xs, p) for p in range(self.n)], dim=1)


def table_from_state(states, amps, n: int, floor: float = -1e30):
    """Tabular ansatz reproducing a real normalised sector state c (e.g. an
    exact eigenvector): l_v = log of the marginal weight of prefix v_<p v,
    phases zero except the last slot, which carries pi where c_x < 0."""
    states = np.asarray(states, dtype=np.uint64)
    w = np.asarray(amps, dtype=np.float64) ** 2
    tables = []
    for p in range(n):
        T = np.zeros((4 ** p, 8))
        marg = np.zeros((4 ** p, 4))
        pre = (states & np.uint64((1 << (2 * p)) - 1)).astype(np.int64)
        vp = ((states >> np.uint64(2 * p)) & np.uint64(3)).astype(np.int64)
        np.add.at(marg, (pre, vp), w)
        with np.errstate(divide="ignore"):
            T[:, :4] = np.where(marg > 0, np.log(np.where(marg > 0, marg, 1.0)), floor)
        if p == n - 1:
            sgn = np.zeros((4 ** p, 4))
            sgn[pre, vp] = np.where(np.asarray(amps) < 0, math.pi, 0.0)
            T[:, 4:] = sgn
        tables.append(T)
    return tables


def log_psi(model, isphys: IsPhys, xs, forced_phase_zero: bool = False, du_levels: int = 0):
    """(log|psi(x)|, arg psi(x)) in FP64 for a batch of determinants (MU-d
    strategy with d = du_levels; 0 = MU)."""
    xs = np.asarray(xs, dtype=np.uint64)
    mask = allowed_masks(isphys, xs, model.n)
    return log_psi_from_logits(model.outputs(xs), xs, mask, forced_phase_zero, du_levels)


def conditionals(model, isphys: IsPhys, prefixes, p: int):
    """Masked conditional probabilities p~(v | v_<p) of slot p, [B, 4] FP64
    (zero for masked outcomes), and the raw modulus logits [B, 4]."""
    prefixes = np.asarray(prefixes, dtype=np.uint64)
    out = model.slot_out(prefixes, p)
    mask = allowed_masks(isphys, prefixes, model.n)[:, p]
    lp = masked_log_prob(out[:, :4], torch.as_tensor(mask))
    return torch.exp(lp).detach().numpy(), out[:, :4].detach().numpy(), mask
