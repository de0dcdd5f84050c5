"""Autoregressive statistics sampling with MU masking (Sec. II.C, Sec. III.C).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The tree is walked level by level (slot p = 0..n-1).  A node holds a prefix
(slots < p) and the number of samples n_in that entered it; the root holds
all N_s.  At each node the n_in samples are split among the four outcomes of
slot p according to the masked conditional p~(v | v_<p), so that MU passes
every sample to an allowed child and none is lost (Sec. III.C, Fig. 1C.iii);
children with zero samples are dropped (Sec. II.C).  The leaves are the
unique samples x^(l) with their occurrence numbers n^(l).

Split rule (the paper fixes the distribution, a multinomial split, but not
the procedure; reading): the node draws n_in uniforms u_i, i = 0..n_in-1,
from Philox4x64-10 with counter (prefix, i >> 2, p, counter) and key
(seed, 0), taking word i & 3 of each block; a uniform is the top 53 bits of
the word times 2^-53.  Sample i goes to the first allowed outcome v with
u_i < C_v, C_v the running sum of p~ over allowed outcomes in ascending v
(the last allowed outcome if rounding leaves u_i >= C_last).  p~ is the
softmax over allowed outcomes of the float32 logits, and it is evaluated in
float32 by a fixed sequence of IEEE operations (reading: the precision in
which the split decision is taken): e_v = exp(l_v - max) by Cody-Waite
reduction with ln2 split in two parts and the degree-7 Taylor polynomial of
e^r, s = sum of e_v in ascending v, p~_v = e_v / s, C_v = running sum.  The
outcome is an integer decided by floating point, so both implementations
take it in the same precision; the conditional's own error (about 1e-7
relative) is far below sampling noise.
Children are emitted in ascending v, so the leaves come out in lexicographic
order of (v_0, v_1, ..., v_{n-1}).

Pins: sum of counts = N_s under MU, all leaves in the sector, and a
chi-square test of the counts against N_s |psi(x)|^2 (tests/test_oracle_sampler.py).
"""
from __future__ import annotations

import numpy as np

from .anqs import allowed_masks
from .philox import philox4x64_np, uniform_from_word


F32 = np.float32
INV_LN2 = F32(1.44269502162933349609375)
LN2_HI = F32(0.693145751953125)       # 16 significant bits: k * LN2_HI is exact
LN2_LO = F32(1.428606765330187045e-06)
TAYLOR = [F32(1.0), F32(1.0), F32(0.5), F32(1.0) / F32(6.0), F32(1.0) / F32(24.0), F32(1.0) / F32(120.0),
          F32(1.0) / F32(720.0), F32(1.0) / F32(5040.0)]


def exp_det(x) -> np.float32:
    """e^x for float32 x <= 0: k = floor(x / ln2 + 1/2), r = x - k ln2 (two
    parts), Horner on the degree-7 Taylor polynomial, times 2^k; every step a
    single rounded float32 operation."""
    x = F32(x)
    if x < F32(-80.0):
        return F32(0.0)
    k = np.floor(F32(F32(x * INV_LN2) + F32(0.5)))
    r = F32(F32(x - F32(k * LN2_HI)) - F32(k * LN2_LO))
    q = TAYLOR[7]
    for c in TAYLOR[6::-1]:
        q = F32(F32(q * r) + c)
    return F32(np.ldexp(q, int(k)))


def split_probabilities(logits, mask) -> np.ndarray:
    """p~ of one node from its 4 modulus logits (rounded to float32) and
    allowed mask, in float32 (zero for masked outcomes)."""
    l = np.asarray(logits, dtype=np.float64).astype(np.float32)
    m = max(l[v] for v in range(4) if mask[v])
    e = [exp_det(F32(l[v] - m)) if mask[v] else F32(0.0) for v in range(4)]
    s = F32(0.0)
    for v in range(4):
        if mask[v]:
            s = F32(s + e[v])
    return np.array([F32(e[v] / s) if mask[v] else F32(0.0) for v in range(4)], dtype=np.float32)


def node_uniforms(prefix: int, count: int, p: int, seed: int, counter: int) -> np.ndarray:
    i = np.arange(count, dtype=np.uint64)
    blk = i >> np.uint64(2)
    words = philox4x64_np(np.full_like(blk, np.uint64(prefix)), blk, np.full_like(blk, np.uint64(p)),
                          np.full_like(blk, np.uint64(counter)), seed, 0)
    w = np.stack(words, axis=1)[np.arange(count), (i & np.uint64(3)).astype(np.int64)]
    return uniform_from_word(w)


def split_node(probs: np.ndarray, mask, u: np.ndarray, tol: float = 0.0):
    """Counts per outcome, the smallest |u - C_v| over the draws and the
    number of draws closer than tol to a boundary C_v."""
    C = np.zeros(4)
    run = F32(0.0)
    allowed = [v for v in range(4) if mask[v]]
    for v in range(4):
        if mask[v]:
            run = F32(run + probs[v])
        C[v] = float(run)
    out = np.full(len(u), allowed[-1], dtype=np.int64)
    undecided = np.ones(len(u), dtype=bool)
    for v in allowed:
        hit = undecided & (u < C[v])
        out[hit] = v
        undecided &= ~hit
    counts = np.bincount(out, minlength=4)
    margin = np.inf
    close = np.zeros(len(u), dtype=bool)
    if len(u):
        for v in allowed[:-1]:
            d = np.abs(u - C[v])
            margin = min(margin, float(np.min(d)))
            close |= d < tol
    return counts, margin, int(close.sum())


def sample(model, isphys, n: int, n_samples: int, seed: int, counter: int = 0,
           logits_fn=None, tol: float | None = None, shard=None, du_levels: int = 0):
    """Unique samples and counts, in the tree's lexicographic order.

    ``du_levels = d`` selects the MU-d strategy (Sec. III.C): on the last d
    slots the split uses the conditional over all four outcomes and the
    samples drawn into an unphysical child are discarded (d = 0: MU).

    ``shard = (rank, world, level)`` keeps, of the frontier reached after
    ``level`` slots (the leaves when level = n), the nodes i with
    i % world == rank, and walks on from those only: the subtrees below a
    node are independent (Sec. II.C), so the union over the ranks is the
    unsharded result.

    ``logits_fn(prefixes, p)`` may replace the network (returns [B, 4]
    modulus logits); by default the model's slot outputs are used.
    Returns (x uint64[N_unq], counts int64[N_unq], min_margin), plus the
    number of draws within tol of a boundary when tol is given (draws that
    a sampler with conditionals perturbed by less than tol may assign
    differently).
    """
    pre = np.zeros(1, dtype=np.uint64)
    cnt = np.array([n_samples], dtype=np.int64)
    margin = np.inf
    n_close = 0
    def keep(pre, cnt, p):
        if shard is None or shard[1] <= 1 or shard[2] != p:
            return pre, cnt
        sel = np.arange(len(pre)) % shard[1] == shard[0]
        return pre[sel], cnt[sel]

    for p in range(n):
        pre, cnt = keep(pre, cnt, p)
        if logits_fn is None:
            L = model.slot_out(pre, p)[:, :4].detach().numpy()
        else:
            L = np.asarray(logits_fn(pre, p), dtype=np.float64)
        M = allowed_masks(isphys, pre, n)[:, p]
        NM = M if p < n - du_levels else np.ones_like(M)
        new_pre, new_cnt = [], []
        for k in range(len(pre)):
            probs = split_probabilities(L[k], NM[k])
            u = node_uniforms(int(pre[k]), int(cnt[k]), p, seed, counter)
            c, mg, nc = split_node(probs, NM[k], u, tol or 0.0)
            c = np.where(M[k], c, 0)  # DU levels: samples of unphysical children are lost
            margin = min(margin, mg)
            n_close += nc
            for v in range(4):
                if c[v] > 0:
                    new_pre.append(int(pre[k]) | (v << (2 * p)))
                    new_cnt.append(int(c[v]))
        pre = np.array(new_pre, dtype=np.uint64)
        cnt = np.array(new_cnt, dtype=np.int64)
    pre, cnt = keep(pre, cnt, n)
    if tol is not None:
        return pre, cnt, margin, n_close
    return pre, cnt, margin


def lexicographic_key(xs, n: int) -> np.ndarray:
    """sum_p v_p 4^(n-1-p): ascending key = the tree's output order."""
    xs = np.asarray(xs, dtype=np.uint64)
    key = np.zeros(len(xs), dtype=np.uint64)
    for p in range(n):
        key = key * np.uint64(4) + ((xs >> np.uint64(2 * p)) & np.uint64(3))
    return key


def sample_binomial(model, isphys, n: int, n_samples: int, rng, logits_fn=None, du_levels: int = 0):
    """Binomial statistics sampling (Sec. II.C): at every node the n_in
    samples are split among the allowed outcomes by chained binomials,
    k_v ~ B(rest, p_v / (p_v + ... + p_last)) in ascending v, the last
    allowed outcome taking the rest (MU: nothing is lost).  p is the masked
    conditional in FP64; the binomial draws come from ``rng`` (a numpy
    Generator: a library primitive, so parity with the device sampler is in
    distribution only).  Returns (x uint64[N_unq], counts int64[N_unq]) in
    the tree's lexicographic order."""
    from .anqs import masked_log_prob
    import torch
    pre = np.zeros(1, dtype=np.uint64)
    cnt = np.array([n_samples], dtype=np.int64)
    for p in range(n):
        if logits_fn is None:
            L = model.slot_out(pre, p)[:, :4].detach()
        else:
            L = torch.as_tensor(np.asarray(logits_fn(pre, p), dtype=np.float64))
        M = allowed_masks(isphys, pre, n)[:, p]
        NM = M if p < n - du_levels else np.ones_like(M)
        P = torch.exp(masked_log_prob(L, torch.as_tensor(NM))).numpy()
        new_pre, new_cnt = [], []
        for k in range(len(pre)):
            allowed = [v for v in range(4) if NM[k][v]]
            rest, tail = int(cnt[k]), 1.0
            for v in allowed:
                if v == allowed[-1]:
                    c = rest
                else:
                    q = min(P[k][v] / tail, 1.0) if tail > 0 else 1.0
                    c = int(rng.binomial(rest, q))
                    tail -= P[k][v]
                rest -= c
                if c > 0 and M[k][v]:
                    new_pre.append(int(pre[k]) | (v << (2 * p)))
                    new_cnt.append(c)
        pre = np.array(new_pre, dtype=np.uint64)
        cnt = np.array(new_cnt, dtype=np.int64)
    return pre, cnt
