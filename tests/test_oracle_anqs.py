"""Pins for the oracle ansatz: normalisation over the sector, zero amplitude
outside it, the autoregressive property, and scalar-loop evaluations of tiny
networks (independent index-by-index restatements of the layer definitions)."""
import math

import numpy as np
import pytest

from oracle.anqs import MLPAnsatz, TableAnsatz, TFAnsatz, log_psi, table_from_state
from oracle.sector import molecular_isphys, sector_states
from synthetic import mlp_params, tf_params


def _brute_allowed(n, na, nb, x, p):
    """Outcome v of slot p allowed iff some sector state shares x's slots < p
    and has v in slot p."""
    sector = sector_states(n, na, nb)
    mask = (1 << (2 * p)) - 1
    return [any((s & mask) == (x & mask) and ((s >> (2 * p)) & 3) == v for s in sector) for v in range(4)]


def _mlp_scalar(slots, n, x):
    outs = []
    for p in range(n):
        u = [0.0] * (4 * p)
        for q in range(p):
            u[4 * q + ((x >> (2 * q)) & 3)] = 1.0
        hcur = u
        layers = slots[p]
        for k, (W, b) in enumerate(layers):
            z = []
            for o in range(W.shape[0]):
                acc = float(b[o])
                for i in range(W.shape[1]):
                    acc += float(W[o][i]) * hcur[i]
                z.append(math.tanh(acc) if k < len(layers) - 1 else acc)
            hcur = z
        outs.append(hcur)
    return outs


def _logpsi_scalar(outs, n, na, nb, x):
    la, ph = 0.0, 0.0
    for p in range(n):
        al = _brute_allowed(n, na, nb, x, p)
        v = (x >> (2 * p)) & 3
        lse = math.log(sum(math.exp(outs[p][u]) for u in range(4) if al[u]))
        la += 0.5 * (outs[p][v] - lse)
        ph += outs[p][4 + v]
    return la, ph


def test_mlp_matches_scalar_loops():
    n, na, nb = 3, 1, 2
    slots = mlp_params(5, n, 3, 2, bias_std=0.3)
    model = MLPAnsatz(slots, n)
    ip = molecular_isphys(n, na, nb)
    st = sector_states(n, na, nb)
    la, ph = log_psi(model, ip, st)
    for k, x in enumerate(st):
        a, b = _logpsi_scalar(_mlp_scalar(slots, n, x), n, na, nb, x)
        assert abs(a - la[k].item()) < 1e-13 and abs(b - ph[k].item()) < 1e-13


def _ln(x, g, b):
    mu = sum(x) / len(x)
    var = sum((t - mu) ** 2 for t in x) / len(x)
    return [(t - mu) / math.sqrt(var + 1e-5) * gg + bb for t, gg, bb in zip(x, g, b)]


def _lin(W, b, x):
    return [float(b[o]) + sum(float(W[o][i]) * x[i] for i in range(len(x))) for o in range(W.shape[0])]


def _tf_scalar(P, n, H, x):
    d = P["tok"].shape[1]
    dh = d // H
    toks = [4] + [(x >> (2 * q)) & 3 for q in range(n - 1)]
    hs = [[float(P["tok"][toks[t]][c] + P["pos"][t][c]) for c in range(d)] for t in range(n)]
    for L in P["layers"]:
        a = [_ln(hs[t], L["ln1_g"], L["ln1_b"]) for t in range(n)]
        q = [_lin(L["wq"], L["bq"], a[t]) for t in range(n)]
        k = [_lin(L["wk"], L["bk"], a[t]) for t in range(n)]
        v = [_lin(L["wv"], L["bv"], a[t]) for t in range(n)]
        new = []
        for t in range(n):
            o = [0.0] * d
            for hh in range(H):
                sl = range(hh * dh, (hh + 1) * dh)
                sc = [sum(q[t][c] * k[s][c] for c in sl) / math.sqrt(dh) for s in range(t + 1)]
                m = max(sc)
                e = [math.exp(z - m) for z in sc]
                Z = sum(e)
                for c in sl:
                    o[c] = sum(e[s] / Z * v[s][c] for s in range(t + 1))
            proj = _lin(L["wo"], L["bo"], o)
            new.append([hs[t][c] + proj[c] for c in range(d)])
        hs = new
        out = []
        for t in range(n):
            f = _ln(hs[t], L["ln2_g"], L["ln2_b"])
            m1 = [max(0.0, z) for z in _lin(L["w1"], L["b1"], f)]
            m2 = _lin(L["w2"], L["b2"], m1)
            out.append([hs[t][c] + m2[c] for c in range(d)])
        hs = out
    return [_lin(P["head_w"], P["head_b"], _ln(hs[t], P["lnf_g"], P["lnf_b"])) for t in range(n)]


def test_transformer_matches_scalar_loops():
    n, na, nb, H = 3, 2, 1, 2
    P = tf_params(4, n, 4, 2, bias_std=0.2)
    model = TFAnsatz(P, n, H)
    ip = molecular_isphys(n, na, nb)
    st = sector_states(n, na, nb)
    la, ph = log_psi(model, ip, st)
    for k, x in enumerate(st):
        a, b = _logpsi_scalar(_tf_scalar(P, n, H, x), n, na, nb, x)
        assert abs(a - la[k].item()) < 1e-12 and abs(b - ph[k].item()) < 1e-12


def _models(n):
    yield MLPAnsatz(mlp_params(1, n, 16, 2, bias_std=0.5), n)
    yield TFAnsatz(tf_params(1, n, 8, 2, bias_std=0.2), n, 2)


@pytest.mark.parametrize("n,na,nb", [(3, 1, 1), (4, 2, 2), (5, 3, 2)])
def test_normalised_on_sector_zero_outside(n, na, nb):
    ip = molecular_isphys(n, na, nb)
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    allx = np.arange(1 << (2 * n), dtype=np.uint64)
    outside = allx[~np.isin(allx, st)]
    for model in _models(n):
        la, _ = log_psi(model, ip, st)
        assert abs(np.exp(2 * la.numpy()).sum() - 1.0) < 1e-12
        lo, _ = log_psi(model, ip, outside)
        assert np.all(np.exp(2 * lo.numpy()) == 0.0)


def test_autoregressive_property():
    """Slot p's outputs do not depend on slots >= p."""
    n = 5
    rng = np.random.default_rng(0)
    xs = rng.integers(0, 1 << (2 * n), size=20).astype(np.uint64)
    for model in _models(n):
        for p in range(n):
            keep = np.uint64((1 << (2 * p)) - 1)
            scrambled = (xs & keep) | (rng.integers(0, 1 << (2 * n), size=20).astype(np.uint64) & ~keep)
            a = model.slot_out(xs, p).detach().numpy()
            b = model.slot_out(scrambled, p).detach().numpy()
            assert np.abs(a - b).max() < 1e-12


def test_table_reproduces_state():
    n, na, nb = 4, 2, 1
    ip = molecular_isphys(n, na, nb)
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    c = np.random.default_rng(2).normal(size=len(st))
    c /= np.linalg.norm(c)
    tab = TableAnsatz(table_from_state(st, c, n), n)
    la, ph = log_psi(tab, ip, st)
    psi = np.exp(la.numpy()) * np.cos(ph.numpy())
    assert np.abs(psi - c).max() < 1e-13
