"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the method: it only draws random numbers
(molecular-shaped integrals, network weights) and packs them into the flat
parameter layout declared in ``include/anqs.h``.  Both the CUDA path and the
CPU oracle read their inputs from here; nothing here evaluates a Hamiltonian,
a wave function or a sampler.

Workloads (the paper's molecules, Table I, are replaced by integrals of the
same size; the molecular integrals themselves are not available):

* ``small``   4 spatial orbitals, 2+2 electrons, 8 Cholesky vectors, seed 0,
  MLP 2x64, N_s = 1e4 (sector 36).
* ``h2o``     7 spatial orbitals, 5+5 electrons (the H2O shape of Table I,
  14 qubits, 441 determinants), 14 Cholesky vectors, seed 1, MLP 3x128,
  N_s = 1e5.
* ``n2``      10 spatial orbitals, 7+7 electrons (the N2 shape of Table I,
  20 qubits, 14400 determinants), 20 Cholesky vectors, seed 2, causal
  transformer d=64, 4 heads, 2 layers, N_s = 1e6.
* ``batch32`` 32 problems, seeds 100..131, n in [6, 14], N_a = N_b in
  [1, n-1], 2n Cholesky vectors, MLP 3x128 each, N_s = 1e5 each.
* ``large``   26 spatial orbitals, 9+9 electrons, 52 Cholesky vectors,
  seed 3, transformer d=128, 8 heads, 4 layers, 4096 unique samples.
"""
from __future__ import annotations

import numpy as np

# Slot outcome v = x_alpha + 2 * x_beta, qubit q = 2 p + sigma (Appendix A:
# odd 1-based qubits carry spin up, i.e. interleaved alpha/beta ordering).
N_OUT = 8  # per slot: 4 modulus logits followed by 4 phases


def integrals(seed: int, n: int, n_chol: int, rng: np.random.Generator | None = None):
    """Molecular-shaped one- and two-body integrals (chemist notation).

    h: symmetric n x n, diagonal evenly spaced in [-2, 1] Ha ascending, upper
    triangle (p < q, row-major order) drawn N(0, 0.05^2) then mirrored.
    g[p,q,r,s] = sum_L B^L[p,q] B^L[r,s], each B^L symmetric with its upper
    triangle including the diagonal drawn N(0, 0.1^2) row-major.  g has the
    8-fold symmetry of real orbitals and is positive semidefinite as a
    (pq),(rs) matrix.  E_nuc = 0.
    """
    if rng is None:
        rng = np.random.default_rng(seed)
    h = np.zeros((n, n))
    h[np.diag_indices(n)] = np.linspace(-2.0, 1.0, n)
    iu = np.triu_indices(n, 1)
    h[iu] = rng.normal(0.0, 0.05, size=len(iu[0]))
    h[(iu[1], iu[0])] = h[iu]
    iu0 = np.triu_indices(n, 0)
    g = np.zeros((n, n, n, n))
    for _ in range(n_chol):
        B = np.zeros((n, n))
        B[iu0] = rng.normal(0.0, 0.1, size=len(iu0[0]))
        B[(iu0[1], iu0[0])] = B[iu0]
        g += np.einsum("pq,rs->pqrs", B, B)
    return h, g, 0.0


def integrals_z2(seed: int, n: int, n_chol: int, labels):
    """Integrals with planted abelian point-group symmetry: orbital p carries
    the irrep label labels[p] in [0, 2^k) (irrep product = XOR).  Drawn as
    `integrals`, then h_pq is kept only within one irrep and each Cholesky
    factor B^L, of irrep L mod 2^k, only where labels[p] ^ labels[q] equals
    it, so that g_pqrs vanishes unless the four labels XOR to zero.  Under the
    Jordan-Wigner transform every bit j of the labels gives a Z2 symmetry:
    the Pauli-Z string on both spin-qubits of the orbitals with bit j set
    (`z2_qubit_masks`)."""
    labels = np.asarray(labels, dtype=np.int64)
    k = max(1, int(labels.max()).bit_length())
    rng = np.random.default_rng(seed)
    h = np.zeros((n, n))
    h[np.diag_indices(n)] = np.linspace(-2.0, 1.0, n)
    iu = np.triu_indices(n, 1)
    h[iu] = rng.normal(0.0, 0.05, size=len(iu[0]))
    h[(iu[1], iu[0])] = h[iu]
    h[labels[:, None] != labels[None, :]] = 0.0
    iu0 = np.triu_indices(n, 0)
    g = np.zeros((n, n, n, n))
    for L in range(n_chol):
        B = np.zeros((n, n))
        B[iu0] = rng.normal(0.0, 0.1, size=len(iu0[0]))
        B[(iu0[1], iu0[0])] = B[iu0]
        B[(labels[:, None] ^ labels[None, :]) != (L % (1 << k))] = 0.0
        g += np.einsum("pq,rs->pqrs", B, B)
    return h, g, 0.0


def z2_qubit_masks(labels):
    """Qubit supports of the Z2 symmetries of `integrals_z2` (bit q = qubit
    q = 2p + sigma): one per bit of the irrep labels."""
    labels = [int(v) for v in labels]
    k = max(1, max(labels).bit_length())
    return [sum(3 << (2 * p) for p, v in enumerate(labels) if (v >> j) & 1) for j in range(k)]


# ----------------------------------------------------------------------------
# network parameters
# ----------------------------------------------------------------------------

def _bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def mlp_params(seed: int, n: int, width: int, n_hidden: int, bias_std: float = 0.0):
    """Per-slot MLP weights: slot p has its own network (Appendix B.1).

    Slot p (0-based) reads the one-hot encoding of the previous p slot values
    (4 p inputs, index 4 q + v_q).  Layer 1 maps 4p -> width (slot 0 has no
    input: its first layer is a bias only), layers 2..n_hidden map
    width -> width, the head maps width -> 8 (4 modulus logits, 4 phases).
    Weights ~ N(0, 1/fan_in), biases ~ N(0, bias_std^2).  Returned as a list
    over slots of lists of (W[out][in], b[out]) pairs, float64 holding
    float32-representable values.
    """
    rng = np.random.default_rng(1000 + seed)
    slots = []
    for p in range(n):
        layers = []
        fan_in = 4 * p
        for k in range(n_hidden + 1):
            out_dim = width if k < n_hidden else N_OUT
            in_dim = fan_in if k == 0 else width
            if in_dim > 0:
                W = rng.normal(0.0, 1.0 / np.sqrt(in_dim), size=(out_dim, in_dim))
            else:
                W = np.zeros((out_dim, 0))
            b = rng.normal(0.0, bias_std, size=out_dim) if bias_std > 0 else np.zeros(out_dim)
            layers.append((W.astype(np.float32).astype(np.float64),
                           b.astype(np.float32).astype(np.float64)))
        slots.append(layers)
    return slots


def flatten_mlp(slots) -> np.ndarray:
    """Pack per-slot MLP weights into the flat float32 layout of anqs.h.

    For each slot p in order, for each layer in order: W (row-major
    [out][in], absent when in == 0) then b ([out]).
    """
    parts = []
    for layers in slots:
        for W, b in layers:
            if W.size:
                parts.append(W.reshape(-1))
            parts.append(b.reshape(-1))
    return np.concatenate(parts).astype(np.float32)


def unflatten_mlp(flat: np.ndarray, n: int, width: int, n_hidden: int):
    """Inverse of flatten_mlp (float64 output), for reading gradients."""
    flat = np.asarray(flat, dtype=np.float64)
    off = 0
    slots = []
    for p in range(n):
        layers = []
        for k in range(n_hidden + 1):
            out_dim = width if k < n_hidden else N_OUT
            in_dim = 4 * p if k == 0 else width
            W = flat[off:off + out_dim * in_dim].reshape(out_dim, in_dim)
            off += out_dim * in_dim
            b = flat[off:off + out_dim]
            off += out_dim
            layers.append((W, b))
        slots.append(layers)
    assert off == flat.size, (off, flat.size)
    return slots


def mlp_param_count(n: int, width: int, n_hidden: int) -> int:
    tot = 0
    for p in range(n):
        tot += 4 * p * width + width
        tot += (n_hidden - 1) * (width * width + width)
        tot += N_OUT * width + N_OUT
    return tot


TF_KEYS = ("ln1_g", "ln1_b", "wq", "bq", "wk", "bk", "wv", "bv", "wo", "bo",
           "ln2_g", "ln2_b", "w1", "b1", "w2", "b2")


def tf_params(seed: int, n: int, d: int, n_layers: int, bias_std: float = 0.0):
    """Causal-transformer weights, rounded to bfloat16 values.

    Token table tok[5][d] (rows 0..3: slot values, row 4: start token),
    positions pos[n][d], per layer the pre-LayerNorm block weights of
    TF_KEYS (matrices [out][in], FFN hidden 4d), final LayerNorm and the
    head [8][d].  Matrices ~ N(0, 1/fan_in), embeddings ~ N(0, 1), LayerNorm
    gains 1 and shifts 0, biases ~ N(0, bias_std^2).
    """
    rng = np.random.default_rng(2000 + seed)
    r = _bf16_round
    P = {"tok": r(rng.normal(0, 1, (5, d))), "pos": r(rng.normal(0, 1, (n, d)))}
    layers = []

    def bias(k):
        return r(rng.normal(0, bias_std, k)) if bias_std > 0 else np.zeros(k)

    for _ in range(n_layers):
        L = {}
        L["ln1_g"] = np.ones(d) if bias_std == 0 else r(1 + rng.normal(0, bias_std, d))
        L["ln1_b"] = bias(d)
        for nm in ("q", "k", "v", "o"):
            L["w" + nm] = r(rng.normal(0, 1 / np.sqrt(d), (d, d)))
            L["b" + nm] = bias(d)
        L["ln2_g"] = np.ones(d) if bias_std == 0 else r(1 + rng.normal(0, bias_std, d))
        L["ln2_b"] = bias(d)
        L["w1"] = r(rng.normal(0, 1 / np.sqrt(d), (4 * d, d)))
        L["b1"] = bias(4 * d)
        L["w2"] = r(rng.normal(0, 1 / np.sqrt(4 * d), (d, 4 * d)))
        L["b2"] = bias(d)
        layers.append(L)
    P["layers"] = layers
    P["lnf_g"] = np.ones(d) if bias_std == 0 else r(1 + rng.normal(0, bias_std, d))
    P["lnf_b"] = bias(d)
    P["head_w"] = r(rng.normal(0, 1 / np.sqrt(d), (N_OUT, d)))
    P["head_b"] = bias(N_OUT)
    return P


def flatten_tf(P) -> np.ndarray:
    """Pack transformer weights into the flat float32 layout of anqs.h:
    tok, pos, per layer TF_KEYS in order, lnf_g, lnf_b, head_w, head_b."""
    parts = [P["tok"].reshape(-1), P["pos"].reshape(-1)]
    for L in P["layers"]:
        for k in TF_KEYS:
            parts.append(L[k].reshape(-1))
    parts += [P["lnf_g"], P["lnf_b"], P["head_w"].reshape(-1), P["head_b"]]
    return np.concatenate(parts).astype(np.float32)


def unflatten_tf(flat: np.ndarray, n: int, d: int, n_layers: int):
    flat = np.asarray(flat, dtype=np.float64)
    off = 0

    def take(shape):
        nonlocal off
        k = int(np.prod(shape))
        a = flat[off:off + k].reshape(shape)
        off += k
        return a

    P = {"tok": take((5, d)), "pos": take((n, d))}
    shapes = {"ln1_g": (d,), "ln1_b": (d,), "wq": (d, d), "bq": (d,), "wk": (d, d), "bk": (d,),
              "wv": (d, d), "bv": (d,), "wo": (d, d), "bo": (d,), "ln2_g": (d,), "ln2_b": (d,),
              "w1": (4 * d, d), "b1": (4 * d,), "w2": (d, 4 * d), "b2": (d,)}
    P["layers"] = [{k: take(shapes[k]) for k in TF_KEYS} for _ in range(n_layers)]
    P["lnf_g"] = take((d,))
    P["lnf_b"] = take((d,))
    P["head_w"] = take((N_OUT, d))
    P["head_b"] = take((N_OUT,))
    assert off == flat.size
    return P


def tf_param_count(n: int, d: int, n_layers: int) -> int:
    per_layer = 4 * d + 4 * (d * d + d) + 2 * (4 * d * d) + 4 * d + d
    return 5 * d + n * d + n_layers * per_layer + 2 * d + N_OUT * d + N_OUT


def nade_params(seed: int, n: int, width: int = 64, bias_std: float = 0.0):
    """Per-qubit NADE weights (Appendix B.1): one complex MLP per qubit
    i = 0..2n-1 (0-based) reading the i previous bits, two hidden layers of
    `width`, 2 complex outputs.  Per qubit: (W1 [w][i], b1 [w], W2 [w][w],
    b2 [w], W3 [2][w], b3 [2]) as complex128 arrays holding float32-
    representable parts; real and imaginary parts of a matrix with fan-in f
    ~ N(0, 1/(2 f)) each, biases ~ N(0, bias_std^2) each part."""
    rng = np.random.default_rng(3000 + seed)

    def cplx(shape, std):
        if std == 0.0 or 0 in shape:
            return np.zeros(shape, dtype=np.complex128)
        re = rng.normal(0.0, std, shape).astype(np.float32).astype(np.float64)
        im = rng.normal(0.0, std, shape).astype(np.float32).astype(np.float64)
        return re + 1j * im

    qubits = []
    for i in range(2 * n):
        W1 = cplx((width, i), 1.0 / np.sqrt(2 * max(i, 1)))
        b1 = cplx((width,), bias_std)
        W2 = cplx((width, width), 1.0 / np.sqrt(2 * width))
        b2 = cplx((width,), bias_std)
        W3 = cplx((2, width), 1.0 / np.sqrt(2 * width))
        b3 = cplx((2,), bias_std)
        qubits.append((W1, b1, W2, b2, W3, b3))
    return qubits


def flatten_nade(qubits) -> np.ndarray:
    """Flat float32 layout of anqs.h: per qubit W1, b1, W2, b2, W3, b3, each
    row-major with (re, im) interleaved."""
    parts = []
    for arrs in qubits:
        for a in arrs:
            parts.append(np.stack([a.real, a.imag], axis=-1).reshape(-1))
    return np.concatenate(parts).astype(np.float32)


def nade_param_count(n: int, width: int) -> int:
    return sum(2 * (width * i + width + width * width + width + 2 * width + 2) for i in range(2 * n))


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

WORKLOADS = {
    "small": dict(n=4, n_alpha=2, n_beta=2, seed=0, n_chol=8, kind="mlp", width=64,
                  n_hidden=2, n_samples=10_000),
    "h2o": dict(n=7, n_alpha=5, n_beta=5, seed=1, n_chol=14, kind="mlp", width=128,
                n_hidden=3, n_samples=100_000),
    "n2": dict(n=10, n_alpha=7, n_beta=7, seed=2, n_chol=20, kind="tf", d_model=64,
               n_heads=4, n_layers=2, n_samples=1_000_000),
    "h2o_nade": dict(n=7, n_alpha=5, n_beta=5, seed=1, n_chol=14, kind="nade", width=64,
                     n_samples=100_000),
    "large": dict(n=26, n_alpha=9, n_beta=9, seed=3, n_chol=52, kind="tf", d_model=128,
                  n_heads=8, n_layers=4, n_unique=4096),
}


def batch32_problem(k: int):
    """Problem k (0..31) of the 32-Hamiltonian batch: seed 100 + k draws the
    orbital count n in [6, 14] and N_a = N_b in [1, n - 1] first, then the
    integrals with 2n Cholesky vectors from the same generator."""
    seed = 100 + k
    rng = np.random.default_rng(seed)
    n = int(rng.integers(6, 15))
    na = int(rng.integers(1, n))
    h, g, e = integrals(seed, n, 2 * n, rng=rng)
    return dict(n=n, n_alpha=na, n_beta=na, seed=seed, n_chol=2 * n, kind="mlp", width=128,
                n_hidden=3, n_samples=100_000, h=h, g=g, e_nuc=e)


def workload(name: str, bias_std: float = 0.0):
    """Integrals and flat parameters of a named workload."""
    w = dict(WORKLOADS[name])
    h, g, e = integrals(w["seed"], w["n"], w["n_chol"])
    w.update(h=h, g=g, e_nuc=e)
    if w["kind"] == "mlp":
        w["params_struct"] = mlp_params(w["seed"], w["n"], w["width"], w["n_hidden"], bias_std)
        w["params"] = flatten_mlp(w["params_struct"])
    elif w["kind"] == "nade":
        w["params_struct"] = nade_params(w["seed"], w["n"], w["width"], bias_std)
        w["params"] = flatten_nade(w["params_struct"])
    else:
        w["params_struct"] = tf_params(w["seed"], w["n"], w["d_model"], w["n_layers"], bias_std)
        w["params"] = flatten_tf(w["params_struct"])
    return w
