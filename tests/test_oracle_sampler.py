"""Pins for the oracle's statistics sampler (MU)."""
import numpy as np
import pytest
from scipy.stats import chi2

from oracle.anqs import MLPAnsatz, TFAnsatz, log_psi
from oracle.sampler import lexicographic_key, sample
from oracle.sector import molecular_isphys, sector_states
from synthetic import mlp_params, tf_params


@pytest.mark.parametrize("kind", ["mlp", "tf"])
def test_counts_match_born_distribution(kind):
    n, na, nb = 4, 2, 2
    if kind == "mlp":
        model = MLPAnsatz(mlp_params(3, n, 32, 2, bias_std=0.7), n)
    else:
        model = TFAnsatz(tf_params(3, n, 8, 1, bias_std=0.3), n, 2)
    ip = molecular_isphys(n, na, nb)
    st = np.array(sector_states(n, na, nb), dtype=np.uint64)
    la, _ = log_psi(model, ip, st)
    prob = np.exp(2 * la.numpy())
    Ns = 200_000
    xs, cnt, _ = sample(model, ip, n, Ns, seed=11, counter=2)
    assert cnt.sum() == Ns  # MU: no sample is lost (Sec. III.C)
    assert set(xs.tolist()) <= set(st.tolist())
    full = np.zeros(len(st))
    full[np.searchsorted(st, xs)] = cnt
    stat = ((full - Ns * prob) ** 2 / (Ns * prob)).sum()
    assert stat < chi2.ppf(1 - 1e-6, len(st) - 1)


def test_order_unique_and_deterministic():
    n = 5
    model = MLPAnsatz(mlp_params(2, n, 16, 2, bias_std=0.5), n)
    ip = molecular_isphys(n, 3, 2)
    a = sample(model, ip, n, 5000, seed=1)
    b = sample(model, ip, n, 5000, seed=1)
    c = sample(model, ip, n, 5000, seed=1, counter=1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not (np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]))
    key = lexicographic_key(a[0], n)
    assert np.all(np.diff(key.astype(np.float64)) > 0)


def test_single_sample_and_forced_path():
    """N_s = 1 yields one leaf with count 1; a sector with a single
    determinant (all orbitals filled) is always reached."""
    n = 3
    model = MLPAnsatz(mlp_params(0, n, 8, 2, bias_std=0.5), n)
    xs, cnt, _ = sample(model, molecular_isphys(n, 1, 2), n, 1, seed=5)
    assert len(xs) == 1 and cnt[0] == 1
    xs, cnt, _ = sample(model, molecular_isphys(n, 3, 3), n, 777, seed=5)
    assert xs.tolist() == [0b111111] and cnt.tolist() == [777]


def test_deterministic_exp_accuracy():
    """exp_det is within one float32 ulp (2^-23 relative) of e^x on [-80, 0]
    and exact at 0; the conditional it feeds sums to 1 to float32 rounding."""
    import math
    from oracle.sampler import exp_det, split_probabilities
    assert exp_det(0.0) == 1.0
    xs = np.concatenate([np.linspace(-80.0, 0.0, 4001), -np.logspace(-8, 1, 500)]).astype(np.float32)
    rel = max(abs(float(exp_det(x)) - math.exp(float(x))) / math.exp(float(x)) for x in xs)
    assert rel < 2.0 ** -23
    rng = np.random.default_rng(0)
    for _ in range(200):
        l = rng.normal(0, 3, 4)
        mask = rng.random(4) < 0.7
        if not mask.any():
            mask[rng.integers(4)] = True
        p = split_probabilities(l, mask)
        assert abs(float(p.sum()) - 1.0) < 4 * 2.0 ** -24 and np.all(p[~mask] == 0)
        ref = np.where(mask, np.exp(l - l[mask].max()), 0.0)
        assert np.abs(p - ref / ref.sum()).max() < 1e-6


# ---------------------------------------------------------------------------
# binomial statistics sampling (Sec. II.C)
# ---------------------------------------------------------------------------
def test_binomial_sampler_conserves_and_follows_born_distribution():
    from scipy.stats import chi2
    from oracle.anqs import MLPAnsatz, log_psi
    from oracle.sampler import sample_binomial
    from oracle.sector import molecular_isphys, sector_states
    from synthetic import workload
    w = workload("small", bias_std=0.3)
    om = MLPAnsatz(w["params_struct"], w["n"])
    ip = molecular_isphys(w["n"], w["n_alpha"], w["n_beta"])
    Ns = 10 ** 7
    x, c = sample_binomial(om, ip, w["n"], Ns, np.random.default_rng(3))
    assert c.sum() == Ns and np.all(c > 0)
    st = np.array(sector_states(w["n"], w["n_alpha"], w["n_beta"]), dtype=np.uint64)
    assert np.all(np.isin(x, st))
    la, _ = log_psi(om, ip, st)
    prob = np.exp(2 * la.numpy())
    full = np.zeros(len(st))
    full[np.searchsorted(st, x)] = c
    stat = ((full - Ns * prob) ** 2 / (Ns * prob)).sum()
    assert stat < chi2.ppf(1 - 1e-6, len(st) - 1)


def test_binomial_chain_has_multinomial_moments():
    """One free node (2 orbitals, 1 + 1 electrons: slot 0 takes any of the 4
    values, slot 1 is forced): the chained binomials reproduce the mean
    N p_v and the variance N p_v (1 - p_v) of the multinomial split."""
    from oracle.sampler import sample_binomial
    from oracle.sector import molecular_isphys
    p = np.array([0.5, 0.3, 0.15, 0.05])
    ip = molecular_isphys(2, 1, 1)
    logits = lambda pre, q: np.tile(np.log(p), (len(pre), 1))
    rng = np.random.default_rng(7)
    N, R = 1000, 4000
    counts = np.zeros((R, 4))
    for r in range(R):
        x, c = sample_binomial(None, ip, 2, N, rng, logits_fn=logits)
        counts[r, (x & np.uint64(3)).astype(int)] = c
    assert np.all(counts.sum(1) == N)
    mean, var = counts.mean(0), counts.var(0, ddof=1)
    assert np.all(np.abs(mean - N * p) < 5 * np.sqrt(N * p * (1 - p) / R))
    assert np.all(np.abs(var / (N * p * (1 - p)) - 1) < 5 * np.sqrt(2 / R))
