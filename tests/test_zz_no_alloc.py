"""The allocation-free local energy (anqs_local_energy_static) against the
workspace form (anqs_local_energy), called through the C ABI.

anqs_local_energy_static serves callers that cannot allocate device memory
while they run (its scratch is a fixed array inside the library).  This file
is collected last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_04166_gb300 as mod
    from paper_2310_04166_gb300 import _lib
    _lib.load()
    return mod


def _static_call(A, model, ham, x, n, ere, eim, stats):
    from paper_2310_04166_gb300 import _lib
    lib = _lib.load()
    return lib.anqs_local_energy_static(model._m, ham.handle, x.data_ptr(), n.data_ptr() if n is not None else None,
                                        x.numel(), ere.data_ptr(), eim.data_ptr(),
                                        stats.data_ptr() if stats is not None else None,
                                        torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("name,Ns", [("small", 10_000), ("h2o", 100_000)])
def test_static_scratch_matches_workspace_form(A, name, Ns):
    from paper_2310_04166_gb300 import _lib
    from synthetic import workload
    w = workload(name, bias_std=0.2)
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], torch.tensor(w["params"], device="cuda"), "fp32")
    x, n = A.sample(model, ham, Ns, seed=21)
    ref_re, ref_im, ref_st = A.local_energy(model, ham, x, n)
    for call in range(2):  # two calls in a row share (and reuse) the static scratch
        ere = torch.full_like(ref_re, float("nan"))
        eim = torch.full_like(ref_im, float("nan"))
        st = torch.full_like(ref_st, float("nan"))
        _lib.check(_static_call(A, model, ham, x, n, ere, eim, st))
        torch.cuda.synchronize()
        assert torch.allclose(ere, ref_re, rtol=0, atol=1e-10), call
        assert torch.allclose(eim, ref_im, rtol=0, atol=1e-10), call
        assert torch.allclose(st, ref_st, rtol=1e-12, atol=1e-12), call


def _other_models(A, kind):
    """(model, Hamiltonian, samples, counts or None) for the other FP32 kinds
    and edge sizes the entry point serves."""
    import numpy as np
    from synthetic import (flatten_mlp, flatten_nade, flatten_tf, integrals, mlp_params, nade_params, tf_params,
                           workload)
    if kind == "table":  # 4 orbitals, random slot logits, no counts (no statistics)
        h, g, e = integrals(3, 4, 4)
        ham = A.Hamiltonian(h, g, e, 2, 2)
        rows = sum(4 ** p for p in range(4))
        logits = np.random.default_rng(3).normal(0, 1, (rows, 8)).astype(np.float32)
        model = A.Model.table(4, torch.tensor(logits.ravel(), device="cuda"))
        x, _ = A.sample(model, ham, 5000, seed=4)
        return model, ham, x, None
    if kind == "one_orbital":  # 1 spatial orbital, 1 + 0 electrons: no connected determinant
        h, g, e = integrals(5, 1, 1)
        ham = A.Hamiltonian(h, g, e, 1, 0)
        model = A.Model.mlp(1, 64, 2, torch.tensor(flatten_mlp(mlp_params(5, 1, 64, 2, 0.2)), device="cuda"))
        x, n = A.sample(model, ham, 100, seed=6)
        return model, ham, x, n
    if kind == "transformer":
        w = workload("small", bias_std=0.2)
        ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
        P = tf_params(7, w["n"], 64, 2, bias_std=0.2)
        model = A.Model.transformer(w["n"], 64, 4, 2, torch.tensor(flatten_tf(P), device="cuda"))
        x, n = A.sample(model, ham, 10_000, seed=8)
        return model, ham, x, n
    w = workload("small", bias_std=0.2)  # per-qubit NADE
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    model = A.Model.nade(w["n"], 32, torch.tensor(flatten_nade(nade_params(9, w["n"], 32, 0.2)), device="cuda"))
    x, n = A.sample(model, ham, 10_000, seed=10)
    return model, ham, x, n


@pytest.mark.parametrize("kind", ["table", "one_orbital", "transformer", "nade"])
def test_static_scratch_other_models_and_edges(A, kind):
    from paper_2310_04166_gb300 import _lib
    model, ham, x, n = _other_models(A, kind)
    ref_re, ref_im, ref_st = A.local_energy(model, ham, x, n)
    for call in range(2):
        ere = torch.full_like(ref_re, float("nan"))
        eim = torch.full_like(ref_im, float("nan"))
        st = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda") if n is not None else None
        _lib.check(_static_call(A, model, ham, x, n, ere, eim, st))
        torch.cuda.synchronize()
        if kind == "nade":
            # the workspace form reuses the parent's slot terms for the NADE,
            # the static form evaluates every connected determinant in full:
            # equal up to the float32 rounding of the log-amplitude sums
            assert torch.allclose(ere, ref_re, rtol=1e-5, atol=1e-6), (kind, call)
            assert torch.allclose(eim, ref_im, rtol=1e-5, atol=1e-6), (kind, call)
        else:  # the same kernels on the same inputs
            assert torch.equal(ere, ref_re) and torch.equal(eim, ref_im), (kind, call)
        if n is not None:
            tol = 1e-5 if kind == "nade" else 1e-9
            assert torch.allclose(st, ref_st, rtol=tol, atol=tol), (kind, call)


def test_static_scratch_rejects_oversized_requests(A):
    from paper_2310_04166_gb300 import _lib
    from synthetic import workload
    w = workload("h2o")
    ham = A.Hamiltonian(w["h"], w["g"], w["e_nuc"], w["n_alpha"], w["n_beta"])
    model = A.Model.mlp(w["n"], w["width"], w["n_hidden"], torch.tensor(w["params"], device="cuda"), "fp32")
    n_x = 8000  # 8000 * 140 connected * 24 bytes > 16 MiB
    x = torch.zeros(n_x, dtype=torch.int64, device="cuda")
    out = torch.empty(n_x, dtype=torch.float64, device="cuda")
    rc = _static_call(A, model, ham, x, None, out, out.clone(), None)
    assert rc == -2  # ANQS_ERR_CAPACITY, reported on the host before any work
    buf = C.create_string_buffer(256)
    _lib.load().anqs_last_error(buf, 256)
    assert b"static scratch" in buf.value
