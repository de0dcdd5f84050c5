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
