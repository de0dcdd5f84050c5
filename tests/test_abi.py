"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/anqs.h declares; host-only entry points behave without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_04166_gb300 import _lib
    from paper_2310_04166_gb300 import build as b

    b.build()
    return _lib.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "anqs.h")).read()
    return sorted(set(re.findall(r"ANQS_API\s+[\w\s\*]*?\b(anqs_\w+)\s*\(", txt)))


def test_header_declares_the_hot_path():
    names = _declared()
    for must in ("anqs_sample", "anqs_connected", "anqs_logpsi", "anqs_local_energy", "anqs_grad"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_only_the_abi_is_exported():
    from paper_2310_04166_gb300 import _lib
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = sorted(l.split()[-1] for l in out.splitlines() if " T " in l)
    assert exported == _declared()


def test_param_counts_match_layouts(lib):
    from paper_2310_04166_gb300._lib import ModelDesc
    from synthetic import mlp_param_count, tf_param_count
    for n, w, L in [(4, 64, 2), (7, 128, 3), (14, 128, 3), (26, 256, 1)]:
        d = ModelDesc(0, 0, n, w, L, 0, 0, 0)
        k = C.c_uint64()
        assert lib.anqs_model_param_count(C.byref(d), C.byref(k)) == 0
        assert k.value == mlp_param_count(n, w, L)
    for n, dm, H, L in [(10, 64, 4, 2), (26, 128, 8, 4)]:
        d = ModelDesc(1, 1, n, 0, 0, dm, H, L)
        k = C.c_uint64()
        assert lib.anqs_model_param_count(C.byref(d), C.byref(k)) == 0
        assert k.value == tf_param_count(n, dm, L)
    from synthetic import nade_param_count
    for n, w in [(1, 32), (7, 64), (32, 128)]:
        d = ModelDesc(3, 0, n, w, 0, 0, 0, 0)
        k = C.c_uint64()
        assert lib.anqs_model_param_count(C.byref(d), C.byref(k)) == 0
        assert k.value == nade_param_count(n, w)
    for bad in (ModelDesc(3, 1, 4, 64, 0, 0, 0, 0), ModelDesc(3, 0, 4, 96, 0, 0, 0, 0)):  # BF16, width 96
        assert lib.anqs_model_param_count(C.byref(bad), C.byref(C.c_uint64())) == -5
    d = ModelDesc(2, 0, 5, 0, 0, 0, 0, 0)
    k = C.c_uint64()
    assert lib.anqs_model_param_count(C.byref(d), C.byref(k)) == 0
    assert k.value == 8 * sum(4 ** p for p in range(5))


def test_invalid_descriptions_rejected_on_host(lib):
    from paper_2310_04166_gb300._lib import ModelDesc
    k = C.c_uint64()
    for d in [ModelDesc(0, 0, 33, 128, 3, 0, 0, 0), ModelDesc(0, 0, 4, 96, 3, 0, 0, 0),
              ModelDesc(1, 0, 4, 0, 0, 64, 3, 2), ModelDesc(2, 1, 4, 0, 0, 0, 0, 0), ModelDesc(7, 0, 4, 0, 0, 0, 0, 0)]:
        assert lib.anqs_model_param_count(C.byref(d), C.byref(k)) < 0
    buf = C.create_string_buffer(256)
    assert lib.anqs_last_error(buf, 256) < 0 and len(buf.value) > 0


def test_null_arguments_rejected(lib):
    assert lib.anqs_hamiltonian_create(None, 4, 2, 2, None, None, 0.0) == -1
    assert lib.anqs_connected(None, None, 0, None, None, None, None, None) == -1


def test_shard_and_combine_arguments_rejected_on_host(lib):
    assert lib.anqs_stats_combine(None, 1, None, None) == -1
    buf = C.create_string_buffer(8 * 8)
    assert lib.anqs_stats_combine(buf, 0, buf, None) == -1
    assert lib.anqs_sample_shard(None, None, 10, 0, 0, None, 0, 2, 1, None, None, 0, None, None, 0, None) == -1


def test_batch_arguments_rejected_on_host(lib):
    """The batched local energy's argument checks come before any CUDA call."""
    h = C.c_void_p()
    assert lib.anqs_batch_create(None, 4) == -1
    assert lib.anqs_batch_create(C.byref(h), 0) == -1 and not h.value
    assert lib.anqs_batch_create(C.byref(h), 5000) == -1 and not h.value
    assert lib.anqs_batch_destroy(None) == 0
    assert lib.anqs_batched_local_energy(None, None, 0, None) == -1


def test_sampler_barrier_test_hook_is_host_only(lib):
    """The failure-detection hook only sets host-side launch parameters: it
    needs no GPU, always succeeds, and (0, 0) restores the defaults."""
    assert lib.anqs_test_sampler_barrier(1, 20_000_000) == 0
    assert lib.anqs_test_sampler_barrier(0, 0) == 0
