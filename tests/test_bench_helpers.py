"""Host-side helpers of bench.py (no GPU)."""
import bench


def test_guarded_returns_the_value_or_the_error():
    assert bench._guarded(lambda: {"value": 1.0}) == {"value": 1.0}

    def boom():
        raise RuntimeError("CUDA error: out of memory")

    r = bench._guarded(boom)
    assert r == {"error": "RuntimeError: CUDA error: out of memory"}


def test_compact_drops_the_enclosing_line_keys():
    sub = {"metric": "m", "unit": "u", "value": 2.0, "n_gpus": 1, "config": {"workload": "w"}}
    assert bench._compact(sub) == {"value": 2.0, "config": {"workload": "w"}}
