"""Host-side helpers of bench.py: the JSON line stays strict JSON when a run diverges, the
roofline's per-unit flop counts, the Morton order of the W.q leg, the FP32-pair split of the
mixed storage. No GPU."""
import importlib.util
import json
import math
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_helpers_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_json_line_is_strict_json():
    b = _bench()
    line = b.json_safe({"a": float("nan"), "b": [1.0, float("inf"), np.float64(2.5)], "c": {"d": np.int64(3)},
                        "e": (np.float32(-math.inf), "x")})
    text = json.dumps(line, allow_nan=False)
    assert json.loads(text) == {"a": None, "b": [1.0, None, 2.5], "c": {"d": 3}, "e": [None, "x"]}


def test_per_unit_flop_counts():
    b = _bench()
    m = 109
    assert math.isclose(b.weights_flops(m), 2 * m ** 3 / 3 + 2 * m * m)     # one solve, elimination's count
    assert round(b.weights_flops(m)) == 887115
    assert math.isclose(b.weights_kernel_flops(m), m ** 3 / 3 + 2 * m * m)  # what the L D L^T executes
    assert round(b.weights_kernel_flops(m)) == 455438


def test_morton_order_is_a_local_permutation():
    b = _bench()
    rng = np.random.default_rng(0)
    X = rng.standard_normal((5000, 3))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    p = b.morton_order(X)
    assert sorted(p.tolist()) == list(range(5000))
    # consecutive points along the curve are much closer than random pairs
    step = np.linalg.norm(np.diff(X[p], axis=0), axis=1).mean()
    rand = np.linalg.norm(X[rng.permutation(5000)] - X, axis=1).mean()
    assert step < 0.2 * rand


def test_pair_split_is_exact_to_fp32_pairs():
    b = _bench()
    a = np.random.default_rng(1).standard_normal(1000)
    p = b.pairs_of(a)
    assert p.shape == (1000, 2) and p.dtype == np.float32
    back = p[:, 0].astype(np.float64) + p[:, 1].astype(np.float64)
    assert np.all(np.abs(back - a) <= 2.0 ** -48 * np.abs(a))
