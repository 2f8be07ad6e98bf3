"""Batches of uneven problems in one CUDA-graph launch: bitwise equal to the
plain one-at-a-time evaluation, and equal to the oracle."""
import numpy as np
import pytest

import workloads as w
from tests._helpers import assert_close, oracle_eval

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


def _problems():
    probs = w.batch_problems(9, seed=311, sizes=(3, 4, 5), depths=(3, 5, 7))
    probs.append(w.make_problem(4, 5, 0.3, seed=312, structure=1, tied=True))
    probs.append(w.make_problem(3, 4, 0.7, seed=313, structure=1))
    return probs


def test_batched_equals_plain_and_oracle(rq):
    probs = _problems()
    b = rq.Batch(0)
    for p in probs:
        b.add_problem(p)
    dirs = [w.random_directions(p.n_params, 2, 400 + i) for i, p in enumerate(probs)]
    gates = [p.gates for p in probs]
    f1, g1, h1 = b.hvp(gates, dirs)            # autotunes, captures, launches the graph
    info = b.info()
    assert info["n_problems"] == len(probs) and info["columns_per_tile"] in (64, 128, 256, 512)
    f2, g2, h2 = b.hvp(gates, dirs)            # graph replay
    f3, g3, h3 = b.hvp(gates, dirs, plain=True)
    assert np.array_equal(f1, f2) and np.array_equal(f1, f3)
    for i in range(len(probs)):
        assert np.array_equal(g1[i], g3[i]) and np.array_equal(h1[i], h3[i])
        assert np.array_equal(g1[i], g2[i]) and np.array_equal(h1[i], h2[i])
    for i, p in enumerate(probs):
        if p.n > 8:
            continue
        f, g, hv, _ = oracle_eval(p, range(1 << p.n), dirs[i], chunk=64)
        assert abs(f1[i] - f) <= 1e-12 * abs(f)
        assert_close(g1[i], g, p.n, what=f"problem {i} grad")
        assert_close(h1[i], hv, p.n, what=f"problem {i} hvp")


def test_batch_fixed_tile_and_new_gates(rq):
    probs = _problems()[:4]
    b = rq.Batch(0)
    for p in probs:
        b.add_problem(p)
    b.set_tile(64)
    gates = [p.gates for p in probs]
    dirs = [w.random_directions(p.n_params, 1, 500 + i) for i, p in enumerate(probs)]
    f1, g1, h1 = b.hvp(gates, dirs)
    gates2 = [g * np.exp(0.2j) for g in gates]   # new inputs replay the same graph
    f2, g2, h2 = b.hvp(gates2, dirs)
    f3, g3, h3 = b.hvp(gates2, dirs, plain=True)
    assert np.array_equal(f2, f3)
    assert not np.array_equal(f1, f2)
    for i in range(len(probs)):
        assert np.array_equal(h2[i], h3[i])


def test_batch_fusion_window_autotuned_and_fixed(rq):
    """The gates-per-pass autotuner times windows 0, 4, 5, 6 after the tile;
    a fixed window gives batched == plain bit for bit and the oracle's values."""
    probs = _problems()[:6]
    gates = [p.gates for p in probs]
    dirs = [w.random_directions(p.n_params, 1, 600 + i) for i, p in enumerate(probs)]
    b = rq.Batch(0)
    for p in probs:
        b.add_problem(p)
    f0, g0, h0 = b.hvp(gates, dirs)
    info = b.info()
    assert all(v > 0 for v in info["fusion_tune_ms"].values()), info
    assert info["fusion_window"] in (0, 4, 5, 6)
    b.set_fusion(6)
    f1, g1, h1 = b.hvp(gates, dirs)
    f2, g2, h2 = b.hvp(gates, dirs, plain=True)
    assert b.info()["fusion_window"] == 6
    assert np.array_equal(f1, f2)
    for i, p in enumerate(probs):
        assert np.array_equal(g1[i], g2[i]) and np.array_equal(h1[i], h2[i])
        assert abs(f1[i] - f0[i]) <= 1e-13 * abs(f0[i])
        assert_close(h1[i], h0[i], p.n, rtol=1e-13)
        if p.n <= 8:
            f, g, hv, _ = oracle_eval(p, range(1 << p.n), dirs[i], chunk=64)
            assert abs(f1[i] - f) <= 1e-12 * abs(f)
            assert_close(g1[i], g, p.n)
            assert_close(h1[i], hv, p.n)
