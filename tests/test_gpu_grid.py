"""Sweep grid (rq_set_grid, rq_batch_set_grid): fewer CTAs per sweep change
only the rounding of the environment sums; results stay within the parity
tolerance of the default grid and of the oracle, reproducible for a given
grid, and a batch evaluated as one graph equals its plain evaluation bit for
bit at the same grid."""
import numpy as np
import pytest

import workloads as w
from tests._helpers import assert_close, load_golden, oracle_eval

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


@pytest.mark.parametrize("structure", [0, 1])
def test_grid_changes_only_rounding(rq, structure):
    prob = w.make_problem(5, 5, 0.4, seed=71, structure=structure)   # n = 10: 1024 columns
    X = w.random_directions(prob.n_params, 2, 72)
    f0, g0, h0, _ = oracle_eval(prob, range(1 << prob.n), X, chunk=64)
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        ctx.set_tile(256, 2)
        base = ctx.hvp(prob.gates, X)
        ctas0 = ctx.info()["ctas_per_sweep"]
        seen = {ctas0}
        for m in (1, 3, 16, 1000):
            ctx.set_grid(m)
            ctas = ctx.info()["ctas_per_sweep"]
            assert 1 <= ctas <= ctas0
            seen.add(ctas)
            f, g, hv = ctx.hvp(prob.gates, X)
            f2, g2, hv2 = ctx.hvp(prob.gates, X)          # reproducible for a given grid
            assert f == f2 and np.array_equal(g, g2) and np.array_equal(hv, hv2)
            assert abs(f - base[0]) <= 1e-13 * abs(base[0])
            assert_close(g, base[1], prob.n, rtol=1e-13, what=f"grid {m} grad")
            assert_close(hv, base[2], prob.n, rtol=1e-13, what=f"grid {m} hvp")
            assert abs(f - f0) <= 1e-12 * abs(f0)
            assert_close(g, g0, prob.n, what=f"grid {m} grad vs oracle")
            assert_close(hv, h0, prob.n, what=f"grid {m} hvp vs oracle")
        assert len(seen) >= 3, seen                        # the grid really changed
        ctx.set_grid(1000)
        assert ctx.info()["ctas_per_sweep"] == 1           # one CTA sweeps the whole tile
        ctx.set_grid(0)
        assert ctx.info()["ctas_per_sweep"] == ctas0
        f, g, hv = ctx.hvp(prob.gates, X)
        assert f == base[0] and np.array_equal(hv, base[2])  # back to the default grid: same bits


def test_grid_at_benchmark_shape(rq):
    """n = 16, one 512-column tile: a grid of 256 items per thread (128 CTAs
    instead of the default 304) against the oracle-written values of those
    columns."""
    gold = load_golden("tile16_general.json")
    prob = w.config_problem("n16")
    X = w.random_directions(prob.n_params, 1, gold["direction_seed"])
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        ctx.set_columns(*gold["columns"])
        ctx.set_grid(256)
        assert ctx.info()["ctas_per_sweep"] == (1 << 14) * 512 // (256 * 256)
        f, g, hv = ctx.hvp(prob.gates, X)
    assert abs(f - gold["f"]) <= 1e-12 * abs(gold["f"])
    assert_close(g, gold["rgrad"], prob.n, what="rgrad")
    assert_close(hv, gold["hvp"], prob.n, what="hvp")


def test_grid_invalid(rq):
    prob = w.make_problem(3, 3, 0.4, seed=73)
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        with pytest.raises(rq.RQError):
            ctx.set_grid(-1)
        with pytest.raises(rq.RQError):
            ctx.set_grid(1 << 21)
    b = rq.Batch(0)
    try:
        with pytest.raises(rq.RQError):
            b.set_grid(-2)
    finally:
        b.close()


def test_batch_grid_autotuned_and_fixed(rq):
    probs = w.batch_problems(8, seed=331, sizes=(3, 4, 5), depths=(3, 5))
    gates = [p.gates for p in probs]
    dirs = [w.random_directions(p.n_params, 1, 700 + i) for i, p in enumerate(probs)]
    b = rq.Batch(0)
    try:
        for p in probs:
            b.add_problem(p)
        f1, g1, h1 = b.hvp(gates, dirs)                  # tile, grid and window autotuned
        info = b.info()
        assert info["grid_items"] in (0, 8, 16, 32, 64)
        assert all(v > 0 for v in info["grid_tune_ms"].values()), info
        f2, g2, h2 = b.hvp(gates, dirs, plain=True)      # same grid: same bits
        assert np.array_equal(f1, f2)
        for i in range(len(probs)):
            assert np.array_equal(g1[i], g2[i]) and np.array_equal(h1[i], h2[i])
        b.set_grid(0)
        f3, g3, h3 = b.hvp(gates, dirs)
        f4, g4, h4 = b.hvp(gates, dirs, plain=True)
        assert b.info()["grid_items"] == 0 and np.array_equal(f3, f4)
        for i, p in enumerate(probs):
            assert np.array_equal(h3[i], h4[i])
            assert abs(f3[i] - f1[i]) <= 1e-13 * abs(f1[i])
            assert_close(h3[i], h1[i], p.n, rtol=1e-13)
            if p.n <= 8:
                f, g, hv, _ = oracle_eval(p, range(1 << p.n), dirs[i], chunk=64)
                assert abs(f1[i] - f) <= 1e-12 * abs(f)
                assert_close(g1[i], g, p.n)
                assert_close(h1[i], hv, p.n)
    finally:
        b.close()
