"""Parity at the launch shape of the benchmark.

The sweep kernels hand items to threads in a grid-stride loop whose loads of
the next item are in flight while the current one is computed.  Small
problems give a thread one or two items; the benchmark's 512-column tiles at
n = 16 give each thread of the general-gate backward kernels about a hundred
(2^14 x 512 items over 152 x 2 CTAs of 256 threads), so every stage of the
pipeline is reused many times.  These tests run that shape (and n = 14 with
512-column tiles, ~27 items per thread) in FP64 and in double-float, and
compare f, the Riemannian gradient and the HVP with values the CPU oracle
wrote for the same columns (tests/golden/make_golden.py), element-wise under
the 1e-12 relative rule.
"""
import numpy as np
import pytest

import workloads as w
from tests._helpers import assert_close, load_golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


def _check(got, gold, n, what):
    f, g, hv = got
    assert abs(f - gold["f"]) <= 1e-12 * max(abs(gold["f"]), 1e-6 * 2 ** n), (what, f, gold["f"])
    assert_close(g, gold["rgrad"], n, what=f"{what} rgrad")
    assert_close(hv, gold["hvp"], n, what=f"{what} hvp")
    # element-wise as well: every entry within the norm-wise bound of its array
    for name, a, b in (("rgrad", g, gold["rgrad"]), ("hvp", hv, gold["hvp"])):
        bound = 1e-12 * max(float(np.linalg.norm(b)), 1e-6 * 2 ** n)
        assert float(np.abs(a - b).max()) <= bound, (what, name)


@pytest.mark.parametrize("arith", [0, 1])
def test_n14_tile512(rq, arith):
    gold = load_golden("tile14_general.json")
    prob = w.config_problem("n14")
    X = w.random_directions(prob.n_params, 1, gold["direction_seed"])
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        ctx.set_arithmetic(arith)
        ctx.set_tile(512, 1)
        ctx.set_columns(*gold["columns"])
        assert ctx.info()["columns_per_tile"] == 512 and ctx.info()["n_tiles"] == 1
        _check(ctx.hvp(prob.gates, X), gold, prob.n, f"n14 arith {arith}")


@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("structure,fname,tile,B,n_tiles", [
    (0, "tile16_general.json", 0, 512, 1),   # the benchmark: automatic choice, one 512-column tile
    (1, "tile16_parity.json", 0, 256, 4),    # parity, automatic choice: 256-column tiles (as benchmarked)
    (1, "tile16_parity.json", 512, 512, 2),  # parity: an even and an odd 512-column tile
])
def test_n16_benchmark_tile(rq, arith, structure, fname, tile, B, n_tiles):
    """The benchmark instance in the benchmark's launch configuration (its
    automatic tile choice) and one more tile size, its first columns."""
    gold = load_golden(fname)
    prob = w.config_problem("n16", structure=structure)
    X = w.random_directions(prob.n_params, 1, gold["direction_seed"])
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        ctx.set_arithmetic(arith)
        if tile:
            ctx.set_tile(tile, 1)
        ctx.set_columns(*gold["columns"])
        info = ctx.info()
        assert info["columns_per_tile"] == B and info["n_tiles"] == n_tiles, info
        _check(ctx.hvp(prob.gates, X), gold, prob.n, f"n16 structure {structure} tile {B} arith {arith}")
