"""Translation-representative basis sums against full basis sums and the oracle."""
import time

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


@pytest.mark.parametrize("structure", [0, 1])
def test_representatives_match_oracle_n8(rq, structure):
    prob = w.make_problem(4, 6, 0.45, seed=81, tied=True, periodic=True, structure=structure)
    X = w.random_directions(prob.n_params, 2, 82)
    f, g, hv, _ = oracle_eval(prob, range(256), X, chunk=64)
    ctx = rq.Context(0).setup_problem(prob)
    ctx.set_translation(2)
    info = ctx.info()
    assert info["columns"] == 256            # the range is the whole basis
    f2, g2, hv2 = ctx.hvp(prob.gates, X)
    assert abs(f2 - f) <= 1e-12 * abs(f)
    assert_close(g2, g, 8, what="rgrad")
    assert_close(hv2, hv, 8, what="hvp")


@pytest.mark.parametrize("arith", [0, 1])
def test_representatives_match_full_sum_n12(rq, arith):
    prob = w.make_problem(6, 9, 0.5, seed=83, tied=True, periodic=True, structure=1)
    X = w.random_directions(prob.n_params, 1, 84)
    ctx = rq.Context(0).setup_problem(prob)
    ctx.set_arithmetic(arith)
    t0 = time.perf_counter()
    full = ctx.hvp(prob.gates, X)
    t_full = time.perf_counter() - t0
    ctx.set_translation(2)
    t0 = time.perf_counter()
    rep = ctx.hvp(prob.gates, X)
    t_rep = time.perf_counter() - t0
    assert abs(rep[0] - full[0]) <= 1e-12 * abs(full[0])
    assert_close(rep[1], full[1], 12, what="rgrad")
    assert_close(rep[2], full[2], 12, what="hvp")
    assert ctx.info()["n_tiles"] >= 1
    print(f"full {t_full:.3f}s representatives {t_rep:.3f}s")
    ctx.set_translation(0)
    again = ctx.hvp(prob.gates, X)
    assert again[0] == full[0] and np.array_equal(again[1], full[1])


def test_translation_rejections(rq):
    ctx = rq.Context(0).setup_problem(w.make_problem(4, 5, 0.3, seed=1, tied=True))   # open chain
    with pytest.raises(rq.RQError):
        ctx.set_translation(2)
    ctx = rq.Context(0).setup_problem(w.make_problem(4, 5, 0.3, seed=1, periodic=True))  # untied gates
    with pytest.raises(rq.RQError):
        ctx.set_translation(2)
    ctx = rq.Context(0).setup_problem(w.make_problem(4, 5, 0.3, seed=1, periodic=True, tied=True))
    with pytest.raises(rq.RQError):
        ctx.set_translation(3)
    ctx.set_translation(2)
    with pytest.raises(rq.RQError):
        ctx.set_columns(0, 100)
