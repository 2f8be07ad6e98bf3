"""Checkpointing every r gates with recomputation gives bitwise the results
of keeping every state, with a smaller workspace."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


@pytest.mark.parametrize("name,structure,arith,cols", [
    ("small", 0, 0, None), ("small", 1, 1, None), ("tied12", 1, 0, (0, 700)), ("n16", 0, 0, (1795, 1799))])
def test_recompute_is_bitwise_equal(rq, name, structure, arith, cols):
    prob = w.config_problem(name, structure=structure)
    X = w.random_directions(prob.n_params, 3, 11)
    ctx = rq.Context(0).setup_problem(prob)
    ctx.set_arithmetic(arith)
    if cols:
        ctx.set_columns(*cols)
    ctx.set_tile(0, 2)
    ref = ctx.hvp(prob.gates, X)
    bytes1 = ctx.info()["workspace_bytes"]
    for r in (2, 5, 7, prob.n_gates):
        ctx.set_checkpointing(r)
        ctx.set_tile(0, 2)
        got = ctx.hvp(prob.gates, X)
        assert got[0] == ref[0], r
        assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2]), r
    ctx.set_checkpointing(7)
    assert ctx.info()["workspace_bytes"] <= bytes1
    with pytest.raises(rq.RQError):
        ctx.hessian(prob.gates)
    ctx.set_checkpointing(1)
    ctx.set_tile(0, 2)
    assert ctx.hvp(prob.gates, X)[0] == ref[0]
