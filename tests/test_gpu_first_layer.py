"""First-layer support: the FP64 general-gate sweeps of the leading run of
disjoint gates visit only the items where the state can be nonzero.  Results
equal the full sweeps up to the order of the sums, for every column layout."""
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


def _both(rq, prob, setup, gates, X):
    out = []
    for on in (False, True):
        ctx = rq.Context(0).setup_problem(prob)
        setup(ctx)
        ctx.set_first_layer(on)
        out.append(ctx.hvp(gates, X))
        ctx.close()
    return out


@pytest.mark.parametrize("case,structure,arith", [
    ("full", 0, 0), ("padded_range", 0, 0), ("checkpointed", 0, 0), ("four_dirs", 0, 0), ("small_tile", 0, 0),
    ("full", 1, 0), ("checkpointed", 1, 0), ("four_dirs", 1, 0),
    ("full", 0, 1), ("padded_range", 0, 1), ("full", 1, 1), ("four_dirs", 1, 1)])
def test_first_layer_matches_full_sweeps(rq, case, structure, arith):
    prob = w.config_problem("small" if case != "checkpointed" else "tied12", structure=structure)
    k = 4 if case == "four_dirs" else 1
    X = w.random_directions(prob.n_params, k, 31)

    def setup(ctx):
        ctx.set_arithmetic(arith)
        if case == "padded_range":
            ctx.set_columns(3, 200)   # not a multiple of the tile: padding columns
        if case == "checkpointed":
            ctx.set_columns(1000, 1300)
            ctx.set_checkpointing(5)
        if case == "small_tile":
            ctx.set_tile(16, 2)

    off, on = _both(rq, prob, setup, prob.gates, X)
    if arith == 1:  # double-float: the same sums in another order, ~48-bit arithmetic
        assert abs(on[0] - off[0]) <= 1e-12 * abs(off[0])
        assert_close(on[1], off[1], prob.n, rtol=1e-12, what="rgrad")
        for i in range(k):
            assert_close(on[2][i], off[2][i], prob.n, rtol=1e-12, what=f"hvp {i}")
        return
    assert abs(on[0] - off[0]) <= 1e-13 * abs(off[0])
    assert_close(on[1], off[1], prob.n, rtol=1e-13, what="rgrad")
    for i in range(k):
        assert_close(on[2][i], off[2][i], prob.n, rtol=1e-13, what=f"hvp {i}")


def test_first_layer_against_oracle_fourteen_qubits(rq):
    prob = w.config_problem("n14")
    X = w.random_directions(prob.n_params, 1, 32)
    cols = [0, 1, 777, 5000, 16383, 0b10101010101010]
    ref = oracle_eval(prob, cols, X)
    ctx = rq.Context(0).setup_problem(prob)
    ctx.set_first_layer(True)
    f = g = h = None
    for c in cols:   # one column at a time: a single-column tile with padding
        ctx.set_columns(c, c + 1)
        fc, gc, hc = ctx.hvp(prob.gates, X)
        f = fc if f is None else f + fc
        g = gc if g is None else g + gc
        h = hc if h is None else h + hc
    assert abs(f - ref[0]) <= 1e-12 * max(abs(ref[0]), 1e-6 * 2 ** prob.n)
    assert_close(g, ref[1], prob.n, what="rgrad")
    assert_close(h[0], ref[2][0], prob.n, what="hvp")


def test_first_layer_is_faster(rq):
    prob = w.config_problem("n14")
    X = w.random_directions(prob.n_params, 1, 33)
    ms = {}
    for on in (False, True):
        ctx = rq.Context(0).setup_problem(prob)
        ctx.set_first_layer(on)
        ctx.set_columns(0, 1024)
        ctx.hvp(prob.gates, X)
        ctx.profile_start()
        ctx.hvp(prob.gates, X)
        prof = ctx.profile_stop()
        ms[on] = sum(v["ms"] for k2, v in prof.items() if k2.startswith(("fwd", "bwd")))
        ctx.close()
    print(f"sweep kernels: full {ms[False]:.2f} ms, first-layer support {ms[True]:.2f} ms")
    assert ms[True] < ms[False]
