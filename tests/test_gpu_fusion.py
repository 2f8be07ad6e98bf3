"""Window fusion of the forward pass (rq_set_fusion) against the unfused
schedule and the oracle.

A fused pass applies several gates that fit in a window of stored qubits to
shared-memory blocks of the tile; gates move only past gates on disjoint
qubits, with which they commute, so f, the gradient and the HVPs agree with
the unfused schedule up to the order of the floating-point sums.
"""
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


def _pair(rq, prob, q, arith=0, tile=0, dirs=0):
    out = []
    for fq in (0, q):
        c = rq.Context(0).setup_problem(prob)
        c.set_arithmetic(arith)
        if tile or dirs:
            c.set_tile(tile, dirs)
        c.set_fusion(fq)
        out.append(c)
    return out


def _same(a, b, n, tol=1e-13):
    assert abs(a[0] - b[0]) <= tol * max(abs(b[0]), 1e-6 * 2 ** n), (a[0], b[0])
    for x, y in zip(a[1:], b[1:]):
        assert_close(x, y, n, rtol=tol)


@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("structure", [0, 1])
@pytest.mark.parametrize("q", [4, 6])
def test_fused_equals_unfused_and_oracle_n8(rq, q, structure, arith):
    prob = w.config_problem("small", structure=structure)
    X = w.random_directions(prob.n_params, 2, 102)
    plain, fused = _pair(rq, prob, q, arith)
    info = fused.fusion_info()
    assert info["fused_gates"] > 0 and info["passes"] < prob.n_gates, info
    got = fused.hvp(prob.gates, X)
    _same(got, plain.hvp(prob.gates, X), prob.n)
    f, g, hv, _ = oracle_eval(prob, range(1 << prob.n), X, chunk=64)
    _same(got, (f, g, hv), prob.n, tol=1e-12)
    assert abs(fused.cost(prob.gates) - f) <= 1e-12 * abs(f)
    _same(fused.grad(prob.gates), plain.grad(prob.gates), prob.n)


@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("structure,fname,tile", [(0, "tile16_general.json", 0), (1, "tile16_parity.json", 256)])
def test_fused_benchmark_tile_against_oracle(rq, arith, structure, fname, tile):
    gold = load_golden(fname)
    prob = w.config_problem("n16", structure=structure)
    X = w.random_directions(prob.n_params, 1, gold["direction_seed"])
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        ctx.set_arithmetic(arith)
        ctx.set_fusion(6)
        if tile:
            ctx.set_tile(tile, 1)
        ctx.set_columns(*gold["columns"])
        f, g, hv = ctx.hvp(prob.gates, X)
        assert abs(f - gold["f"]) <= 1e-12 * abs(gold["f"])
        assert_close(g, gold["rgrad"], prob.n, what="rgrad")
        assert_close(hv, gold["hvp"], prob.n, what="hvp")
        assert abs(ctx.cost(prob.gates) - gold["f"]) <= 1e-12 * abs(gold["f"])


@pytest.mark.parametrize("q", [3, 5])
def test_fused_n14_tile_and_four_directions(rq, q):
    gold = load_golden("tile14_general.json")
    prob = w.config_problem("n14")
    X = w.random_directions(prob.n_params, 1, gold["direction_seed"])
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        ctx.set_fusion(q)
        ctx.set_tile(512, 1)
        ctx.set_columns(*gold["columns"])
        f, g, hv = ctx.hvp(prob.gates, X)
        assert abs(f - gold["f"]) <= 1e-12 * abs(gold["f"])
        assert_close(g, gold["rgrad"], prob.n, what="rgrad")
        assert_close(hv, gold["hvp"], prob.n, what="hvp")
    # four directions swept together: four tangent blocks per fused pass
    X4 = w.random_directions(prob.n_params, 4, 403)
    plain, fused = _pair(rq, prob, q, tile=64, dirs=4)
    for c in (plain, fused):
        c.set_columns(1000, 1200)
    _same(fused.hvp(prob.gates, X4), plain.hvp(prob.gates, X4), prob.n)


def test_fusion_falls_back_and_keeps_options(rq):
    """Tiles below 32 columns, a checkpoint interval above 1, first-layer
    support off, translation sums, ragged ranges and a trust-region step."""
    prob = w.make_problem(4, 6, 0.45, seed=81, tied=True, periodic=True, structure=1)
    X = w.random_directions(prob.n_params, 2, 82)
    f, g, hv, _ = oracle_eval(prob, range(256), X, chunk=64)
    for setup in (lambda c: c.set_tile(16, 1), lambda c: c.set_checkpointing(3),
                  lambda c: c.set_first_layer(False), lambda c: c.set_translation(2)):
        with rq.Context(0) as ctx:
            ctx.setup_problem(prob)
            ctx.set_fusion(6)
            setup(ctx)
            got = ctx.hvp(prob.gates, X)
            _same(got, (f, g, hv), prob.n, tol=1e-12)
    plain, fused = _pair(rq, w.config_problem("small"), 5, tile=32)
    p = w.config_problem("small")
    for c in (plain, fused):
        c.set_columns(7, 200)                  # ragged: 193 = 6 * 32 + 1
    Xs = w.random_directions(p.n_params, 1, 5)
    _same(fused.hvp(p.gates, Xs), plain.hvp(p.gates, Xs), p.n)
    s0, s1 = rq.tr_state(), rq.tr_state()
    g0, g1 = plain.tr_step(p.gates, s0), fused.tr_step(p.gates, s1)
    assert s0.n_inner == s1.n_inner and s0.tcg_exit == s1.tcg_exit
    assert np.abs(g0 - g1).max() < 1e-12


def test_fusion_argument_checks(rq):
    with rq.Context(0) as ctx:
        for bad in (1, 2, 7, -1):
            with pytest.raises(rq.RQError) as e:
                ctx.set_fusion(bad)
            assert e.value.code == rq.RQ_EINVAL
