"""Every switch of a context crossed with the others: arithmetic (FP64,
double-float), forward-pass fusion (off, window of 5 qubits), sweep grid
(fill the GPU, 8 items per thread), checkpointing (every state, every third),
first-layer and last-layer support (on, off) -- for general and parity gates with tiles and
direction chunks.  Each combination against the oracle at 1e-12 (f, the
Riemannian gradient, two HVPs), and the FP64 combinations with each other at
1e-13 (they differ only in rounding order)."""
import itertools

import numpy as np
import pytest

import workloads as w
from tests._helpers import assert_close, oracle_eval

pytestmark = pytest.mark.gpu

COMBOS = list(itertools.product((0, 1), (0, 5), (0, 8), (1, 3), (True, False), (True, False)))


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


@pytest.mark.parametrize("structure", [0, 1])
def test_all_switch_combinations(rq, structure):
    prob = w.make_problem(4, 7, 0.35, seed=881 + structure, structure=structure)   # n = 8, 7 layers
    X = w.random_directions(prob.n_params, 2, 882)
    f0, g0, h0, _ = oracle_eval(prob, range(1 << prob.n), X, chunk=64)
    ref = None
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        for arith, fusion, grid, ckpt, first, last in COMBOS:
            what = (f"structure {structure} arith {arith} fusion {fusion} grid {grid} ckpt {ckpt} first {first} "
                    f"last {last}")
            ctx.set_arithmetic(arith)
            ctx.set_fusion(fusion)
            ctx.set_checkpointing(ckpt)
            ctx.set_first_layer(first)
            ctx.set_last_layer(last)
            ctx.set_tile(64, 1)          # several tiles (and both parities), two direction chunks
            ctx.set_grid(grid)
            f, g, hv = ctx.hvp(prob.gates, X)
            assert abs(f - f0) <= 1e-12 * abs(f0), what
            assert_close(g, g0, prob.n, what=what + " grad")
            assert_close(hv, h0, prob.n, what=what + " hvp")
            if arith == 0:
                if ref is None:
                    ref = (f, g, hv)
                assert abs(f - ref[0]) <= 1e-13 * abs(ref[0]), what
                assert_close(g, ref[1], prob.n, rtol=1e-13, what=what + " grad vs first")
                assert_close(hv, ref[2], prob.n, rtol=1e-13, what=what + " hvp vs first")


TARGET_COMBOS = list(itertools.product((0, 1), (0, 5), (1, 3), (True, False)))


@pytest.mark.parametrize("kind", ["translation", "dense"])
def test_switch_combinations_other_targets(rq, kind):
    """The same switches (arithmetic, fusion, checkpointing, last-layer
    support) on a periodic tied circuit summed over translation
    representatives, and on a dense random-unitary target (no sectors: the
    last-layer switch must change nothing), against their oracles."""
    if kind == "translation":
        prob = w.make_problem(4, 6, 0.45, seed=883, tied=True, periodic=True)
        X = w.random_directions(prob.n_params, 2, 884)
        f0, g0, h0, _ = oracle_eval(prob, range(1 << prob.n), X, chunk=64)
    else:
        from oracle import dense, riemann
        prob = w.make_problem(3, 5, 0.4, seed=885)
        Umat = w.random_unitary(1 << prob.n, 886)
        X = w.random_directions(prob.n_params, 2, 887)
        f0, g0 = dense.cost(prob, Umat), dense.rgrad(prob, Umat)
        h0 = np.stack([dense.rhess(prob, Umat, riemann.tangent_direction(prob.gates, X[i], 0)) for i in range(2)])
    with rq.Context(0) as ctx:
        if kind == "translation":
            ctx.setup_problem(prob)
        else:
            ctx.setup(0, prob.pairs, prob.param_of, prob.n_params, prob.structure, model=2, dense_U=Umat,
                      n_qubits=prob.n)
        for arith, fusion, ckpt, last in TARGET_COMBOS:
            what = f"{kind} arith {arith} fusion {fusion} ckpt {ckpt} last {last}"
            ctx.set_arithmetic(arith)
            ctx.set_fusion(fusion)
            ctx.set_checkpointing(ckpt)
            ctx.set_last_layer(last)
            if kind == "translation":
                ctx.set_translation(2)
            else:
                ctx.set_tile(32, 1)
            f, g, hv = ctx.hvp(prob.gates, X)
            assert abs(f - f0) <= 1e-12 * max(abs(f0), 1e-6 * 2 ** prob.n), what
            assert_close(g, g0, prob.n, what=what + " grad")
            assert_close(hv, h0, prob.n, what=what + " hvp")
