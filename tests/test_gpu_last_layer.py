"""Last-layer support (rq_set_last_layer): the backward kernels of the
trailing run of disjoint gates skip the items whose adjoint amplitudes are
zero because U|j> lives in j's particle-number sector.  Skipping must change
nothing but the rounding: on and off agree to 1e-13 and both match the
oracle; the items the profile counts as skipped equal a brute-force count of
the zero items of U|j> propagated backwards through the run with the actual
gates."""
import numpy as np
import pytest

import workloads as w
from tests._helpers import assert_close, oracle_eval, target_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


def _problems():
    return {
        "spinful open n8": (w.make_problem(4, 5, 0.3, seed=901), {}),
        "spinful open n10 depth 7": (w.make_problem(5, 7, 0.45, seed=902), {}),
        "spinful periodic tied n8, translation": (w.make_problem(4, 6, 0.45, seed=903, tied=True, periodic=True),
                                                  {"translation": 2}),
        "spinless open n8": (w.make_spinless_problem(8, 5, 0.4, seed=904), {}),
        "spinful n8, fusion 5, tiles, df64": (w.make_problem(4, 7, 0.35, seed=905), {"fusion": 5, "tile": 64,
                                                                                      "arith": 1}),
        "spinful n8, checkpoints": (w.make_problem(4, 9, 0.35, seed=906), {"ckpt": 3, "tile": 32}),
    }


@pytest.mark.parametrize("name", list(_problems()))
def test_on_equals_off_and_oracle(rq, name):
    prob, opt = _problems()[name]
    X = w.random_directions(prob.n_params, 2, 907)
    res = {}
    for on in (True, False):
        with rq.Context(0) as ctx:
            ctx.setup_problem(prob)
            if "translation" in opt:
                ctx.set_translation(opt["translation"])
            if "fusion" in opt:
                ctx.set_fusion(opt["fusion"])
            if "ckpt" in opt:
                ctx.set_checkpointing(opt["ckpt"])
            if "tile" in opt:
                ctx.set_tile(opt["tile"], 1)
            if "arith" in opt:
                ctx.set_arithmetic(opt["arith"])
            ctx.set_last_layer(on)
            res[on] = ctx.hvp(prob.gates, X)
    (f1, g1, h1), (f0, g0, h0) = res[True], res[False]
    assert abs(f1 - f0) <= 1e-13 * abs(f0), name
    assert_close(g1, g0, prob.n, rtol=1e-13, what=f"{name} grad on vs off")
    assert_close(h1, h0, prob.n, rtol=1e-13, what=f"{name} hvp on vs off")
    f, g, hv, _ = oracle_eval(prob, range(1 << prob.n), X, chunk=64)
    assert abs(f1 - f) <= 1e-12 * abs(f), name
    assert_close(g1, g, prob.n, what=f"{name} grad vs oracle")
    assert_close(h1, hv, prob.n, what=f"{name} hvp vs oracle")


def _zero_items_bruteforce(prob):
    """Items of the trailing run of disjoint gates whose four adjoint
    amplitudes are all exactly zero, summed over all columns: U|j> from the
    oracle's sector blocks, propagated backwards with the conjugate-transposed
    gates of the run (exact zeros are structural: the gates are generic)."""
    from oracle import statevector as sv
    n, g = prob.n, prob.n_gates
    tail, used = [], set()
    for l in range(g - 1, -1, -1):
        a, b = (int(q) for q in prob.pairs[l])
        if a in used or b in used:
            break
        used |= {a, b}
        tail.append(l)
    lam = target_for(prob).columns(range(1 << n))     # [columns, 2^n]: row j = U|j>
    zeros = 0
    for l in tail:
        a, b = (int(q) for q in prob.pairs[l])
        sa, sb = 1 << (n - 1 - a), 1 << (n - 1 - b)
        x0 = np.array([x for x in range(1 << n) if not (x & sa) and not (x & sb)])
        nz = (lam[:, x0] != 0) | (lam[:, x0 | sb] != 0) | (lam[:, x0 | sa] != 0) | (lam[:, x0 | sa | sb] != 0)
        zeros += int((~nz).sum())
        G = prob.gates[prob.param_of[l]]
        lam = sv.apply_gate(G.conj().T, (a, b), lam, n)
    return zeros, len(tail)


def test_skipped_items_match_bruteforce(rq):
    prob = w.make_problem(4, 5, 0.3, seed=911)           # 16 gates: first layer and last layer disjoint
    X = w.random_directions(prob.n_params, 1, 912)
    zeros, run = _zero_items_bruteforce(prob)
    assert run == 4 and zeros > 0
    flops = {}
    for on in (True, False):
        with rq.Context(0) as ctx:
            ctx.setup_problem(prob)
            ctx.set_last_layer(on)
            ctx.hvp(prob.gates, X)
            ctx.profile_start()
            ctx.hvp(prob.gates, X)
            prof = ctx.profile_stop()
        flops[on] = (prof["bwd_gate_dir"]["flops"], prof["bwd_gate_base"]["flops"])
    # per general-gate item: direction step 64 complex multiply-adds, base step 32 (8 flops each)
    assert flops[False][0] - flops[True][0] == pytest.approx(zeros * 512.0, rel=1e-12)
    assert flops[False][1] - flops[True][1] == pytest.approx(zeros * 256.0, rel=1e-12)


@pytest.mark.parametrize("structure", [0, 1])
def test_gates_in_both_runs(rq, structure):
    """A one-layer circuit: every gate is in the leading and in the trailing
    run of disjoint gates.  Every combination of first- and last-layer
    support gives the same results, and the oracle's."""
    prob = w.make_problem(4, 1, 0.6, seed=921, structure=structure)
    X = w.random_directions(prob.n_params, 2, 922)
    f0, g0, h0, _ = oracle_eval(prob, range(1 << prob.n), X, chunk=64)
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        ctx.set_tile(64, 2)
        for first in (True, False):
            for last in (True, False):
                what = f"structure {structure} first {first} last {last}"
                ctx.set_first_layer(first)
                ctx.set_last_layer(last)
                f, g, hv = ctx.hvp(prob.gates, X)
                assert abs(f - f0) <= 1e-12 * max(abs(f0), 1e-6 * 2 ** prob.n), what
                assert_close(g, g0, prob.n, what=what + " grad")
                assert_close(hv, h0, prob.n, what=what + " hvp")
