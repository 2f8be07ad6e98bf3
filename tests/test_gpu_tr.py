"""Trust-region iterations on the device against the oracle trust region."""
import json
import os

import numpy as np
import pytest

import workloads as w
from tests._helpers import load_golden, target_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


def _oracle_fns(prob):
    from oracle import statevector as sv
    st = target_for(prob)
    cols = range(1 << prob.n)
    cost = lambda G: sv.cost_grad_hvp(prob, st, cols, None, gates=G, chunk=64)[0]

    def grad(G):
        f, g, _, _ = sv.cost_grad_hvp(prob, st, cols, None, gates=G, chunk=64)
        return f, g

    def hess(G, X):
        # X is already tangent; the projection inside is then the identity
        _, _, hv, _ = sv.cost_grad_hvp(prob, st, cols, X[None], gates=G, chunk=64)
        return hv[0]
    return cost, grad, hess


@pytest.mark.parametrize("structure", [0, 1])
def test_tr_steps_match_oracle(rq, structure):
    from oracle import trust_region as tr
    prob = w.make_problem(3, 5, 0.6, seed=61, structure=structure, sigma=5e-2)
    cost, grad, hess = _oracle_fns(prob)
    params = tr.TRParams(radius=0.05, max_radius=0.2)
    G0, radius0 = prob.gates.copy(), params.radius
    ctx = rq.Context(0).setup_problem(prob)
    st = rq.tr_state(radius=0.05, max_radius=0.2)
    G1 = prob.gates.copy()
    for it in range(4):
        G0, radius0, info = tr.tr_step(cost, grad, hess, G0, radius0, params, structure)
        G1 = ctx.tr_step(G1, st)
        assert st.n_inner == info["n_inner"] and st.tcg_exit == info["tcg_exit"], (it, st.n_inner, info)
        assert bool(st.accepted) == bool(info["accepted"])
        assert abs(st.f - info["f"]) <= 1e-12 * abs(info["f"])
        assert abs(st.f_new - info["f_new"]) <= 1e-11 * abs(info["f_new"])
        assert abs(st.rho - info["rho"]) <= 1e-6 * max(1.0, abs(info["rho"]))
        assert st.radius == pytest.approx(radius0, rel=1e-12)
        assert np.abs(G1 - G0).max() <= 1e-10, (it, np.abs(G1 - G0).max())


def test_thirty_iterations_tied_parity_twelve_qubits(rq):
    prob = w.config_problem("tied12")
    path = os.path.join(os.path.dirname(__file__), "golden", "tied12_full_basis.json")
    gold = json.load(open(path))
    g_gold = (np.array(gold["rgrad"]["re"]) + 1j * np.array(gold["rgrad"]["im"]))
    ctx = rq.Context(0).setup_problem(prob)
    st = rq.tr_state(radius=0.01, max_radius=0.1)
    G = prob.gates.copy()
    f_prev = None
    for it in range(30):
        G = ctx.tr_step(G, st)
        if it == 0:
            assert abs(st.f - gold["f"]) <= 1e-12 * abs(gold["f"])
            assert abs(st.grad_norm - np.linalg.norm(g_gold)) <= 1e-12 * np.linalg.norm(g_gold)
        if f_prev is not None:
            assert st.f <= f_prev + 1e-9
        f_prev = st.f_new if st.accepted else st.f
    assert f_prev < gold["f"]
    mask = w.parity_mask()
    for p in range(prob.n_params):
        np.testing.assert_allclose(G[p].conj().T @ G[p], np.eye(4), atol=1e-12)
        assert np.all(G[p][~mask] == 0)


def _follow(rq, ctx, prob, gold, r0, rmax, what, f_rtol=1e-12):
    """Device trust-region steps against the oracle's trajectory step by step:
    identical acceptance, inner iterations and tCG exit; f to ``f_rtol``, rho
    to 1e-6, the radius after the step to 1e-12 and the gates (where stored)
    to 1e-10.  Rounding differences between the two sides grow along a long
    trajectory, so a long one is held to 1e-10 per step (and its final f to
    1e-9) instead of 1e-12."""
    st = rq.tr_state(radius=r0, max_radius=rmax)
    G = prob.gates.copy()
    for rec in gold:
        G = ctx.tr_step(G, st)
        it = (what, rec["step"])
        assert st.n_inner == rec["n_inner"] and st.tcg_exit == rec["tcg_exit"], (it, st.n_inner, st.tcg_exit)
        assert bool(st.accepted) == rec["accepted"], it
        assert abs(st.f - rec["f"]) <= f_rtol * abs(rec["f"]), (it, st.f, rec["f"])
        assert abs(st.f_new - rec["f_new"]) <= 10 * f_rtol * abs(rec["f_new"]), (it, st.f_new, rec["f_new"])
        assert abs(st.rho - rec["rho"]) <= 1e-6 * max(1.0, abs(rec["rho"])), (it, st.rho, rec["rho"])
        assert st.radius == pytest.approx(rec["radius"], rel=1e-12), (it, st.radius, rec["radius"])
        if "gates" in rec:
            assert np.abs(G - rec["gates"]).max() <= 1e-10, (it, np.abs(G - rec["gates"]).max())
    return G, st


def test_tied_parity_twelve_qubits_trajectory_matches_oracle(rq):
    """Three iterations over all 4096 columns of the tied parity n = 12
    workload against the oracle's trust region (tests/golden/make_golden.py)."""
    gold = load_golden("tr12_trajectory.json")
    prob = w.config_problem("tied12")
    ctx = rq.Context(0).setup_problem(prob)
    _follow(rq, ctx, prob, gold["steps"], gold["radius0"], gold["max_radius"], "tied12")


@pytest.mark.parametrize("key", ["long", "shrink"])
def test_n8_trajectory_matches_oracle(rq, key):
    """Thirty iterations (radius growth, boundary and interior tCG exits), and
    six from a far start with an oversized radius (rejections, shrinks), at
    n = 8 against the oracle's trajectories; the final f to 1e-9."""
    gold = load_golden("tr8_trajectory.json")[key]
    prob = w.make_problem(gold["L"], gold["depth"], gold["t"], seed=gold["seed"], sigma=gold["sigma"])
    ctx = rq.Context(0).setup_problem(prob)
    G, st = _follow(rq, ctx, prob, gold["steps"], gold["radius0"], gold["max_radius"], key,
                    f_rtol=1e-10 if key == "long" else 1e-12)
    last = gold["steps"][-1]
    f_last = last["f_new"] if last["accepted"] else last["f"]
    f_dev = st.f_new if st.accepted else st.f
    assert abs(f_dev - f_last) <= 1e-9 * abs(f_last)
