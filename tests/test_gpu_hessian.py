"""Full Hessian (hole application + second forward passes) against the
oracle's two-hole networks and the device HVP; full-Hessian trust region."""
import numpy as np
import pytest

import workloads as w
from tests._helpers import assert_close, target_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


def _oracle_contracted(prob, X):
    """tie(sum_l' d2F/dG_l dG_l' X_l') from the dense two-hole networks."""
    from oracle import dense, model, riemann
    Um = model.target_unitary_dense(model.hamiltonian_dense(prob.L, prob.J, prob.U, prob.periodic), prob.t)
    Ed = dense.holomorphic_env_dot(prob, Um, X)
    return riemann.tie(Ed, prob.param_of, prob.n_params)


@pytest.mark.parametrize("structure,tied", [(0, False), (1, False), (0, True), (1, True)])
def test_hessian_blocks_against_two_hole_networks(rq, structure, tied):
    prob = w.make_problem(3, 4, 0.6, seed=91, structure=structure, tied=tied)
    ctx = rq.Context(0).setup_problem(prob)
    f, eg, H = ctx.hessian(prob.gates)
    assert np.array_equal(H, H.T)                      # symmetric second derivatives
    X = w.random_directions(prob.n_params, 1, 92)[0]
    if structure == 1:
        X = X * w.parity_mask()
    ref = _oracle_contracted(prob, X)
    got = (H @ X.reshape(-1)).reshape(prob.n_params, 4, 4)
    assert_close(got, ref, prob.n, what="H vec(X)")
    if not tied:                                       # same-gate blocks vanish
        for p in range(prob.n_params):
            assert np.abs(H[p * 16:(p + 1) * 16, p * 16:(p + 1) * 16]).max() == 0
    ctx.set_gradient_space(1)
    f2, eg2 = ctx.grad(prob.gates)
    assert abs(f - f2) <= 1e-12 * abs(f2)
    assert_close(eg, eg2, prob.n, what="euclidean gradient")


def test_hessian_matches_device_hvp_tied12(rq):
    prob = w.config_problem("tied12")
    ctx = rq.Context(0).setup_problem(prob)
    f, eg, H = ctx.hessian(prob.gates)
    ctx.set_gradient_space(1)
    X = w.random_directions(prob.n_params, 1, 93) * w.parity_mask()
    _, _, hv = ctx.hvp(prob.gates, X)
    got = -np.conj(H @ X[0].reshape(-1)).reshape(prob.n_params, 4, 4) * w.parity_mask()
    assert_close(got, hv[0], 12, what="-conj(H X) vs device Euclidean HVP")


@pytest.mark.parametrize("structure", [0, 1])
def test_full_hessian_trust_region_equals_hvp_trust_region(rq, structure):
    prob = w.make_problem(3, 5, 0.6, seed=61, structure=structure, sigma=5e-2)
    c1 = rq.Context(0).setup_problem(prob)
    c2 = rq.Context(0).setup_problem(prob)
    s1 = rq.tr_state(radius=0.05, max_radius=0.2)
    s2 = rq.tr_state(radius=0.05, max_radius=0.2, full_hessian=True)
    G1 = G2 = prob.gates.copy()
    for it in range(4):
        G1 = c1.tr_step(G1, s1)
        G2 = c2.tr_step(G2, s2)
        assert s1.n_inner == s2.n_inner and s1.tcg_exit == s2.tcg_exit and s1.accepted == s2.accepted
        assert abs(s1.rho - s2.rho) <= 1e-6 * max(1.0, abs(s1.rho))
        assert np.abs(G1 - G2).max() <= 1e-10


def test_hessian_with_translation_representatives(rq):
    prob = w.make_problem(4, 5, 0.4, seed=95, tied=True, periodic=True, structure=1)
    ctx = rq.Context(0).setup_problem(prob)
    f, eg, H = ctx.hessian(prob.gates)
    ctx.set_translation(2)
    f2, eg2, H2 = ctx.hessian(prob.gates)
    assert abs(f2 - f) <= 1e-12 * abs(f)
    assert_close(eg2, eg, 8)
    assert_close(H2, H, 8, what="H with orbit representatives")
