"""Degenerate cases with closed forms, on the device.

* J = 0: the chain's H is diagonal (on-site terms only) and the Trotter
  circuit is exact, so C(G) = U, f = -2^n and the Riemannian gradient
  vanishes; the HVP (not zero at an optimum) is compared with the oracle.
* t = 0: U = I and every Trotter gate is the identity: f = -2^n, gradient 0.
* One site (n = 2), one gate G on (up, down): f = -Re Tr(U^dagger G) with
  U = diag(1, 1, 1, exp(-i U t)); f is linear in G, so the Euclidean gradient
  is -U, the Riemannian gradient is P_G(-U) = G skew(G^dagger (-U)), and the
  Euclidean Hessian vanishes: Hess f(G)[X] = P_G(-X sym(G^dagger gbar)) =
  P_G(X sym(G^dagger U)) (Eq. hessian_def with the Euclidean-to-Riemannian
  correction; X the projected direction).  With parity gates the gate touches
  the implied qubit 0 (the two-amplitude kernels).
"""
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


def _dag(A):
    return A.conj().T


def _skew(A):
    return 0.5 * (A - _dag(A))


def _sym(A):
    return 0.5 * (A + _dag(A))


@pytest.mark.parametrize("L,structure,arith", [(4, 0, 0), (4, 1, 1), (8, 0, 0)])
def test_hopping_free_chain_is_exact(rq, L, structure, arith):
    prob = w.make_problem(L, 5, 0.7, J=0.0, sigma=0.0, seed=3, structure=structure)
    X = w.random_directions(prob.n_params, 1, 4)
    n = prob.n
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        ctx.set_arithmetic(arith)
        if n > 8:
            ctx.set_columns(0, 4096)
        f, g, hv = ctx.hvp(prob.gates, X)
        cols = 4096 if n > 8 else 1 << n
        assert abs(f + cols) <= 1e-12 * cols, f
        assert np.linalg.norm(g) <= 1e-12 * cols, np.linalg.norm(g)
        if n <= 8:
            f0, g0, hv0, _ = oracle_eval(prob, range(1 << n), X, chunk=64)
            assert_close(hv, hv0, n, what="hvp")


def test_zero_time_is_the_identity(rq):
    prob = w.make_problem(4, 5, 0.0, sigma=0.0, seed=6)
    assert np.allclose(prob.gates, np.eye(4))
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        f, g = ctx.grad(prob.gates)
    assert abs(f + 256) <= 1e-12 * 256
    assert np.linalg.norm(g) <= 1e-12 * 256


@pytest.mark.parametrize("structure", [0, 1])
@pytest.mark.parametrize("arith", [0, 1])
def test_single_gate_closed_form(rq, structure, arith):
    Uint, t = 3.0, 0.7
    prob = w.make_problem(1, 3, t, U=Uint, seed=5, sigma=0.3, structure=structure)
    assert prob.n == 2 and prob.n_gates == 1 and tuple(prob.pairs[0]) == (0, 1)
    G = prob.gates[0]
    Ut = np.diag([1.0, 1.0, 1.0, np.exp(-1j * Uint * t)])
    Xraw = w.random_directions(1, 1, 7)
    Xt = G @ _skew(_dag(G) @ Xraw[0, 0])             # P_G
    if structure == 1:
        Xt = Xt * w.parity_mask()
    f_ref = -np.trace(_dag(Ut) @ G).real
    g_ref = G @ _skew(_dag(G) @ (-Ut))
    h_ref = G @ _skew(_dag(G) @ (Xt @ _sym(_dag(G) @ Ut)))
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        ctx.set_arithmetic(arith)
        f, g, hv = ctx.hvp(prob.gates, Xraw)
    assert abs(f - f_ref) <= 1e-12 * max(abs(f_ref), 4e-6), (f, f_ref)
    assert_close(g[0], g_ref, 2, what="gradient")
    assert_close(hv[0, 0], h_ref, 2, what="hvp")
