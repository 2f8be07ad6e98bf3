"""Pins of the oracle trust-region driver."""
import numpy as np

import workloads as w
from oracle import dense, model, riemann, trust_region as tr


def test_tcg_solves_convex_quadratic(rng):
    # Algorithm 11 with a huge radius on an SPD quadratic is plain CG: it
    # converges to -H^{-1} g (a textbook linear solve)
    n = 12
    A = rng.standard_normal((n, n))
    H = A @ A.T + n * np.eye(n)
    g = rng.standard_normal(n)
    eta, Heta, it, code = tr.tcg(g.reshape(1, n), lambda d: (H @ d.ravel()).reshape(1, n),
                                 1e6, 1e-14, 1.0, 200)
    np.testing.assert_allclose(eta.ravel(), -np.linalg.solve(H, g), rtol=1e-8)
    np.testing.assert_allclose(Heta.ravel(), H @ eta.ravel(), rtol=1e-8)
    assert code == 0


def test_tcg_negative_curvature_goes_to_boundary():
    g = np.array([[1.0, 0.0]])
    eta, _, it, code = tr.tcg(g, lambda d: -d, 0.5, 0.1, 1.0, 10)
    assert code == 1
    np.testing.assert_allclose(np.linalg.norm(eta), 0.5, rtol=1e-14)


def test_tr_decreases_cost():
    p = w.make_problem(2, 5, 0.6, seed=5, sigma=5e-2)
    Um = model.target_unitary_dense(model.hamiltonian_dense(2, 1.0, 4.0), 0.6)
    cost = lambda G: dense.cost(p, Um, G)
    grad = lambda G: (dense.cost(p, Um, G), dense.rgrad(p, Um, G))
    hess = lambda G, X: dense.rhess(p, Um, X, gates=G, method="cauchy")
    G, radius = p.gates.copy(), 0.01
    f0 = cost(G)
    prev = f0
    for _ in range(6):
        G, radius, info = tr.tr_step(cost, grad, hess, G, radius, tr.TRParams())
        cur = cost(G)
        assert cur <= prev + 1e-12
        prev = cur
    assert prev < f0
    for i in range(p.n_params):
        np.testing.assert_allclose(G[i].conj().T @ G[i], np.eye(4), atol=1e-13)
