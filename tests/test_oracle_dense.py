"""Pins of the dense oracle O1 and of the Riemannian layer: closed forms,
invariants, exact special cases and brute-force finite differences."""
import numpy as np
import pytest
import scipy.linalg

import workloads as w
from oracle import dense, model, riemann


def _setup(L=3, depth=3, t=0.4, seed=11, structure=0, tied=False, U=4.0, J=1.0, sigma=1e-2):
    p = w.make_problem(L, depth, t, U=U, J=J, seed=seed, structure=structure, tied=tied, sigma=sigma)
    Um = model.target_unitary_dense(model.hamiltonian_dense(L, J, U), t)
    return p, Um


def test_embed_is_kronecker_for_neighbours(rng):
    n = 5
    G = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    for q in range(n - 1):
        ref = np.kron(np.kron(np.eye(1 << q), G), np.eye(1 << (n - q - 2)))
        np.testing.assert_array_equal(dense.embed(G, (q, q + 1), n), ref)


def test_embed_reversed_pair_is_swap_conjugate(rng):
    G = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    S = np.eye(4)[[0, 2, 1, 3]]
    np.testing.assert_array_equal(dense.embed(G, (1, 0), 2), S @ G @ S)
    # long range pair (0, 2) on 3 qubits = SWAP(1,2) (G x I) SWAP(1,2)
    P = dense.embed(S, (1, 2), 3)
    np.testing.assert_allclose(dense.embed(G, (0, 2), 3), P @ np.kron(G, np.eye(2)) @ P, atol=0)


def test_cost_bound_and_frobenius_identity():
    # Eq. opt_distance: ||C - U||_F^2 = 2 Tr I - 2 Re Tr[U^dag C] = 2*2^n + 2 f
    p, Um = _setup()
    f = dense.cost(p, Um)
    W = dense.circuit_matrix(dense.expand(p), p.pairs, p.n)
    np.testing.assert_allclose(np.linalg.norm(W - Um) ** 2, 2 * 2 ** p.n + 2 * f, rtol=1e-12)
    assert f >= -2 ** p.n
    np.testing.assert_allclose(-np.trace(Um.conj().T @ Um).real, -2 ** p.n, rtol=1e-14)


def test_exact_trotter_without_hopping():
    # J = 0: every term commutes, the noise-free Trotter circuit is exact:
    # f = -2^n and the Riemannian gradient vanishes
    p, Um = _setup(L=3, depth=7, J=0.0, sigma=0.0)
    np.testing.assert_allclose(dense.cost(p, Um), -2 ** p.n, rtol=1e-14)
    assert np.abs(dense.rgrad(p, Um)).max() < 1e-12


def test_exact_trotter_two_sites_no_interaction():
    # L = 2, U = 0: one bond per spin chain, the two hops commute
    p, Um = _setup(L=2, depth=5, U=0.0, sigma=0.0, t=0.8)
    np.testing.assert_allclose(dense.cost(p, Um), -16.0, rtol=1e-14)


def test_single_gate_closed_form(rng):
    # n = 2 with one gate: F = Tr[U^dag G] so dF/dG = conj(U), gbar = -U,
    # grad = P_G(-U)
    p, Um = _setup(L=1, depth=3, t=0.7)  # A and B layers are empty for one site
    assert p.n_gates == 1
    np.testing.assert_allclose(dense.cost(p, Um), -np.trace(Um.conj().T @ p.gates[0]).real, rtol=1e-14)
    np.testing.assert_allclose(dense.holomorphic_env(p, Um)[0], Um.conj(), atol=1e-15)
    G = p.gates[0]
    ref = G @ (0.5 * (G.conj().T @ -Um - (G.conj().T @ -Um).conj().T))
    np.testing.assert_allclose(dense.rgrad(p, Um)[0], ref, atol=1e-15)


def _fd_euclid(p, Um, h=1e-6):
    out = np.zeros_like(p.gates)
    for q in range(p.n_params):
        for a in range(4):
            for b in range(4):
                for unit in (1.0, 1j):
                    gp = p.gates.copy(); gp[q, a, b] += h * unit
                    gm = p.gates.copy(); gm[q, a, b] -= h * unit
                    d = (dense.cost(p, Um, gp) - dense.cost(p, Um, gm)) / (2 * h)
                    out[q, a, b] += d * unit  # d_x f + i d_y f (Eq. def_grad)
    return out


@pytest.mark.parametrize("tied", [False, True])
def test_euclidean_gradient_vs_finite_differences(tied):
    p, Um = _setup(L=2, depth=4, tied=tied, seed=3)
    ref = _fd_euclid(p, Um)
    got = dense.euclid_gradient(p, Um)
    np.testing.assert_allclose(got, ref, atol=1e-7 * np.abs(ref).max())


def _tangent(p, seed, structure=None):
    structure = p.structure if structure is None else structure
    X = w.random_directions(p.n_params, 1, seed)[0]
    return riemann.tangent_direction(p.gates, X, structure)


@pytest.mark.parametrize("structure", [0, 1])
def test_riemannian_gradient_tangent_and_geodesic(structure):
    p, Um = _setup(L=2, depth=5, structure=structure, seed=4)
    g = dense.rgrad(p, Um)
    M = np.conj(np.swapaxes(p.gates, 1, 2)) @ g
    np.testing.assert_allclose(M, -np.conj(np.swapaxes(M, 1, 2)), atol=1e-13)
    if structure == 1:
        assert np.abs(g[:, ~riemann.PARITY_MASK]).max() == 0
    X = _tangent(p, 9)
    h = 1e-5
    d = (dense.cost(p, Um, riemann.geodesic(p.gates, X, h))
         - dense.cost(p, Um, riemann.geodesic(p.gates, X, -h))) / (2 * h)
    np.testing.assert_allclose(d, riemann.inner(g, X), rtol=1e-7, atol=1e-9)


def test_hessian_two_dense_routes_agree():
    p, Um = _setup(L=3, depth=3, seed=21)
    X = _tangent(p, 5)
    a = dense.holomorphic_env_dot(p, Um, X)
    b = dense.holomorphic_env_dot_cauchy(p, Um, X)
    np.testing.assert_allclose(a, b, atol=1e-12 * np.abs(a).max())


def test_same_gate_second_derivative_vanishes():
    # Sec. "Gradient and Hessian tensor diagrams": f is linear in each gate,
    # so the second derivative w.r.t. one (untied) gate is zero
    p, Um = _setup(L=2, depth=3, seed=8)
    X = np.zeros_like(p.gates)
    X[2] = _tangent(p, 3)[2]
    Ed = dense.holomorphic_env_dot_cauchy(p, Um, X)
    assert np.abs(Ed[2]).max() < 1e-13
    assert np.abs(Ed).max() > 1e-3


@pytest.mark.parametrize("structure,tied", [(0, False), (1, False), (0, True)])
def test_hessian_symmetric_tangent_linear(structure, tied):
    p, Um = _setup(L=2, depth=5, structure=structure, tied=tied, seed=13)
    X, Y = _tangent(p, 1), _tangent(p, 2)
    HX = dense.rhess(p, Um, X, method="cauchy")
    HY = dense.rhess(p, Um, Y, method="cauchy")
    np.testing.assert_allclose(riemann.inner(Y, HX), riemann.inner(HY, X), rtol=1e-11)
    M = np.conj(np.swapaxes(p.gates, 1, 2)) @ HX
    np.testing.assert_allclose(M, -np.conj(np.swapaxes(M, 1, 2)), atol=1e-12)
    H2 = dense.rhess(p, Um, 2.0 * X - 0.5 * Y, method="cauchy")
    np.testing.assert_allclose(H2, 2.0 * HX - 0.5 * HY, atol=1e-11)
    if structure == 1:
        assert np.abs(HX[:, ~riemann.PARITY_MASK]).max() == 0


@pytest.mark.parametrize("structure", [0, 1])
def test_hessian_geodesic_second_derivative(structure):
    p, Um = _setup(L=2, depth=5, structure=structure, seed=17)
    X = _tangent(p, 4)
    h = 1e-3
    f0 = dense.cost(p, Um)
    fp = dense.cost(p, Um, riemann.geodesic(p.gates, X, h))
    fm = dense.cost(p, Um, riemann.geodesic(p.gates, X, -h))
    d2 = (fp - 2 * f0 + fm) / h ** 2
    HX = dense.rhess(p, Um, X, method="pairs")
    np.testing.assert_allclose(d2, riemann.inner(HX, X), rtol=1e-5)


def test_hessian_is_projected_derivative_of_gradient_field():
    # Eq. vector_field_derivative: Hess[X] = P_G( d/de grad f(c(e)) ) along a
    # curve with c'(0) = X
    p, Um = _setup(L=2, depth=4, seed=19)
    X = _tangent(p, 6)
    h = 1e-5
    gp = dense.rgrad(p, Um, riemann.geodesic(p.gates, X, h))
    gm = dense.rgrad(p, Um, riemann.geodesic(p.gates, X, -h))
    fd = riemann.proj(p.gates, (gp - gm) / (2 * h))
    HX = dense.rhess(p, Um, X)
    np.testing.assert_allclose(fd, HX, atol=1e-7 * np.abs(HX).max())


def test_polar_retraction(rng):
    G = w.config_problem("small").gates[:3]
    np.testing.assert_allclose(riemann.retract(G, 0 * G), G, atol=1e-14)
    A = rng.standard_normal((3, 4, 4)) + 1j * rng.standard_normal((3, 4, 4))
    Q = riemann.polar_unitary(A)
    for i in range(3):
        np.testing.assert_allclose(Q[i].conj().T @ Q[i], np.eye(4), atol=1e-13)
        P = Q[i].conj().T @ A[i]  # Hermitian positive definite
        np.testing.assert_allclose(P, P.conj().T, atol=1e-12)
        assert np.linalg.eigvalsh(0.5 * (P + P.conj().T)).min() > 0


def test_fourth_order_trotter_initialisation():
    # 21 layers; the times of each kind add up to t; the noise-free circuit's
    # error ||C - U||_F^2 = 2 * 2^n + 2 f falls like t^10 (local error O(t^5))
    taus = w.trotter4_times(0.3)
    kinds = w.layer_pattern(21)
    assert len(taus) == 21
    for k in "ABC":
        np.testing.assert_allclose(sum(t for t, kk in zip(taus, kinds) if kk == k), 0.3, rtol=1e-14)
    errs = []
    for t in (0.2, 0.1):
        p, Um = _setup(L=3, depth=21, t=t, sigma=0.0)
        p = w.make_problem(3, 21, t, sigma=0.0, order=4)
        Um = model.target_unitary_dense(model.hamiltonian_dense(3, 1.0, 4.0), t)
        errs.append(2 * 2 ** p.n + 2 * dense.cost(p, Um))
        p2 = w.make_problem(3, 5, t, sigma=0.0)
        assert errs[-1] < 2 * 2 ** p.n + 2 * dense.cost(p2, Um)   # better than 2nd order
    assert 2 ** 9 < errs[0] / errs[1] < 2 ** 11
