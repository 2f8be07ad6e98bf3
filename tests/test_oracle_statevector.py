"""O2 (the paper's matrix-free recursion) against O1 (dense definitions)."""
import numpy as np
import pytest

import workloads as w
from oracle import dense, model, riemann, statevector as sv


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("L,depth,structure,tied", [
    (2, 5, 0, False), (3, 5, 0, False), (3, 4, 1, False), (3, 6, 0, True), (3, 5, 1, True)])
def test_matrix_free_equals_dense(L, depth, structure, tied):
    p = w.make_problem(L, depth, 0.45, seed=31 + L, structure=structure, tied=tied)
    Um = model.target_unitary_dense(model.hamiltonian_dense(L, 1.0, 4.0), 0.45)
    st = model.SectorTarget(L, 1.0, 4.0, 0.45)
    Xraw = w.random_directions(p.n_params, 2, 77)
    f, g, hv, Xt = sv.cost_grad_hvp(p, st, range(1 << p.n), Xraw)
    assert abs(f - dense.cost(p, Um)) <= 1e-13 * 2 ** p.n
    assert _rel(g, dense.rgrad(p, Um)) < 1e-12
    for i in range(2):
        ref = dense.rhess(p, Um, Xt[i], method="cauchy" if L > 2 else "pairs")
        assert _rel(hv[i], ref) < 1e-11


def test_full_basis_sum_n8_against_dense():
    p = w.config_problem("small")
    Um = model.target_unitary_dense(model.hamiltonian_dense(4, 1.0, 4.0), 0.25)
    st = model.SectorTarget(4, 1.0, 4.0, 0.25)
    F, dF, _ = sv.evaluate(p, st, range(256), chunk=64)
    assert abs(-F.real - dense.cost(p, Um)) < 1e-11
    assert _rel(dF, dense.holomorphic_env(p, Um)) < 1e-12


def test_column_additivity():
    p = w.make_problem(3, 5, 0.5, seed=3)
    st = model.SectorTarget(3, 1.0, 4.0, 0.5)
    X = w.random_directions(p.n_params, 1, 4)
    cols = np.arange(64)
    a = sv.cost_grad_hvp(p, st, cols[:23], X)
    b = sv.cost_grad_hvp(p, st, cols[23:], X)
    c = sv.cost_grad_hvp(p, st, cols, X)
    np.testing.assert_allclose(a[0] + b[0], c[0], rtol=1e-13)
    np.testing.assert_allclose(a[1] + b[1], c[1], atol=1e-13)
    np.testing.assert_allclose(a[2] + b[2], c[2], atol=1e-12)


def test_parity_columns_stay_in_sector():
    # parity-conserving gates keep every column in its parity sector
    p = w.make_problem(3, 5, 0.5, seed=9, structure=1)
    mats = p.gates[p.param_of]
    psi = np.zeros((1, 64), dtype=np.complex128)
    psi[0, 0b000101] = 1.0
    for l in range(p.n_gates):
        psi = sv.apply_gate(mats[l], p.pairs[l], psi, 6)
    par = np.array([bin(x).count("1") & 1 for x in range(64)])
    assert np.abs(psi[0, par == 1]).max() < 1e-300 or np.abs(psi[0, par == 1]).max() == 0
    assert abs(np.linalg.norm(psi) - 1) < 1e-14


def test_gate_application_and_hole_match_dense_embedding(rng):
    # every ordered qubit pair, including pairs listed high-to-low
    n = 4
    G = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    psi = rng.standard_normal((3, 16)) + 1j * rng.standard_normal((3, 16))
    phi = rng.standard_normal((3, 16)) + 1j * rng.standard_normal((3, 16))
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            E = dense.embed(G, (a, b), n)
            np.testing.assert_allclose(sv.apply_gate(G, (a, b), psi, n), psi @ E.T, atol=1e-14)
            h = sv.hole(phi, psi, (a, b), n)
            for x in range(4):
                for y in range(4):
                    e = np.zeros((4, 4)); e[x, y] = 1.0
                    ref = np.sum(phi * (psi @ dense.embed(e, (a, b), n).T))
                    assert abs(h[x, y] - ref) < 1e-13


def test_periodic_wrap_bond_matches_dense():
    # the periodic chain lists its wrap bond high-to-low: (L-1, 0)
    L = 4
    p = w.make_problem(L, 4, 0.3, seed=41, periodic=True)
    assert any(a > b for a, b in p.pairs.tolist())
    Um = model.target_unitary_dense(model.hamiltonian_dense(L, 1.0, 4.0, True), 0.3)
    st = model.SectorTarget(L, 1.0, 4.0, 0.3, True)
    Xraw = w.random_directions(p.n_params, 1, 5)
    f, g, hv, Xt = sv.cost_grad_hvp(p, st, range(1 << p.n), Xraw, chunk=64)
    assert abs(f - dense.cost(p, Um)) <= 1e-13 * 2 ** p.n
    assert _rel(g, dense.rgrad(p, Um)) < 1e-12
    assert _rel(hv[0], dense.rhess(p, Um, Xt[0], method="cauchy")) < 1e-11


@pytest.mark.parametrize("structure,tied,periodic", [(0, False, False), (1, True, True), (0, True, True)])
def test_spinless_matrix_free_equals_dense(structure, tied, periodic):
    p = w.make_spinless_problem(6, 5, 0.6, U=2.0, seed=71, structure=structure, tied=tied, periodic=periodic)
    assert p.n == 6
    Um = model.target_unitary_dense(model.hamiltonian_dense(6, 1.0, 2.0, periodic, model=1), 0.6)
    st = model.SectorTarget(6, 1.0, 2.0, 0.6, periodic, model=1)
    Xraw = w.random_directions(p.n_params, 1, 72)
    f, g, hv, Xt = sv.cost_grad_hvp(p, st, range(64), Xraw, chunk=64)
    assert abs(f - dense.cost(p, Um)) <= 1e-13 * 64
    assert _rel(g, dense.rgrad(p, Um)) < 1e-12
    assert _rel(hv[0], dense.rhess(p, Um, Xt[0], method="cauchy")) < 1e-11
