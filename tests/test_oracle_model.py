"""Pins of the oracle's model layer against closed forms and library routines."""
import numpy as np
import pytest
import scipy.linalg
from math import comb

import workloads as w
from oracle import model


def _hloc(J, U):
    # two-site Hamiltonian printed in the paper (Sec. "Model system and
    # circuit topology", the matrix h_loc), local index 2*bit_a + bit_b
    h = np.zeros((4, 4))
    h[1, 2] = h[2, 1] = -J
    h[3, 3] = U
    return h


@pytest.mark.parametrize("tau", [0.0, 0.125, 0.37, 1.3])
def test_trotter_gate_closed_form(tau):
    # the paper's closed form for exp(-i t h_loc), split into its hopping
    # (U = 0) and on-site (J = 0) factors, against scipy's Pade expm
    J, U = 1.0, 4.0
    hop = w.trotter_gate("A", tau, J, U)
    ons = w.trotter_gate("C", tau, J, U)
    np.testing.assert_allclose(hop, scipy.linalg.expm(-1j * tau * _hloc(J, 0.0)), atol=1e-14)
    np.testing.assert_allclose(ons, scipy.linalg.expm(-1j * tau * _hloc(0.0, U)), atol=1e-14)
    # the full local gate of the paper: hop and on-site commute here
    np.testing.assert_allclose(hop @ ons, scipy.linalg.expm(-1j * tau * _hloc(J, U)), atol=1e-14)
    # it has the parity-conserving pattern of Eq. paritygatematrix
    assert np.all(np.abs(hop[~w.parity_mask()]) == 0)


def test_jw_strings_cancel_on_open_chain():
    # nearest-neighbour hops in the up-first ordering carry no Z string:
    # the JW-built H equals the one built from string-free local operators
    L, n = 3, 6
    H = model.hamiltonian_dense(L, 1.0, 4.0, periodic=False)
    Hb = np.zeros_like(H)
    for off in (0, L):
        for (i, k) in model.chain_bonds(L, False):
            ai = model.hardcore_annihilator(off + i, n)
            ak = model.hardcore_annihilator(off + k, n)
            Hb += -(ai.T @ ak + ak.T @ ai)
    for j in range(L):
        nu = model.hardcore_annihilator(j, n)
        nd = model.hardcore_annihilator(L + j, n)
        Hb += 4.0 * (nu.T @ nu) @ (nd.T @ nd)
    np.testing.assert_array_equal(H, Hb)


def test_jw_anticommutation():
    n = 4
    for i in range(n):
        for k in range(n):
            ai, ak = model.jw_annihilator(i, n), model.jw_annihilator(k, n)
            anti = ai @ ak.T + ak.T @ ai
            np.testing.assert_array_equal(anti, np.eye(1 << n) * (i == k))
            np.testing.assert_array_equal(ai @ ak + ak @ ai, 0 * anti)


@pytest.mark.parametrize("periodic", [False, True])
def test_hamiltonian_symmetries(periodic):
    L, n = 3, 6
    H = model.hamiltonian_dense(L, 1.0, 4.0, periodic)
    np.testing.assert_array_equal(H, H.T)
    xs = np.arange(1 << n)
    Nup = np.diag(sum(model.bit(xs, q, n) for q in range(L)).astype(float))
    Ndn = np.diag(sum(model.bit(xs, q, n) for q in range(L, n)).astype(float))
    assert np.abs(H @ Nup - Nup @ H).max() == 0
    assert np.abs(H @ Ndn - Ndn @ H).max() == 0


def test_half_filling_single_site():
    # one site (n = 2): H = U n_up n_dn; U = exp(-iHt) = diag(1, 1, 1, e^{-iUt})
    H = model.hamiltonian_dense(1, 1.0, 4.0)
    np.testing.assert_array_equal(H, np.diag([0.0, 0.0, 0.0, 4.0]))
    U = model.target_unitary_dense(H, 0.3)
    np.testing.assert_allclose(U, np.diag([1, 1, 1, np.exp(-1.2j)]), atol=1e-15)


@pytest.mark.parametrize("L,periodic", [(2, False), (3, False), (3, True), (4, False)])
def test_sector_hamiltonian_matches_dense(L, periodic):
    H = model.hamiltonian_dense(L, 1.0, 4.0, periodic)
    total = 0
    for a in range(L + 1):
        for b in range(L + 1):
            Hs, basis = model.hamiltonian_sector(L, 1.0, 4.0, periodic, (a, b))
            assert len(basis) == comb(L, a) * comb(L, b) == model.sector_size(L, (a, b))
            np.testing.assert_array_equal(Hs, H[np.ix_(basis, basis)])
            total += len(basis)
    assert total == 1 << (2 * L)


def test_target_unitary_vs_pade():
    L, t = 3, 0.5
    H = model.hamiltonian_dense(L, 1.0, 4.0)
    U = model.target_unitary_dense(H, t)
    np.testing.assert_allclose(U.conj().T @ U, np.eye(64), atol=1e-13)
    np.testing.assert_allclose(U, scipy.linalg.expm(-1j * t * H), atol=1e-13)


@pytest.mark.parametrize("L,t,periodic", [(3, 0.5, False), (4, 0.25, False), (3, 0.9, True)])
def test_sector_target_equals_dense(L, t, periodic):
    H = model.hamiltonian_dense(L, 1.0, 4.0, periodic)
    U = model.target_unitary_dense(H, t)
    st = model.SectorTarget(L, 1.0, 4.0, t, periodic)
    cols = np.arange(1 << (2 * L))
    np.testing.assert_allclose(st.columns(cols).T, U, atol=1e-13)


def test_memory_of_sixteen_qubit_state():
    # Sec. "Memory considerations for 16 qubits": one complex128 state of
    # 16 qubits is exactly 1 MiB; a dense layer would be 64 GiB.
    assert (1 << 16) * 16 == 1 << 20
    assert 16 * (1 << 16) ** 2 == 64 << 30


# ------------------------------------------------------------ spinless chain

@pytest.mark.parametrize("tau", [0.1, 0.77])
def test_spinless_trotter_gate_is_the_printed_closed_form(tau):
    # the full two-site Hamiltonian h_loc of the spinless chain (hop + U n n)
    J, U = 1.0, 2.5
    np.testing.assert_allclose(w.spinless_gate(tau, J, U), scipy.linalg.expm(-1j * tau * _hloc(J, U)), atol=1e-14)


@pytest.mark.parametrize("L,periodic", [(4, False), (5, True), (6, True)])
def test_spinless_hamiltonian(L, periodic):
    H = model.hamiltonian_dense(L, 1.0, 2.0, periodic, model=1)
    np.testing.assert_array_equal(H, H.T)
    xs = np.arange(1 << L)
    N = np.diag(np.array([bin(x).count("1") for x in xs], dtype=float))
    assert np.abs(H @ N - N @ H).max() == 0
    total = 0
    for Nn in range(L + 1):
        Hs, basis = model.hamiltonian_sector(L, 1.0, 2.0, periodic, (Nn,), model=1)
        np.testing.assert_array_equal(Hs, H[np.ix_(basis, basis)])
        total += len(basis)
    assert total == 1 << L
    # one particle on a periodic ring: hopping band -2J cos(k)
    if periodic:
        Hs, _ = model.hamiltonian_sector(L, 1.0, 2.0, True, (1,), model=1)
        k = 2 * np.pi * np.arange(L) / L
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(Hs)), np.sort(-2 * np.cos(k)), atol=1e-12)


def test_spinless_sector_target_equals_dense():
    H = model.hamiltonian_dense(6, 1.0, 2.0, True, model=1)
    U = model.target_unitary_dense(H, 0.7)
    st = model.SectorTarget(6, 1.0, 2.0, 0.7, True, model=1)
    np.testing.assert_allclose(st.columns(np.arange(64)).T, U, atol=1e-13)
