"""Fermi-Hubbard Hamiltonians and the target unitary (oracle; test infrastructure).

Paper Sec. "Model system and circuit topology": Jordan-Wigner operators
``a_j -> I x ... x I x c x Z x ... x Z`` (j identities first, qubit 0 the
first tensor factor = most significant bit), local ``c = [[0,1],[0,0]]``;
spinful chain Eq. sfFH with all spin-up sites first (qubit j = site j up,
qubit L+j = site j down).  The periodic wrap bond drops its Z string
(hard-core boson mapping, Eq. slFH_qubit), as the paper does.

The target is ``U = exp(-i H t)`` (Eq. f_target).  ``H`` is real symmetric, so
``U = V diag(exp(-i w t)) V^T`` from ``eigh`` is the exact exponential up to
rounding.  ``H`` conserves the spin-resolved particle numbers, so the same
``U`` is also assembled from per-sector blocks for sizes where a dense
``2^n x 2^n`` matrix is out of reach.
"""
from __future__ import annotations

import functools
from math import comb
from typing import Dict, Iterable, List, Tuple

import numpy as np

_C = np.array([[0.0, 1.0], [0.0, 0.0]])  # annihilates |1>
_Z = np.diag([1.0, -1.0])
_I = np.eye(2)


def _kron_all(ops: Iterable[np.ndarray]) -> np.ndarray:
    return functools.reduce(np.kron, ops)


def jw_annihilator(j: int, n: int) -> np.ndarray:
    """Dense Jordan-Wigner annihilator ``a_j`` on ``n`` qubits."""
    return _kron_all([_I] * j + [_C] + [_Z] * (n - j - 1))


def hardcore_annihilator(j: int, n: int) -> np.ndarray:
    """Local ``c_j`` with no string (hard-core boson)."""
    return _kron_all([_I] * j + [_C] + [_I] * (n - j - 1))


def chain_bonds(L: int, periodic: bool) -> List[Tuple[int, int]]:
    bonds = [(j, j + 1) for j in range(L - 1)]
    if periodic and L > 2:
        bonds.append((L - 1, 0))
    return bonds


def hamiltonian_dense(L: int, J: float, U: float, periodic: bool = False, model: int = 0) -> np.ndarray:
    """Dense real matrix built term by term: Eq. sfFH (model 0, n = 2L) or
    the spinless chain of Sec. "Model system and circuit topology" with its
    wrap bond in hard-core boson form, Eq. slFH_qubit (model 1, n = L)."""
    if model == 1:
        return _hamiltonian_dense_spinless(L, J, U, periodic)
    n = 2 * L
    dim = 1 << n
    H = np.zeros((dim, dim))
    for off in (0, L):  # spin up chain, spin down chain
        for (i, k) in chain_bonds(L, periodic):
            wrap = periodic and (i, k) == (L - 1, 0)
            op = hardcore_annihilator if wrap else jw_annihilator
            ai, ak = op(off + i, n), op(off + k, n)
            H += -J * (ai.T @ ak + ak.T @ ai)
    for j in range(L):
        nu = jw_annihilator(j, n)
        nd = jw_annihilator(L + j, n)
        H += U * (nu.T @ nu) @ (nd.T @ nd)
    return H


def _hamiltonian_dense_spinless(L: int, J: float, U: float, periodic: bool) -> np.ndarray:
    n = L
    H = np.zeros((1 << n, 1 << n))
    for (i, k) in chain_bonds(L, periodic):
        wrap = periodic and (i, k) == (L - 1, 0)
        op = hardcore_annihilator if wrap else jw_annihilator
        ai, ak = op(i, n), op(k, n)
        H += -J * (ai.T @ ak + ak.T @ ai)
        ni = jw_annihilator(i, n)
        nk = jw_annihilator(k, n)
        H += U * (ni.T @ ni) @ (nk.T @ nk)
    return H


def target_unitary_dense(H: np.ndarray, t: float) -> np.ndarray:
    """``exp(-i H t)`` for real symmetric ``H`` via its eigendecomposition."""
    w, V = np.linalg.eigh(H)
    return (V * np.exp(-1j * w * t)) @ V.T


# Particle-number sectors ----------------------------------------------------

def bit(x, q: int, n: int):
    """Bit of qubit ``q`` (qubit 0 = most significant) of index ``x``."""
    return (x >> (n - 1 - q)) & 1


def sector_label(x: int, L: int, model: int = 0):
    """``(N_up, N_down)`` of basis state ``x`` (model 1: ``(N,)``)."""
    if model == 1:
        return (bin(int(x)).count("1"),)
    n = 2 * L
    up = sum(bit(x, q, n) for q in range(L))
    dn = sum(bit(x, q, n) for q in range(L, n))
    return up, dn


def sector_basis(L: int, label, model: int = 0) -> np.ndarray:
    """Ascending basis indices of one sector."""
    if model == 1:
        xs = np.arange(1 << L)
        return xs[np.array([bin(int(x)).count("1") for x in xs]) == label[0]]
    n = 2 * L
    xs = np.arange(1 << n)
    up = sum(bit(xs, q, n) for q in range(L))
    dn = sum(bit(xs, q, n) for q in range(L, n))
    return xs[(up == label[0]) & (dn == label[1])]


def sector_size(L: int, label: Tuple[int, int]) -> int:
    return comb(L, label[0]) * comb(L, label[1])


def hamiltonian_sector(L: int, J: float, U: float, periodic: bool,
                       label, model: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Matrix of Eq. sfFH on one sector, from its action on basis states.

    A hop along a bond ``(p, q)`` of one spin chain exchanges an occupied and
    an empty orbital with amplitude ``-J`` (no sign: nearest neighbours in the
    up-first ordering carry no Z string, the wrap bond is hard-core); the
    diagonal is ``U`` times the number of doubly occupied sites.
    """
    if model == 1:
        return _hamiltonian_sector_spinless(L, J, U, periodic, label)
    n = 2 * L
    basis = sector_basis(L, label)
    pos = {int(x): i for i, x in enumerate(basis)}
    H = np.zeros((len(basis), len(basis)))
    for i, x in enumerate(basis):
        x = int(x)
        H[i, i] = U * sum(bit(x, j, n) & bit(x, L + j, n) for j in range(L))
        for off in (0, L):
            for (p, q) in chain_bonds(L, periodic):
                if bit(x, off + p, n) != bit(x, off + q, n):
                    y = x ^ (1 << (n - 1 - off - p)) ^ (1 << (n - 1 - off - q))
                    H[pos[y], i] += -J
    return H, basis


def _hamiltonian_sector_spinless(L, J, U, periodic, label):
    """Spinless chain on one particle-number sector: a hop along a bond
    exchanges an occupied and an empty site with amplitude -J; the diagonal is
    U times the number of bonds with both sites occupied."""
    n = L
    basis = sector_basis(L, label, model=1)
    pos = {int(x): i for i, x in enumerate(basis)}
    H = np.zeros((len(basis), len(basis)))
    for i, x in enumerate(basis):
        x = int(x)
        for (p, q) in chain_bonds(L, periodic):
            bp, bq = bit(x, p, n), bit(x, q, n)
            if bp and bq:
                H[i, i] += U
            elif bp != bq:
                y = x ^ (1 << (n - 1 - p)) ^ (1 << (n - 1 - q))
                H[pos[y], i] += -J
    return H, basis


class SectorTarget:
    """``U = exp(-iHt)`` columns, assembled from per-sector eigendecompositions.

    ``column(j)`` returns ``U |j>`` as a dense vector of length ``2^n``; the
    sector blocks are computed on first use and cached.
    """

    def __init__(self, L: int, J: float, U: float, t: float, periodic: bool = False, model: int = 0):
        self.L, self.J, self.U, self.t, self.periodic, self.model = L, J, U, t, periodic, model
        self.n = 2 * L if model == 0 else L
        self._blocks: Dict[Tuple[int, int], Tuple[np.ndarray, Dict[int, int], np.ndarray]] = {}

    def block(self, label):
        if label not in self._blocks:
            H, basis = hamiltonian_sector(self.L, self.J, self.U, self.periodic, label, self.model)
            Us = target_unitary_dense(H, self.t)
            self._blocks[label] = (basis, {int(x): i for i, x in enumerate(basis)}, Us)
        return self._blocks[label]

    def column(self, j: int) -> np.ndarray:
        basis, pos, Us = self.block(sector_label(int(j), self.L, self.model))
        v = np.zeros(1 << self.n, dtype=np.complex128)
        v[basis] = Us[:, pos[int(j)]]
        return v

    def columns(self, cols) -> np.ndarray:
        return np.stack([self.column(j) for j in cols]) if len(cols) else \
            np.zeros((0, 1 << self.n), dtype=np.complex128)
