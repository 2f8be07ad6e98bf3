"""O1: plain dense definitions (oracle; test infrastructure).

With ``W = emb(G_g) ... emb(G_1)`` (Sec. "Quantum circuits": the gate applied
first stands on the right) and ``U`` the target:

* ``f = -Re Tr[U^dagger W]`` (Eq. f_target);
* ``F = Tr[U^dagger W]`` is linear in each gate, so with
  ``W = A_l emb(G_l) B_l`` its derivative is
  ``dF/dG_l[a, b] = Tr[U^dagger A_l emb(e_ab) B_l]`` (the "gate hole",
  Fig. network_gradient_hole);
* the second derivative w.r.t. two distinct gates puts two holes in the
  network (Fig. network_hessian_holes); along a direction ``X`` it is
  ``sum_{l' != l}`` of the network with ``G_l -> e_ab`` and ``G_l' -> X_l'``
  (same-gate blocks vanish because ``F`` is linear in each gate).

``emb`` places a 4x4 gate on the listed qubit pair ``(a, b)`` with local
index ``2 bit_a + bit_b`` (qubit 0 = most significant bit), Eq.
gate_application_neighboring and its general form.  Everything here is
``O(4^n)`` memory: use it for ``n <= 10``.
"""
from __future__ import annotations

import numpy as np

from . import riemann


def _local_and_rest(n: int, pair):
    a, b = int(pair[0]), int(pair[1])
    xs = np.arange(1 << n)
    ba = (xs >> (n - 1 - a)) & 1
    bb = (xs >> (n - 1 - b)) & 1
    local = 2 * ba + bb
    rest = xs & ~((1 << (n - 1 - a)) | (1 << (n - 1 - b)))
    return local, rest


def embed(G: np.ndarray, pair, n: int) -> np.ndarray:
    """Dense ``2^n x 2^n`` matrix of a two-qubit gate on ``pair``."""
    local, rest = _local_and_rest(n, pair)
    return G[local[:, None], local[None, :]] * (rest[:, None] == rest[None, :])


def circuit_matrix(gates_per_gate, pairs, n: int) -> np.ndarray:
    W = np.eye(1 << n, dtype=np.complex128)
    for G, p in zip(gates_per_gate, pairs):
        W = embed(G, p, n) @ W
    return W


def expand(prob, gates=None):
    """Per-gate matrices ``G_l = gates[param_of[l]]``."""
    gates = prob.gates if gates is None else gates
    return gates[prob.param_of]


def cost(prob, Umat, gates=None) -> float:
    W = circuit_matrix(expand(prob, gates), prob.pairs, prob.n)
    return float(-np.trace(Umat.conj().T @ W).real)


def _hole_network(mats, pairs, n, l, Umat):
    """``dF/dG_l`` for the gate list ``mats`` (the network with a hole at l)."""
    dim = 1 << n
    B = np.eye(dim, dtype=np.complex128)
    for m in range(l):
        B = embed(mats[m], pairs[m], n) @ B
    A = np.eye(dim, dtype=np.complex128)
    for m in range(l + 1, len(mats)):
        A = embed(mats[m], pairs[m], n) @ A
    M = B @ Umat.conj().T @ A  # Tr[U^dag A emb(e_ab) B] = sum_{x,y} M[y,x] emb(e_ab)[x,y]
    out = np.zeros((4, 4), dtype=np.complex128)
    for a in range(4):
        for b in range(4):
            e = np.zeros((4, 4))
            e[a, b] = 1.0
            out[a, b] = np.sum(M.T * embed(e, pairs[l], n))
    return out


def holomorphic_env(prob, Umat, gates=None) -> np.ndarray:
    """``dF/dG_l`` for every sequential gate ``l`` -> ``[g, 4, 4]``."""
    mats = expand(prob, gates)
    return np.stack([_hole_network(mats, prob.pairs, prob.n, l, Umat)
                     for l in range(prob.n_gates)])


def holomorphic_env_dot(prob, Umat, Xdirs, gates=None) -> np.ndarray:
    """Second derivative along ``X``: ``sum_{l' != l} d2F/dG_l dG_l' . X_l'``.

    Written as the two-hole network sum: for every ``l' != l`` the network
    with ``G_l'`` replaced by ``X_l'`` and a hole at ``l``.  ``Xdirs`` holds
    one direction per parameter gate.  ``O(g^2)`` dense networks: ``n <= 6``.
    """
    mats = expand(prob, gates)
    Xs = Xdirs[prob.param_of]
    out = np.zeros((prob.n_gates, 4, 4), dtype=np.complex128)
    for l in range(prob.n_gates):
        for lp in range(prob.n_gates):
            if lp == l:
                continue
            sub = mats.copy()
            sub[lp] = Xs[lp]
            out[l] += _hole_network(sub, prob.pairs, prob.n, l, Umat)
    return out


def holomorphic_env_dot_cauchy(prob, Umat, Xdirs, gates=None, radius: float = 1.0):
    """Second derivative along ``X`` from the polynomial ``eps -> dF/dG_l(G + eps X)``.

    ``dF/dG_l`` is a polynomial of degree ``<= g - 1`` in ``eps``, so its
    linear coefficient is exactly ``(1 / (M r)) sum_k p(r w^k) w^{-k}`` for
    ``M > g - 1`` points on a circle (discrete Cauchy formula).  An
    independent route to :func:`holomorphic_env_dot` for ``n <= 8``.
    """
    gates = prob.gates if gates is None else gates
    M = prob.n_gates + 1
    acc = np.zeros((prob.n_gates, 4, 4), dtype=np.complex128)
    for k in range(M):
        w = np.exp(2j * np.pi * k / M)
        acc += holomorphic_env(prob, Umat, gates + radius * w * Xdirs) * np.conj(w)
    return acc / (M * radius)


def euclid_gradient(prob, Umat, gates=None):
    """Euclidean gradient per parameter gate (tied sums), unmasked."""
    E = holomorphic_env(prob, Umat, gates)
    return riemann.tie(riemann.euclid_from_holomorphic(E), prob.param_of, prob.n_params)


def rgrad(prob, Umat, gates=None):
    gates = prob.gates if gates is None else gates
    return riemann.riemannian_gradient(gates, euclid_gradient(prob, Umat, gates), prob.structure)


def rhess(prob, Umat, Xtan, gates=None, method: str = "pairs"):
    """Riemannian Hessian applied to the tangent direction ``Xtan``."""
    gates = prob.gates if gates is None else gates
    gbar = euclid_gradient(prob, Umat, gates)
    if method == "pairs":
        Ed = holomorphic_env_dot(prob, Umat, Xtan, gates)
    else:
        Ed = holomorphic_env_dot_cauchy(prob, Umat, Xtan, gates)
    Dgbar = riemann.tie(riemann.euclid_from_holomorphic(Ed), prob.param_of, prob.n_params)
    return riemann.riemannian_hessian(gates, gbar, Dgbar, Xtan, prob.structure)
