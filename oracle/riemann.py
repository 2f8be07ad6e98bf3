"""Riemannian geometry of U(4)^{x g} (oracle; test infrastructure).

Paper Sec. "Riemannian optimization":
* tangent space ``T_V U = {V A : A^dagger = -A}`` (Eq. tangent_space_param),
  metric ``<X, Y> = Re Tr[X^dagger Y]`` summed over gates;
* projection ``P_V X = V skew(V^dagger X)`` (Eq. proj_tangent);
* gradient convention ``grad f(z) = d_x f + i d_y f`` (Eq. def_grad); for the
  cost ``f = -Re F`` with ``F`` holomorphic in the gate entries this is
  ``-conj(dF/dG)`` entry-wise;
* ``grad f(V) = P_V grad fbar(V)`` (Eq. grad_proj);
* ``Hess f(G)[X] = P_G(D xi(G)[X])`` with ``xi = grad f`` (Eq.
  vector_field_derivative, Eq. hessian_def) -- written out here by the
  product rule on ``xi(V) = V skew(V^dagger gbar(V))``, not simplified;
* polar retraction ``R_V(xi) = qpolar(V + xi)`` (Eq. retraction_qr);
* tied gates: ``dG_l = sum_i dG_{l,i}`` (Sec. "Brick wall circuit layout");
* parity-conserving gates (Eq. paritygatematrix): the cost is restricted to
  the patterned subspace, so Euclidean derivatives are masked to the pattern.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

_PAR = np.array([0, 1, 1, 0])
PARITY_MASK = (_PAR[:, None] == _PAR[None, :])


def dag(A):
    return np.swapaxes(A, -1, -2).conj()


def skew(A):
    return 0.5 * (A - dag(A))


def sym(A):
    return 0.5 * (A + dag(A))


def proj(V, X):
    """Eq. proj_tangent, batched over leading axes."""
    return V @ skew(dag(V) @ X)


def inner(X, Y) -> float:
    """``sum Re Tr[X^dagger Y]`` over all gates."""
    return float(np.sum((np.conj(X) * Y).real))


def euclid_from_holomorphic(dF):
    """Eq. def_grad applied to ``f = -Re F``: ``grad fbar = -conj(dF/dG)``."""
    return -np.conj(dF)


def tie(per_gate, param_of, n_params):
    """Accumulate per-gate quantities into their parameter gates."""
    out = np.zeros((n_params,) + per_gate.shape[1:], dtype=per_gate.dtype)
    for l, p in enumerate(param_of):
        out[p] += per_gate[l]
    return out


def mask(X, structure: int):
    return X * PARITY_MASK if structure == 1 else X


def tangent_direction(G, Xraw, structure: int):
    """Raw direction -> tangent vector (projection, then the parity pattern)."""
    return mask(proj(G, Xraw), structure)


def riemannian_gradient(G, gbar, structure: int = 0):
    return proj(G, mask(gbar, structure))


def riemannian_hessian(G, gbar, Dgbar, X, structure: int = 0):
    """``P_G( D[V -> P_V gbar(V)](G)[X] )`` by the product rule.

    ``D[V skew(V^dag gbar(V))][X] = X skew(G^dag gbar)
                                   + G skew(X^dag gbar + G^dag Dgbar[X])``.
    """
    gb = mask(gbar, structure)
    dgb = mask(Dgbar, structure)
    dxi = X @ skew(dag(G) @ gb) + G @ skew(dag(X) @ gb + dag(G) @ dgb)
    return proj(G, dxi)


def polar_unitary(A):
    """Unitary factor of the polar decomposition (Eq. retraction_qr)."""
    out = np.empty_like(A)
    for i in range(A.shape[0]):
        out[i] = scipy.linalg.polar(A[i])[0]
    return out


def retract(G, xi):
    return polar_unitary(G + xi)


def geodesic(G, X, eps):
    """``G expm(eps G^dag X)``: for the embedded Euclidean metric on U(m),
    which is bi-invariant, these curves are geodesics through ``G`` with
    velocity ``X``."""
    out = np.empty_like(G)
    for i in range(G.shape[0]):
        out[i] = G[i] @ scipy.linalg.expm(eps * (G[i].conj().T @ X[i]))
    return out
