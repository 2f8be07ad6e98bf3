"""O2: the paper's matrix-free algorithm over basis columns (oracle; test infrastructure).

Follows Sec. "Optimized circuit contraction and derivative computation" and
Appendix "Evaluating Hessian-vector products", one basis summand at a time
(vectorised over a small stack of columns, each column independent):

* summand ``j``: ``psi_0 = |j>`` and ``phi_0 = (U|j>)^*`` (the paper keeps
  ``phi`` unconjugated in the diagram), so the summand is ``phi_0^T C(G) psi_0``
  (Eq. f_target_sum_unit_vec);
* forward pass caching ``psi_l = G_l psi_{l-1}`` (Fig. forward_pass), gate
  application by Eq. gate_application_neighboring / its general 5-leg form;
* backward pass with the transposed gates, ``phi_k = G_{g-k+1}^T phi_{k-1}``,
  and the gate-hole contraction ``dG_l = sum y (x) x`` of ``phi_{g-l}`` with
  ``psi_{l-1}`` on the fly (Fig. backward_pass_gate_gradient, Fig.
  hole_contraction);
* Hessian-vector product along ``Z``: forward-mode for the directed gradient
  ``sum_l phi_{g-l}^T Z_l psi_{l-1}`` (Fig. directed_gradient_graph), i.e.
  ``psi'_l = G_l psi'_{l-1} + Z_l psi_{l-1}``, then a reverse pass over that
  graph, each branching summed: the cotangent of ``psi_l`` obeys
  ``phid_{l-1} = G_l^T phid_l + Z_l^T phi_l`` and
  ``d/dG_l = hole(phid, psi_{l-1}) + hole(phi, psi'_{l-1})``.

All results are complex holomorphic derivatives of ``F = sum_j phi_0^T C psi_0``;
``riemann`` turns them into the Riemannian quantities.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

from . import riemann


def _legs(n: int, pair):
    """Reshape sizes for the 5-leg view (i0, j_lo, i2, j_hi, i4)."""
    a, b = int(pair[0]), int(pair[1])
    lo, hi = min(a, b), max(a, b)
    return (1 << lo, 2, 1 << (hi - lo - 1), 2, 1 << (n - hi - 1)), a < b


def apply_gate(G: np.ndarray, pair, psi: np.ndarray, n: int) -> np.ndarray:
    """``psi'[.., i_a, .., i_b, ..] = sum g[i_a i_b, j_a j_b] psi[.., j_a, .., j_b, ..]``.

    ``psi`` has shape ``[columns, 2^n]``; ``G[2 i_a + i_b, 2 j_a + j_b]``.
    """
    shape, a_first = _legs(n, pair)
    g4 = G.reshape(2, 2, 2, 2)
    v = psi.reshape((psi.shape[0],) + shape)
    if a_first:
        out = np.einsum("xyuv,cAuBvD->cAxByD", g4, v)
    else:
        out = np.einsum("xyuv,cAvBuD->cAyBxD", g4, v)
    return out.reshape(psi.shape)


def hole(phi: np.ndarray, psi: np.ndarray, pair, n: int) -> np.ndarray:
    """Gate-hole contraction summed over columns: ``dG[a, b] = sum phi[a, rest] psi[b, rest]``."""
    shape, a_first = _legs(n, pair)
    y = phi.reshape((phi.shape[0],) + shape)
    x = psi.reshape((psi.shape[0],) + shape)
    if a_first:
        d = np.einsum("cAxByD,cAuBvD->xyuv", y, x)
    else:
        d = np.einsum("cAyBxD,cAvBuD->xyuv", y, x)
    return d.reshape(4, 4)


def evaluate(prob, target, cols: Sequence[int], Xdirs: Optional[np.ndarray] = None,
             gates: Optional[np.ndarray] = None, chunk: int = 8):
    """Sum over the basis columns ``cols`` of the cost and its derivatives.

    Returns ``(F, dF, dFdot)``: ``F = sum_j phi_0^T C psi_0`` (complex),
    ``dF[l] = dF/dG_l`` (``[g, 4, 4]``) and, for each direction ``Z`` in
    ``Xdirs`` (``[k, n_params, 4, 4]``, tied per ``param_of``), the directed
    second derivative ``dFdot[i, l]``.  ``target.columns(js)`` gives ``U|j>``.
    """
    gates = prob.gates if gates is None else gates
    n, g = prob.n, prob.n_gates
    mats = gates[prob.param_of]
    k = 0 if Xdirs is None else Xdirs.shape[0]
    Zs = None if k == 0 else Xdirs[:, prob.param_of]
    F = 0.0 + 0.0j
    dF = np.zeros((g, 4, 4), dtype=np.complex128)
    dFdot = np.zeros((k, g, 4, 4), dtype=np.complex128)
    cols = list(cols)
    for c0 in range(0, len(cols), chunk):
        js = cols[c0:c0 + chunk]
        nc = len(js)
        psi = np.zeros((nc, 1 << n), dtype=np.complex128)
        psi[np.arange(nc), js] = 1.0
        # forward pass, caching every intermediate state
        cache = [psi]
        for l in range(g):
            cache.append(apply_gate(mats[l], prob.pairs[l], cache[-1], n))
        tcache = []
        for i in range(k):
            pd = [np.zeros_like(psi)]
            for l in range(g):
                pd.append(apply_gate(mats[l], prob.pairs[l], pd[-1], n)
                          + apply_gate(Zs[i, l], prob.pairs[l], cache[l], n))
            tcache.append(pd)
        phi = np.conj(target.columns(js))
        F += np.sum(phi * cache[g])
        # backward pass with transposed gates; holes on the fly
        phid = [np.zeros_like(phi) for _ in range(k)]
        for l in range(g - 1, -1, -1):
            dF[l] += hole(phi, cache[l], prob.pairs[l], n)
            for i in range(k):
                dFdot[i, l] += hole(phid[i], cache[l], prob.pairs[l], n) \
                    + hole(phi, tcache[i][l], prob.pairs[l], n)
                phid[i] = apply_gate(mats[l].T, prob.pairs[l], phid[i], n) \
                    + apply_gate(Zs[i, l].T, prob.pairs[l], phi, n)
            phi = apply_gate(mats[l].T, prob.pairs[l], phi, n)
    return F, dF, dFdot


def cost_grad_hvp(prob, target, cols: Sequence[int], Xraw: Optional[np.ndarray] = None,
                  gates: Optional[np.ndarray] = None, chunk: int = 8):
    """Riemannian quantities for the columns ``cols``.

    ``Xraw``: raw directions ``[k, n_params, 4, 4]``; they are projected onto
    the tangent space (and the parity pattern) first.  Returns
    ``(f, rgrad, hvps, Xtan)``.
    """
    gates = prob.gates if gates is None else gates
    Xtan = None
    if Xraw is not None:
        Xtan = np.stack([riemann.tangent_direction(gates, Xraw[i], prob.structure)
                         for i in range(Xraw.shape[0])])
    F, dF, dFdot = evaluate(prob, target, cols, Xtan, gates, chunk)
    gbar = riemann.tie(riemann.euclid_from_holomorphic(dF), prob.param_of, prob.n_params)
    rg = riemann.riemannian_gradient(gates, gbar, prob.structure)
    hv = None
    if Xtan is not None:
        hv = np.stack([
            riemann.riemannian_hessian(
                gates, gbar,
                riemann.tie(riemann.euclid_from_holomorphic(dFdot[i]), prob.param_of, prob.n_params),
                Xtan[i], prob.structure)
            for i in range(Xtan.shape[0])])
    return float(-F.real), rg, hv, Xtan
