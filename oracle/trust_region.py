"""Riemannian trust region with truncated CG (oracle; test infrastructure).

Paper Sec. "Riemannian optimization": the quadratic model
``m(X) = f + <grad f, X> + 1/2 <Hess f[X], X>``, the Riemannian trust-region
method (Absil et al., Algorithm 10) with the truncated conjugate-gradient
(Steihaug) inner solver (Algorithm 11), the polar retraction on every gate
(Eq. retraction_qr) and the metric ``sum Re Tr[X^dagger Y]``.

Constants the paper leaves open (initial/maximal radius, acceptance
threshold, inner stopping rule) are the caller's ``TRParams``; the defaults
are ``radius=0.01``, ``max_radius=0.1``, ``rho_accept=0.125``,
``kappa=0.1``, ``theta=1`` and at most ``dim`` inner iterations.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import riemann


@dataclass
class TRParams:
    radius: float = 0.01
    max_radius: float = 0.1
    rho_accept: float = 0.125
    kappa: float = 0.1
    theta: float = 1.0
    max_inner: int = 0  # 0: the tangent-space dimension


def _to_boundary(eta, delta, radius):
    """Positive ``tau`` with ``||eta + tau delta|| = radius``."""
    a = riemann.inner(delta, delta)
    b = 2.0 * riemann.inner(eta, delta)
    c = riemann.inner(eta, eta) - radius * radius
    return (-b + np.sqrt(b * b - 4.0 * a * c)) / (2.0 * a)


def tcg(grad, hess, radius, kappa, theta, max_inner):
    """Algorithm 11.  Returns ``(eta, H eta, iterations, exit_code)``.

    exit codes: 0 residual small, 1 negative curvature, 2 hit the radius,
    3 iteration cap.
    """
    eta = np.zeros_like(grad)
    Heta = np.zeros_like(grad)
    r = grad.copy()
    delta = -r
    rr = riemann.inner(r, r)
    r0 = np.sqrt(rr)
    for j in range(max_inner):
        Hd = hess(delta)
        dHd = riemann.inner(delta, Hd)
        if dHd <= 0.0:
            tau = _to_boundary(eta, delta, radius)
            return eta + tau * delta, Heta + tau * Hd, j + 1, 1
        alpha = rr / dHd
        eta_new = eta + alpha * delta
        if np.sqrt(riemann.inner(eta_new, eta_new)) >= radius:
            tau = _to_boundary(eta, delta, radius)
            return eta + tau * delta, Heta + tau * Hd, j + 1, 2
        eta = eta_new
        Heta = Heta + alpha * Hd
        r = r + alpha * Hd
        rr_new = riemann.inner(r, r)
        if np.sqrt(rr_new) <= r0 * min(r0 ** theta, kappa):
            return eta, Heta, j + 1, 0
        beta = rr_new / rr
        rr = rr_new
        delta = -r + beta * delta
    return eta, Heta, max_inner, 3


def tr_step(cost, grad_fn, hess_fn, G, radius, params: TRParams, structure: int = 0):
    """One iteration of Algorithm 10.

    ``cost(G) -> f``, ``grad_fn(G) -> (f, rgrad)``, ``hess_fn(G, X) -> Hess[X]``.
    Returns ``(G_next, radius_next, info)``.
    """
    f, g = grad_fn(G)
    dim = G.shape[0] * (8 if structure == 1 else 16)
    max_inner = params.max_inner or dim
    eta, Heta, n_inner, code = tcg(g, lambda X: hess_fn(G, X), radius,
                                   params.kappa, params.theta, max_inner)
    cand = riemann.retract(G, eta)
    f_new = cost(cand)
    model_decrease = -(riemann.inner(g, eta) + 0.5 * riemann.inner(Heta, eta))
    rho = (f - f_new) / model_decrease if model_decrease != 0.0 else 0.0
    norm_eta = np.sqrt(riemann.inner(eta, eta))
    if rho < 0.25:
        new_radius = 0.25 * radius
    elif rho > 0.75 and code in (1, 2):  # the step reached the boundary
        new_radius = min(2.0 * radius, params.max_radius)
    else:
        new_radius = radius
    accepted = rho > params.rho_accept
    info = dict(f=f, f_new=f_new, rho=rho, accepted=accepted, n_inner=n_inner,
                tcg_exit=code, norm_eta=norm_eta)
    return (cand if accepted else G), new_radius, info
