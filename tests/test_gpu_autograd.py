"""torch.autograd through the library's adjoint kernels (n = 14, 7 layers)."""
import numpy as np
import pytest

import workloads as w
from tests._helpers import assert_close, target_for

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    prob = w.config_problem("n14")
    stream = torch.cuda.Stream()
    ctx = rq.Context(0, stream=stream.cuda_stream).setup_problem(prob)
    return prob, ctx


def _oracle_euclid(prob, cols, V=None):
    from oracle import riemann, statevector as sv
    Vs = None if V is None else V[None]
    F, dF, dFd = sv.evaluate(prob, target_for(prob), list(cols), Vs, chunk=len(cols))
    gb = riemann.mask(riemann.tie(riemann.euclid_from_holomorphic(dF), prob.param_of, prob.n_params), prob.structure)
    hv = None
    if V is not None:
        hv = riemann.mask(riemann.tie(riemann.euclid_from_holomorphic(dFd[0]), prob.param_of, prob.n_params),
                          prob.structure)
    return -F.real, gb, hv


def test_gradient_matches_oracle(setup):
    from paper_2506_23775_gb300.autograd import circuit_cost
    prob, ctx = setup
    for c0 in (0, 9000):
        ctx.set_columns(c0, c0 + 4)
        G = torch.tensor(prob.gates, device="cuda", requires_grad=True)
        f = circuit_cost(G, ctx)
        f.backward()
        f0, gb, _ = _oracle_euclid(prob, range(c0, c0 + 4))
        assert abs(f.item() - f0) <= 1e-12 * max(abs(f0), 1.0)
        assert_close(G.grad.cpu().numpy(), gb, prob.n, what="euclidean gradient")


def test_finite_differences_sixteen_tangent_directions(setup):
    from oracle import riemann
    from paper_2506_23775_gb300.autograd import circuit_cost
    prob, ctx = setup
    ctx.set_columns(0, 2048)
    G = torch.tensor(prob.gates, device="cuda", requires_grad=True)
    circuit_cost(G, ctx).backward()
    grad = G.grad.detach()
    h = 1e-6
    worst = 0.0
    for seed in range(402, 418):
        X = riemann.tangent_direction(prob.gates, w.random_directions(prob.n_params, 1, seed)[0], 0)
        Xt = torch.tensor(X, device="cuda")
        with torch.no_grad():
            fp = circuit_cost(G + h * Xt, ctx).item()
            fm = circuit_cost(G - h * Xt, ctx).item()
        fd = (fp - fm) / (2 * h)
        an = float((grad.conj() * Xt).real.sum())
        worst = max(worst, abs(fd - an) / max(abs(an), 1.0))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1.0) + 5e-6, (seed, fd, an)
    assert worst < 1e-6


def test_double_backward_is_the_euclidean_hessian(setup):
    from paper_2506_23775_gb300.autograd import circuit_cost
    prob, ctx = setup
    ctx.set_columns(5000, 5003)
    V = w.random_directions(prob.n_params, 1, 433)[0]
    G = torch.tensor(prob.gates, device="cuda", requires_grad=True)
    f = circuit_cost(G, ctx)
    (g,) = torch.autograd.grad(f, G, create_graph=True)
    Vt = torch.tensor(V, device="cuda")
    (hv,) = torch.autograd.grad((g.conj() * Vt).real.sum(), G)
    f0, gb, hv0 = _oracle_euclid(prob, range(5000, 5003), V)
    assert_close(g.detach().cpu().numpy(), gb, prob.n, what="gradient")
    assert_close(hv.cpu().numpy(), hv0, prob.n, what="euclidean hvp")


def test_projection_of_autograd_gradient_is_rq_grad(setup):
    from oracle import riemann
    from paper_2506_23775_gb300.autograd import circuit_cost
    prob, ctx = setup
    ctx.set_columns(100, 140)
    G = torch.tensor(prob.gates, device="cuda", requires_grad=True)
    circuit_cost(G, ctx).backward()
    rg = riemann.proj(prob.gates, G.grad.cpu().numpy())
    ctx.set_gradient_space(0)
    f, rg2 = ctx.grad(prob.gates)
    assert_close(rg, rg2, prob.n, what="P_G(autograd gradient) vs rq_grad")
