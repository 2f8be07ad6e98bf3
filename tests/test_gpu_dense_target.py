"""Dense targets (model 2): any 2^n x 2^n matrix as U, against the dense
oracle (plain matrix products), for general and parity gates."""
import numpy as np
import pytest

import workloads as w
from tests._helpers import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


def _dense_ctx(rq, prob, Umat):
    return rq.Context(0).setup(0, prob.pairs, prob.param_of, prob.n_params, prob.structure,
                               model=2, dense_U=Umat, n_qubits=prob.n)


@pytest.mark.parametrize("L,depth,structure,seed", [(3, 4, 0, 71), (3, 5, 1, 72), (4, 3, 1, 73)])
def test_random_unitary_target_matches_dense_oracle(rq, L, depth, structure, seed):
    from oracle import dense, riemann
    prob = w.make_problem(L, depth, 0.4, seed=seed, structure=structure)
    Umat = w.random_unitary(1 << prob.n, seed + 1000)
    X = w.random_directions(prob.n_params, 2, seed + 2000)
    ctx = _dense_ctx(rq, prob, Umat)
    f, g, hv = ctx.hvp(prob.gates, X)
    f_ref = dense.cost(prob, Umat)
    assert abs(f - f_ref) <= 1e-12 * max(abs(f_ref), 1e-6 * 2 ** prob.n)
    assert_close(g, dense.rgrad(prob, Umat), prob.n, what="rgrad")
    for i in range(2):
        Xt = riemann.tangent_direction(prob.gates, X[i], structure)
        assert_close(hv[i], dense.rhess(prob, Umat, Xt), prob.n, what=f"hvp {i}")
    # a column range: the sum over its columns only
    ctx.set_columns(5, 23)
    sub = np.zeros_like(Umat)
    sub[:, 5:23] = Umat[:, 5:23]
    assert abs(ctx.cost(prob.gates) - dense.cost(prob, sub)) <= 1e-12 * 2 ** prob.n


def test_dense_target_equals_chain_target(rq):
    """The chain's own U given as a dense matrix reproduces the chain target."""
    from oracle import model
    prob = w.make_problem(4, 5, 0.5, seed=74)
    Umat = model.target_unitary_dense(model.hamiltonian_dense(prob.L, prob.J, prob.U, prob.periodic), prob.t)
    X = w.random_directions(prob.n_params, 1, 75)
    a = rq.Context(0).setup_problem(prob).hvp(prob.gates, X)
    b = _dense_ctx(rq, prob, Umat).hvp(prob.gates, X)
    assert abs(a[0] - b[0]) <= 1e-12 * abs(a[0])
    assert_close(b[1], a[1], prob.n, what="rgrad")
    assert_close(b[2], a[2], prob.n, what="hvp")


def test_dense_target_trust_region_step(rq):
    from oracle import dense
    prob = w.make_problem(3, 4, 0.4, seed=76, structure=1)
    Umat = w.random_unitary(1 << prob.n, 77)
    ctx = _dense_ctx(rq, prob, Umat)
    st = rq.tr_state(radius=0.05, max_radius=0.5)
    G = prob.gates.copy()
    for _ in range(3):
        G = ctx.tr_step(G, st)
    assert abs(ctx.cost(G) - dense.cost(prob, Umat, G)) <= 1e-12 * 2 ** prob.n
    assert ctx.cost(G) < dense.cost(prob, Umat)


def test_dense_target_rejects_bad_input(rq):
    prob = w.make_problem(3, 3, 0.4, seed=78)
    Umat = w.random_unitary(1 << prob.n, 79)
    with pytest.raises(ValueError):
        _dense_ctx(rq, prob, Umat[:32, :32])
    bad = Umat.copy()
    bad[3, 4] = np.nan
    with pytest.raises(rq.RQError):
        _dense_ctx(rq, prob, bad)
    ctx = _dense_ctx(rq, prob, Umat)
    with pytest.raises(rq.RQError):
        ctx.set_translation(2)
