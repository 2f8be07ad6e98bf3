"""Trust-region optimisation from the 4th-order Trotter initialisation
(21 layers, periodic spinful chain), the paper's convergence setting at a
size the test can run: error = ||C(G) - U||_F / ||U||_F = sqrt((2 * 2^n + 2f) / 2^n)."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


def _err(f, n):
    return np.sqrt(max(2 * 2 ** n + 2 * f, 0.0) / 2 ** n)


@pytest.mark.parametrize("full_hessian", [False, True])
def test_trust_region_from_fourth_order_trotter(rq, full_hessian):
    prob = w.make_problem(4, 21, 1.0, sigma=0.0, order=4, periodic=True, tied=True)
    assert prob.n_gates == 84 and prob.n_params == 21
    ctx = rq.Context(0).setup_problem(prob)
    ctx.set_translation(2)                        # periodic, one gate per layer
    st = rq.tr_state(radius=0.01, max_radius=0.1, full_hessian=full_hessian)
    G = prob.gates.copy()
    f0 = ctx.cost(G)
    errs = [_err(f0, prob.n)]
    for it in range(25):
        G = ctx.tr_step(G, st)
        errs.append(_err(st.f_new if st.accepted else st.f, prob.n))
    assert all(b <= a * (1 + 1e-9) for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 0.5 * errs[0], errs
    print("error", errs[0], "->", errs[-1])
    for p in range(prob.n_params):
        np.testing.assert_allclose(G[p].conj().T @ G[p], np.eye(4), atol=1e-12)
