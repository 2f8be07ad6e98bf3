"""Spinless hard-core-boson chain (paper Eq. slFH_qubit) on the device."""
import numpy as np
import pytest

import workloads as w
from tests._helpers import assert_close, oracle_eval, target_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


@pytest.mark.parametrize("L,periodic", [(8, False), (8, True), (10, True)])
def test_spinless_target_columns(rq, L, periodic):
    prob = w.make_spinless_problem(L, 3, 0.6, seed=5, periodic=periodic)
    ctx = rq.Context(0).setup_problem(prob)
    st = target_for(prob)
    for j in np.random.default_rng(L).choice(1 << L, 30, replace=False):
        assert_close(ctx.target_column(int(j)), st.column(int(j)), L, rtol=1e-13)


@pytest.mark.parametrize("structure,tied,periodic", [(0, False, False), (1, False, True), (1, True, True)])
def test_spinless_full_basis(rq, structure, tied, periodic):
    prob = w.make_spinless_problem(8, 6, 0.5, U=2.0, seed=77, structure=structure, tied=tied, periodic=periodic)
    X = w.random_directions(prob.n_params, 2, 78)
    f, g, hv, _ = oracle_eval(prob, range(256), X, chunk=64)
    ctx = rq.Context(0).setup_problem(prob)
    f2, g2, hv2 = ctx.hvp(prob.gates, X)
    assert abs(f2 - f) <= 1e-12 * abs(f)
    assert_close(g2, g, 8)
    assert_close(hv2, hv, 8)
    if tied and periodic:
        ctx.set_translation(2)
        f3, g3, hv3 = ctx.hvp(prob.gates, X)
        assert abs(f3 - f) <= 1e-12 * abs(f)
        assert_close(g3, g, 8)
        assert_close(hv3, hv, 8)


def test_spinless_sixteen_sites_translation_and_hessian(rq):
    # the paper's largest spinless system: 16 sites (n = 16), periodic, tied
    prob = w.make_spinless_problem(16, 5, 0.5, U=2.0, seed=79, structure=1, tied=True, periodic=True)
    X = w.random_directions(prob.n_params, 1, 80)
    ctx = rq.Context(0).setup_problem(prob)
    c0 = 0b0000000011110000
    ctx.set_columns(c0, c0 + 3)
    f, g, hv, _ = oracle_eval(prob, range(c0, c0 + 3), X, chunk=3)
    f2, g2, hv2 = ctx.hvp(prob.gates, X)
    assert abs(f2 - f) <= 1e-12 * max(abs(f), 1.0)
    assert_close(g2, g, 16)
    assert_close(hv2, hv, 16)
    ctx.set_columns(0, 1 << 16)
    full = ctx.hvp(prob.gates, X)
    ctx.set_translation(2)
    rep = ctx.hvp(prob.gates, X)
    assert abs(rep[0] - full[0]) <= 1e-12 * abs(full[0])
    assert_close(rep[1], full[1], 16)
    assert_close(rep[2], full[2], 16)
