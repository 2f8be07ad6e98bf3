"""Double-float sweeps (RQ_ARITH_DF64) against the FP64 oracle and the FP64 path."""
import json
import os

import numpy as np
import pytest

import workloads as w
from tests._helpers import assert_close, oracle_eval

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


def _pair(rq, prob, tile=0, dirs=0):
    out = []
    for arith in (0, 1):
        c = rq.Context(0).setup_problem(prob)
        if tile or dirs:
            c.set_tile(tile, dirs)
        c.set_arithmetic(arith)
        out.append(c)
    return out


@pytest.mark.parametrize("structure", [0, 1])
def test_full_basis_small_df64(rq, structure):
    prob = w.config_problem("small", structure=structure)
    X = w.random_directions(prob.n_params, 4, 102)
    f, g, hv, _ = oracle_eval(prob, range(1 << prob.n), X, chunk=64)
    c64, cdf = _pair(rq, prob)
    f2, g2, hv2 = cdf.hvp(prob.gates, X)
    assert abs(f2 - f) <= 1e-12 * abs(f)
    assert_close(g2, g, prob.n, what="rgrad df64")
    assert_close(hv2, hv, prob.n, what="hvp df64")
    assert abs(cdf.cost(prob.gates) - f) <= 1e-12 * abs(f)
    f3, g3, hv3 = c64.hvp(prob.gates, X)
    rel = np.linalg.norm(hv2 - hv3) / np.linalg.norm(hv3)
    assert rel < 1e-12, rel


def test_tied12_golden_df64(rq):
    path = os.path.join(os.path.dirname(__file__), "golden", "tied12_full_basis.json")
    data = json.load(open(path))
    cplx = lambda d: (np.array(d["re"]) + 1j * np.array(d["im"])).reshape(d["shape"])
    prob = w.config_problem("tied12")
    X = w.random_directions(prob.n_params, 1, data["direction_seed"])
    _, cdf = _pair(rq, prob)
    f, g, hv = cdf.hvp(prob.gates, X)
    assert abs(f - data["f"]) <= 1e-12 * abs(data["f"])
    assert_close(g, cplx(data["rgrad"]), 12, what="rgrad")
    assert_close(hv, cplx(data["hvp"]), 12, what="hvp")


@pytest.mark.parametrize("name,structure,c0,ncols", [("n14", 0, 9000, 6), ("n16", 0, 0b0000011100000011, 3),
                                                     ("n16", 1, 0b0000011100000011, 3)])
def test_sampled_large_df64(rq, name, structure, c0, ncols):
    prob = w.config_problem(name, structure=structure)
    X = w.random_directions(prob.n_params, 1, 1602)
    _, cdf = _pair(rq, prob)
    cdf.set_columns(c0, c0 + ncols)
    f, g, hv, _ = oracle_eval(prob, range(c0, c0 + ncols), X, chunk=ncols)
    f2, g2, hv2 = cdf.hvp(prob.gates, X)
    assert abs(f2 - f) <= 1e-12 * max(abs(f), 1.0)
    assert_close(g2, g, prob.n, what="rgrad")
    assert_close(hv2, hv, prob.n, what="hvp")


@pytest.mark.parametrize("structure", [0, 1])
def test_periodic_and_chunking_df64(rq, structure):
    prob = w.make_problem(4, 6, 0.35, seed=23, periodic=True, structure=structure)
    X = w.random_directions(prob.n_params, 5, 24)
    f, g, hv, _ = oracle_eval(prob, range(256), X, chunk=64)
    _, cdf = _pair(rq, prob, tile=16, dirs=2)
    cdf.set_columns(0, 256)
    f2, g2, hv2 = cdf.hvp(prob.gates, X)
    assert abs(f2 - f) <= 1e-12 * abs(f)
    assert_close(g2, g, 8)
    assert_close(hv2, hv, 8)


def test_df64_trust_region_step(rq):
    prob = w.config_problem("tied12")
    c64, cdf = _pair(rq, prob)
    s64, sdf = rq.tr_state(), rq.tr_state()
    g64 = c64.tr_step(prob.gates, s64)
    gdf = cdf.tr_step(prob.gates, sdf)
    assert s64.n_inner == sdf.n_inner and s64.tcg_exit == sdf.tcg_exit
    assert abs(s64.f_new - sdf.f_new) <= 1e-12 * abs(s64.f_new)
    assert np.abs(g64 - gdf).max() < 1e-10
