"""Parity of the CUDA path (through the C ABI) against the CPU oracle."""
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


def _ctx(rq, prob, tile=0, dirs=0):
    c = rq.Context(0).setup_problem(prob)
    if tile or dirs:
        c.set_tile(tile, dirs)
    return c


# ------------------------------------------------------------- target (a1) --

@pytest.mark.parametrize("L,t,periodic", [(4, 0.25, False), (4, 0.9, True), (6, 0.5, False)])
def test_target_columns(rq, L, t, periodic):
    prob = w.make_problem(L, 3, t, periodic=periodic)
    ctx = _ctx(rq, prob)
    st = target_for(prob)
    rng = np.random.default_rng(L)
    cols = range(1 << prob.n) if L == 4 else rng.choice(1 << prob.n, 40, replace=False)
    for j in cols:
        assert_close(ctx.target_column(int(j)), st.column(int(j)), prob.n, rtol=1e-13, what=f"U|{j}>")


def test_target_columns_sixteen_qubits(rq):
    prob = w.config_problem("n16")
    ctx = _ctx(rq, prob)
    st = target_for(prob)
    for j in (0b0000011100000011, 0b1000000000000001, 0b0000000000000000, 0b1111111111111111):
        assert_close(ctx.target_column(j), st.column(j), 16, rtol=1e-13, what=f"U|{j}>")


# ------------------------------------------------------ full basis sums ----

@pytest.mark.parametrize("name,structure", [("small", 0), ("small", 1)])
def test_full_basis_small(rq, name, structure):
    prob = w.config_problem(name, structure=structure)
    X = w.random_directions(prob.n_params, 4, 102)
    f, g, hv, _ = oracle_eval(prob, range(1 << prob.n), X, chunk=64)
    ctx = _ctx(rq, prob)
    f2, g2, hv2 = ctx.hvp(prob.gates, X)
    assert abs(f2 - f) <= 1e-12 * abs(f)
    assert_close(g2, g, prob.n, what="rgrad")
    for i in range(4):
        assert_close(hv2[i], hv[i], prob.n, what=f"hvp {i}")
    assert abs(ctx.cost(prob.gates) - f) <= 1e-12 * abs(f)
    f3, g3 = ctx.grad(prob.gates)
    assert_close(g3, g, prob.n, what="rgrad (grad call)")


def test_tied_parity_twelve_qubits_sampled(rq):
    prob = w.config_problem("tied12")
    X = w.random_directions(prob.n_params, 2, 202)
    ctx = _ctx(rq, prob)
    for c0, c1 in ((0, 37), (1500, 1561), (4050, 4096)):
        ctx.set_columns(c0, c1)
        f, g, hv, _ = oracle_eval(prob, range(c0, c1), X, chunk=64)
        f2, g2, hv2 = ctx.hvp(prob.gates, X)
        assert abs(f2 - f) <= 1e-12 * max(abs(f), 1e-6 * 2 ** 12)
        assert_close(g2, g, prob.n, what=f"rgrad [{c0},{c1})")
        assert_close(hv2, hv, prob.n, what=f"hvp [{c0},{c1})")


@pytest.mark.parametrize("structure", [0, 1])
def test_fourteen_qubits_sampled(rq, structure):
    prob = w.config_problem("n14", structure=structure)
    X = w.random_directions(prob.n_params, 1, 402)
    ctx = _ctx(rq, prob)
    for c0 in (0, 9000):
        ctx.set_columns(c0, c0 + 6)
        f, g, hv, _ = oracle_eval(prob, range(c0, c0 + 6), X)
        f2, g2, hv2 = ctx.hvp(prob.gates, X)
        assert abs(f2 - f) <= 1e-12 * max(abs(f), 1.0)
        assert_close(g2, g, prob.n, what="rgrad")
        assert_close(hv2, hv, prob.n, what="hvp")


@pytest.mark.parametrize("structure", [0, 1])
def test_sixteen_qubits_sampled(rq, structure):
    # the benchmark instance, in the benchmark's launch configuration
    prob = w.config_problem("n16", structure=structure)
    X = w.random_directions(prob.n_params, 1, 1602)
    ctx = _ctx(rq, prob)
    c0 = 0b0000011100000011  # a column of a 21 x 28 = 588 sector
    ctx.set_columns(c0, c0 + 3)
    f, g, hv, _ = oracle_eval(prob, range(c0, c0 + 3), X, chunk=3)
    f2, g2, hv2 = ctx.hvp(prob.gates, X)
    assert abs(f2 - f) <= 1e-12 * max(abs(f), 1.0)
    assert_close(g2, g, prob.n, what="rgrad")
    assert_close(hv2, hv, prob.n, what="hvp")


@pytest.mark.parametrize("structure", [0, 1])
def test_eighteen_qubits_largest_target_that_fits(rq, structure):
    """n = 18 (9 sites): the largest chain whose target store fits one GPU
    (C(18, 9)^2 complex128 entries = 37.8 GB of sector blocks; n = 20 is
    refused in test_size_limits).  Columns from small particle-number
    sectors keep the oracle's per-sector eigendecompositions cheap; the
    sweeps cost the same for every column."""
    prob = w.make_problem(9, 5, 0.5, seed=1801, structure=structure)
    X = w.random_directions(prob.n_params, 1, 1802)
    cols = [0, (1 << 17) | 1, (1 << 9) | (1 << 3), (0b111111111 << 9) | 0b111111110]
    f, g, hv, _ = oracle_eval(prob, cols, X, chunk=4)
    ctx = _ctx(rq, prob)
    assert ctx.info()["target_entries"] == 48620 ** 2
    fs, gs, hs = 0.0, np.zeros_like(g), np.zeros_like(hv)
    for j in cols:
        ctx.set_columns(j, j + 1)
        a = ctx.hvp(prob.gates, X)
        fs, gs, hs = fs + a[0], gs + a[1], hs + a[2]
    assert abs(fs - f) <= 1e-12 * max(abs(f), 1e-6 * 2 ** 18)
    assert_close(gs, g, prob.n, what="rgrad")
    assert_close(hs, hv, prob.n, what="hvp")


# ------------------------------------------------------------ edge cases ----

def test_empty_range_and_additivity_and_determinism(rq):
    prob = w.make_problem(4, 5, 0.3, seed=7)
    X = w.random_directions(prob.n_params, 1, 8)
    ctx = _ctx(rq, prob, tile=32)
    ctx.set_columns(17, 17)
    f0, g0, h0 = ctx.hvp(prob.gates, X)
    assert f0 == 0.0 and not g0.any() and not h0.any()
    ctx.set_columns(0, 101)          # ragged: 101 = 3 * 32 + 5
    a = ctx.hvp(prob.gates, X)
    ctx.set_columns(101, 256)
    b = ctx.hvp(prob.gates, X)
    ctx.set_columns(0, 256)
    c = ctx.hvp(prob.gates, X)
    c2 = ctx.hvp(prob.gates, X)
    assert c[0] == c2[0] and np.array_equal(c[1], c2[1]) and np.array_equal(c[2], c2[2])
    assert abs(a[0] + b[0] - c[0]) <= 1e-12 * abs(c[0])
    assert_close(a[1] + b[1], c[1], 8, what="grad additivity")
    assert_close(a[2] + b[2], c[2], 8, what="hvp additivity")
    f, g, hv, _ = oracle_eval(prob, range(256), X, chunk=64)
    assert_close(c[1], g, 8)
    assert_close(c[2], hv, 8)


@pytest.mark.parametrize("tile,dirs", [(1, 1), (8, 2), (256, 4)])
def test_tile_and_direction_chunking(rq, tile, dirs):
    prob = w.make_problem(4, 4, 0.4, seed=12, structure=1)
    X = w.random_directions(prob.n_params, 5, 13)  # 5 directions: several chunks
    f, g, hv, _ = oracle_eval(prob, range(256), X, chunk=64)
    ctx = _ctx(rq, prob, tile=tile, dirs=dirs)
    f2, g2, hv2 = ctx.hvp(prob.gates, X)
    assert abs(f2 - f) <= 1e-12 * abs(f)
    assert_close(g2, g, 8)
    assert_close(hv2, hv, 8)


@pytest.mark.parametrize("structure", [0, 1])
def test_periodic_wrap_bond_listed_high_to_low(rq, structure):
    prob = w.make_problem(4, 6, 0.35, seed=23, periodic=True, structure=structure)
    assert any(a > b for a, b in prob.pairs.tolist())
    X = w.random_directions(prob.n_params, 1, 24)
    f, g, hv, _ = oracle_eval(prob, range(256), X, chunk=64)
    ctx = _ctx(rq, prob)
    f2, g2, hv2 = ctx.hvp(prob.gates, X)
    assert abs(f2 - f) <= 1e-12 * abs(f)
    assert_close(g2, g, 8)
    assert_close(hv2, hv, 8)


def test_invalid_arguments(rq):
    prob = w.config_problem("small")
    ctx = rq.Context(0)
    with pytest.raises(rq.RQError) as e:
        ctx.cost(prob.gates)
    assert e.value.code == rq.RQ_ESTATE
    bad = prob.pairs.copy()
    bad[3] = (2, 2)
    with pytest.raises(rq.RQError) as e:
        ctx.setup(prob.L, bad)
    assert e.value.code == rq.RQ_EINVAL
    ctx.setup_problem(prob)
    with pytest.raises(rq.RQError):
        ctx.set_columns(5, 3)
    with pytest.raises(rq.RQError):
        ctx.set_columns(0, 257)
    with pytest.raises(rq.RQError):
        ctx.set_tile(3, 1)


def test_size_limits(rq):
    """n = 20 (10 sites) is within the qubit limit, but the target's sector
    blocks alone would need C(20,10)^2 x 16 B = 546 GB: set-up fails with
    RQ_ENOMEM and the context stays usable; n = 22 is past the limit."""
    ctx = rq.Context(0)
    with pytest.raises(rq.RQError) as e:
        ctx.setup_problem(w.make_problem(10, 1, 0.5, seed=3))
    assert e.value.code == rq.RQ_ENOMEM
    with pytest.raises(rq.RQError) as e:
        ctx.setup_problem(w.make_problem(11, 1, 0.5, seed=3))
    assert e.value.code == rq.RQ_EINVAL
    prob = w.config_problem("small")
    ref = _ctx(rq, prob).cost(prob.gates)
    assert ctx.setup_problem(prob).cost(prob.gates) == ref


def test_context_reuse_across_problems(rq):
    """One context set up for several problems in turn gives exactly what a
    fresh context gives for each (no per-problem state survives a set-up)."""
    seq = [w.config_problem("n14"), w.config_problem("small"), w.config_problem("tied12"),
           w.config_problem("small", structure=1), w.make_problem(5, 4, 0.3, seed=8, periodic=True)]
    ctx = rq.Context(0)
    for prob in seq:
        X = w.random_directions(prob.n_params, 2, 17)
        cols = (0, min(1 << prob.n, 600))
        ctx.setup_problem(prob)
        ctx.set_columns(*cols)
        got = ctx.hvp(prob.gates, X)
        fresh = _ctx(rq, prob)
        fresh.set_columns(*cols)
        ref = fresh.hvp(prob.gates, X)
        assert got[0] == ref[0]
        assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])


def test_device_pointer_variants_match_host(rq):
    torch = pytest.importorskip("torch")
    prob = w.config_problem("small")
    X = w.random_directions(prob.n_params, 2, 5)
    ctx = _ctx(rq, prob)
    f, g, hv = ctx.hvp(prob.gates, X)
    dev = torch.device("cuda:0")
    tg = torch.from_numpy(prob.gates.copy()).to(dev)
    tx = torch.from_numpy(X.copy()).to(dev)
    tf = torch.zeros(1, dtype=torch.float64, device=dev)
    trg = torch.zeros_like(tg)
    thv = torch.zeros_like(tx)
    ctx.hvp_dev(tg.data_ptr(), tx.data_ptr(), 2, tf.data_ptr(), trg.data_ptr(), thv.data_ptr())
    torch.cuda.synchronize()
    assert tf.item() == f
    assert np.array_equal(trg.cpu().numpy(), g)
    assert np.array_equal(thv.cpu().numpy(), hv)


def test_tied_parity_twelve_qubits_full_basis_golden(rq):
    # every one of the 4096 columns, against values the oracle wrote once
    # (tests/golden/make_golden.py)
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tied12_full_basis.json")
    data = json.load(open(path))
    cplx = lambda d: (np.array(d["re"]) + 1j * np.array(d["im"])).reshape(d["shape"])
    prob = w.config_problem("tied12")
    X = w.random_directions(prob.n_params, 1, data["direction_seed"])
    ctx = _ctx(rq, prob)
    f, g, hv = ctx.hvp(prob.gates, X)
    assert abs(f - data["f"]) <= 1e-12 * abs(data["f"])
    assert_close(g, cplx(data["rgrad"]), 12, what="rgrad")
    assert_close(hv, cplx(data["hvp"]), 12, what="hvp")
