"""Host-memory evaluations replayed from captured CUDA graphs give bitwise the
results of direct launches, pick up new inputs on every call, and are
recaptured when the configuration changes."""
import time

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


def _perturbed(prob, seed, eps=0.05):
    """Unitary perturbations of the circuit's gates (new inputs each call)."""
    rng = np.random.default_rng(seed)
    out = prob.gates.copy()
    for i in range(out.shape[0]):
        h = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
        h = eps * (h + h.conj().T) / 2
        wv, v = np.linalg.eigh(h)
        out[i] = (v * np.exp(1j * wv)) @ v.conj().T @ out[i]
    return out


def _all(ctx, gates, X):
    return ctx.cost(gates), ctx.grad(gates), ctx.hvp(gates, X)


def _same(a, b):
    (fa, ga, ha), (fb, gb, hb) = a, b
    assert fa == fb
    assert ga[0] == gb[0] and np.array_equal(ga[1], gb[1])
    assert ha[0] == hb[0] and np.array_equal(ha[1], hb[1]) and np.array_equal(ha[2], hb[2])


@pytest.mark.parametrize("name,structure", [("small", 0), ("small", 1), ("tied12", 1)])
def test_graph_replay_is_bitwise_equal(rq, name, structure):
    prob = w.config_problem(name, structure=structure)
    X = w.random_directions(prob.n_params, 3, 5)
    direct = rq.Context(0).setup_problem(prob)
    direct.set_graphs(False)
    graphed = rq.Context(0).setup_problem(prob)
    for seed in range(4):  # replays see each call's inputs
        gates = _perturbed(prob, seed)
        _same(_all(graphed, gates, X), _all(direct, gates, X))
    # every configuration change is followed by a recapture
    for c in (direct, graphed):
        c.set_columns(3, 40)
    _same(_all(graphed, prob.gates, X), _all(direct, prob.gates, X))
    # another column range of the same size keeps the layout (and the graphs):
    # the column table is read at run time
    for c in (direct, graphed):
        c.set_columns(40, 77)
    _same(_all(graphed, prob.gates, X), _all(direct, prob.gates, X))
    for c in (direct, graphed):
        c.set_arithmetic(1)
    _same(_all(graphed, prob.gates, X), _all(direct, prob.gates, X))
    for c in (direct, graphed):
        c.set_gradient_space(1)
        c.set_tile(0, 1)
    _same(_all(graphed, prob.gates, X), _all(direct, prob.gates, X))
    for c in (direct, graphed):
        c.set_first_layer(False)
    _same(_all(graphed, prob.gates, X), _all(direct, prob.gates, X))
    # more directions than the buffers held: reallocation, then recapture
    X7 = w.random_directions(prob.n_params, 7, 6)
    a, b = graphed.hvp(prob.gates, X7), direct.hvp(prob.gates, X7)
    assert a[0] == b[0] and np.array_equal(a[2], b[2])
    # launch accounting: a replay counts the kernels it ran
    n0 = graphed.info()["kernel_launches"]
    graphed.cost(prob.gates)
    n1 = graphed.info()["kernel_launches"]
    m0 = direct.info()["kernel_launches"]
    direct.cost(prob.gates)
    assert n1 - n0 == direct.info()["kernel_launches"] - m0 > 0


def test_graph_trust_region_steps_bitwise_equal(rq):
    prob = w.config_problem("small", structure=1)
    runs = []
    for use in (False, True):
        ctx = rq.Context(0).setup_problem(prob)
        ctx.set_graphs(use)
        state = rq.tr_state(radius=0.05, max_radius=0.5)
        gates = prob.gates.copy()
        for _ in range(3):
            gates = ctx.tr_step(gates, state)
        runs.append((gates, state.f, state.radius))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert runs[0][1] == runs[1][1] and runs[0][2] == runs[1][2]


def test_graph_replay_is_not_slower_for_small_problems(rq):
    """One graph launch replaces ~50 kernel launches of an n = 8 HVP (about
    10 % of the call time on an idle GPU; the bound leaves room for timer
    noise on a shared host)."""
    prob = w.config_problem("small", structure=0)
    X = w.random_directions(prob.n_params, 1, 3)
    times = {}
    for use in (False, True):
        ctx = rq.Context(0).setup_problem(prob)
        ctx.set_graphs(use)
        for _ in range(5):
            ctx.hvp(prob.gates, X)
        t0 = time.perf_counter()
        for _ in range(50):
            ctx.hvp(prob.gates, X)
        times[use] = (time.perf_counter() - t0) / 50
    print(f"direct {times[False] * 1e6:.0f} us, graph {times[True] * 1e6:.0f} us per HVP call")
    assert times[True] < 1.03 * times[False]
