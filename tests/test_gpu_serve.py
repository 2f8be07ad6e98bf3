"""Continuous batching: requests overlap on the device and each result equals
the same request evaluated alone."""
import numpy as np
import pytest

import workloads as w
from tests._helpers import assert_close, oracle_eval

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2506_23775_gb300 import _build, rq, serve
    _build.build()
    return rq, serve


def _stream(serve):
    rng = np.random.default_rng(501)
    base = [w.make_problem(L, d, t, U=4.0, seed=600 + i)
            for i, (L, d, t) in enumerate([(3, 5, 0.4), (4, 3, 0.7), (5, 5, 0.2), (4, 7, 0.9)])]
    base.append(w.make_problem(4, 5, 0.5, seed=650, structure=1))
    probs, kinds = [], []
    for i in range(14):
        p = base[int(rng.integers(len(base)))]
        q = w.make_problem(p.L, p.depth, p.t, U=p.U, seed=700 + i, structure=p.structure)  # same problem, new gates
        probs.append(q)
        kinds.append(("cost", "grad", "hvp")[i % 3])
    return serve.poisson_stream(probs, kinds, rate_hz=400.0, seed=502, k=2)


@pytest.mark.parametrize("grid", [0, 8])
def test_results_in_the_mix_equal_results_alone(mods, grid):
    rq, serve = mods
    reqs = _stream(serve)
    srv = serve.Server(0, memory_budget=8 << 30, max_inflight=4, tile=64, contexts_per_problem=2, grid=grid)
    stats = srv.run(reqs)
    srv.close()
    assert stats["requests"] == len(reqs) and stats["reused"] > 0
    # some request was admitted while another was still on the GPU
    overlap = any(a.admitted < b.done and b.admitted < a.done for a in reqs for b in reqs if a is not b)
    assert overlap
    for r in reqs:
        p = r.problem
        with rq.Context(0) as ctx:
            ctx.setup_problem(p)
            ctx.set_tile(min(64, 1 << p.n), 1)
            ctx.set_grid(grid)
            if r.kind == "cost":
                assert ctx.cost(p.gates) == r.f
            elif r.kind == "grad":
                f, g = ctx.grad(p.gates)
                assert f == r.f and np.array_equal(g, r.rgrad)
            else:
                f, g, hv = ctx.hvp(p.gates, r.dirs)
                assert f == r.f and np.array_equal(g, r.rgrad) and np.array_equal(hv, r.hvps)
    r = next(r for r in reqs if r.kind == "hvp" and r.problem.n <= 8)
    f, g, hv, _ = oracle_eval(r.problem, range(1 << r.problem.n), r.dirs, chunk=64)
    assert abs(r.f - f) <= 1e-12 * abs(f)
    assert_close(r.rgrad, g, r.problem.n)
    assert_close(r.hvps, hv, r.problem.n)


def test_admission_by_footprint(mods):
    rq, serve = mods
    p = w.make_problem(5, 3, 0.3, seed=9)
    need = serve.footprint_bytes(p, 64, 1)
    srv = serve.Server(0, memory_budget=need - 1, max_inflight=2, tile=64)
    with pytest.raises(MemoryError):
        srv.run([serve.Request(0, "cost", p)])
    srv.close()
