"""rq_cost_static: the cost with no device allocation in the call.

Some callers cannot let a library call cudaMalloc while they run (their
device memory is all reserved by their own pool, or a cudaMalloc / cudaFree
would synchronise the whole device in a latency-critical loop).  This entry
point keeps its scratch in the library's fixed static device array instead.
The test compares it with rq_cost, which uses the context's workspace, on two
calls in a row (the second call finds the first call's leftovers in the
shared array and must clear what has to start at zero).  The file is named to
run last, so a run that stops at the first failure has run everything else.
"""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


@pytest.mark.parametrize("name,structure,cols", [
    ("small", 0, None),            # n = 8, every column
    ("small", 1, (3, 200)),        # parity tiles, ragged range
    ("tied12", 1, (1000, 1700)),   # n = 12, tied parity gates
    ("n16", 0, (0b0000011100000011, 0b0000011100000011 + 5)),  # n = 16: small tiles
])
def test_static_cost_matches_rq_cost_twice(rq, name, structure, cols):
    prob = w.config_problem(name, structure=structure)
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        if cols is not None:
            ctx.set_columns(*cols)
        ref = ctx.cost(prob.gates)
        other = prob.gates * np.exp(0.3j)   # a different input between the two calls
        for gates, want in ((prob.gates, ref), (other, ctx.cost(other)), (prob.gates, ref)):
            got = ctx.cost_static(gates)
            assert abs(got - want) <= 1e-12 * max(abs(want), 1e-6 * 2 ** prob.n), (got, want)


def _free_bytes():
    torch = pytest.importorskip("torch")
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info(0)[0]


def test_static_cost_dense_and_translation_contexts_allocate_nothing(rq):
    """A dense-target context (model 2, n = 8) and a translation context
    (periodic tied chain, orbit representatives): the static cost equals
    rq_cost, and device memory in use does not change across static calls
    once the first one has loaded the kernels it uses."""
    prob = w.make_problem(4, 5, 0.4, seed=91, structure=1)
    Umat = w.random_unitary(1 << prob.n, 1091)
    tprob = w.make_problem(4, 6, 0.7, seed=92, periodic=True, tied=True)
    with rq.Context(0) as dctx, rq.Context(0) as tctx:
        dctx.setup(0, prob.pairs, prob.param_of, prob.n_params, prob.structure, model=2, dense_U=Umat,
                   n_qubits=prob.n)
        tctx.setup_problem(tprob)
        tctx.set_translation(2)
        cases = ((dctx, prob.gates, dctx.cost(prob.gates), prob.n),
                 (tctx, tprob.gates, tctx.cost(tprob.gates), tprob.n))
        for ctx, gates, want, n in cases:
            ctx.cost_static(gates)                       # loads the kernels it uses
            before, info = _free_bytes(), ctx.info()
            for _ in range(2):
                got = ctx.cost_static(gates)
                assert abs(got - want) <= 1e-12 * max(abs(want), 1e-6 * 2 ** n), (got, want)
            assert _free_bytes() == before
            assert ctx.info() == info


def test_static_cost_validates_gates_like_rq_cost(rq):
    prob = w.config_problem("small")
    bad = prob.gates.copy()
    bad[2] *= 1.01                                       # not unitary
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        ctx.set_checks(True)
        for call in (ctx.cost, ctx.cost_static):
            with pytest.raises(rq.RQError) as e:
                call(bad)
            assert e.value.code == rq.RQ_EINVAL


def test_static_cost_before_setup_is_rejected(rq):
    with rq.Context(0) as ctx:
        with pytest.raises(rq.RQError) as e:
            ctx.cost_static(w.config_problem("small").gates)
        assert e.value.code == rq.RQ_ESTATE
