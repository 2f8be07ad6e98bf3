"""Gate validation (rq_set_checks): unitarity and the parity pattern are
checked before any launch, on every entry point that takes gates."""
import numpy as np
import pytest
import torch

import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


def _calls(rq, ctx, gates, X):
    dev = torch.device("cuda", 0)
    g_d = torch.from_numpy(np.ascontiguousarray(gates)).to(dev)
    f_d = torch.zeros(1, dtype=torch.float64, device=dev)
    r_d = torch.zeros_like(g_d)
    return {
        "cost": lambda: ctx.cost(gates),
        "grad": lambda: ctx.grad(gates),
        "hvp": lambda: ctx.hvp(gates, X),
        "hessian": lambda: ctx.hessian(gates),
        "tr_step": lambda: ctx.tr_step(gates, rq.tr_state()),
        "cost_dev": lambda: (ctx.cost_dev(g_d.data_ptr(), f_d.data_ptr()), torch.cuda.synchronize()),
        "grad_dev": lambda: (ctx.grad_dev(g_d.data_ptr(), f_d.data_ptr(), r_d.data_ptr()),
                             torch.cuda.synchronize()),
    }


@pytest.mark.parametrize("structure", [0, 1])
def test_valid_gates_pass_and_give_the_same_results(rq, structure):
    prob = w.config_problem("small", structure=structure)
    X = w.random_directions(prob.n_params, 1, 3)
    ref = rq.Context(0).setup_problem(prob).hvp(prob.gates, X)
    ctx = rq.Context(0).setup_problem(prob)
    ctx.set_checks(True)
    got = ctx.hvp(prob.gates, X)
    assert got[0] == ref[0] and np.array_equal(got[2], ref[2])
    for name, call in _calls(rq, ctx, prob.gates, X).items():
        call()


@pytest.mark.parametrize("structure", [0, 1])
def test_non_unitary_gate_is_rejected_everywhere(rq, structure):
    prob = w.config_problem("small", structure=structure)
    X = w.random_directions(prob.n_params, 1, 3)
    bad = prob.gates.copy()
    bad[5] *= 1.0 + 1e-8
    ctx = rq.Context(0).setup_problem(prob)
    ctx.set_checks(True)
    for name, call in _calls(rq, ctx, bad, X).items():
        with pytest.raises(rq.RQError, match="gate 5 is not unitary"):
            call()
    ctx.cost(prob.gates)  # the context stays usable
    ctx.set_checks(False)
    ctx.cost(bad)         # unchecked: evaluated as given


def test_parity_pattern_violation_is_rejected(rq):
    prob = w.config_problem("small", structure=1)
    bad = prob.gates.copy()
    # a unitary outside the pattern: swap rows 0 and 1 of gate 2
    bad[2] = bad[2][[1, 0, 2, 3]]
    ctx = rq.Context(0).setup_problem(prob)
    ctx.set_checks(True)
    with pytest.raises(rq.RQError, match="parity gate 2"):
        ctx.cost(bad)
    nan = prob.gates.copy()
    nan[0, 1, 1] = np.nan
    with pytest.raises(rq.RQError, match="non-finite"):
        ctx.cost(nan)
