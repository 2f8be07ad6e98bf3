"""Shared test helpers: tolerance rule and cached oracle targets."""
import functools

import numpy as np

RTOL = 1e-12  # relative tolerance of every FP64 parity comparison


def floor(n: int) -> float:
    """Absolute floor s = 1e-6 * 2^n of the relative test (results near an
    optimum are small; a pure relative test would be meaningless there)."""
    return 1e-6 * 2.0 ** n


def assert_close(got, ref, n: int, rtol: float = RTOL, what: str = ""):
    """Norm-wise ``||got - ref|| <= rtol * max(||ref||, s)`` over all entries."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    err = float(np.linalg.norm(np.ravel(got - ref)))
    scale = max(float(np.linalg.norm(np.ravel(ref))), floor(n))
    assert err <= rtol * scale, f"{what}: |err| = {err:.3e} > {rtol:.0e} * {scale:.3e} (rel {err / scale:.2e})"


@functools.lru_cache(maxsize=None)
def sector_target(L, J, U, t, periodic, model_id=0):
    from oracle import model
    return model.SectorTarget(L, J, U, t, periodic, model_id)


def target_for(prob):
    return sector_target(prob.L, prob.J, prob.U, prob.t, prob.periodic, getattr(prob, "model", 0))


def oracle_eval(prob, cols, Xraw=None, gates=None, chunk=16):
    from oracle import statevector as sv
    return sv.cost_grad_hvp(prob, target_for(prob), list(cols), Xraw, gates=gates, chunk=chunk)


def load_golden(fname):
    """A file of oracle-written values under tests/golden/ (make_golden.py),
    with every {"shape", "re", "im"} entry turned into a complex array."""
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", fname)) as fh:
        data = json.load(fh)

    def conv(d):
        if isinstance(d, dict):
            if set(d) == {"shape", "re", "im"}:
                return (np.array(d["re"]) + 1j * np.array(d["im"])).reshape(d["shape"])
            return {k: conv(v) for k, v in d.items()}
        if isinstance(d, list):
            return [conv(v) for v in d]
        return d
    return conv(data)
