"""Write oracle-computed reference values for the full-basis tests.

Calls only the CPU oracle (``oracle/``) and the seeded input generators
(``workloads``); nothing here touches the CUDA path.  Run from the repository
root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as w  # noqa: E402
from oracle import model, statevector as sv  # noqa: E402


def _c(a):
    a = np.asarray(a)
    return {"shape": list(a.shape), "re": a.real.ravel().tolist(), "im": a.imag.ravel().tolist()}


def tied12():
    """n = 12, 9 layers, one parity gate per layer, every basis column."""
    p = w.config_problem("tied12")
    X = w.random_directions(p.n_params, 1, 202)
    st = model.SectorTarget(p.L, p.J, p.U, p.t, p.periodic)
    f, g, hv, _ = sv.cost_grad_hvp(p, st, range(1 << p.n), X, chunk=64)
    return {"workload": "tied12", "direction_seed": 202, "k": 1, "f": f,
            "rgrad": _c(g), "hvp": _c(hv)}


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tied12_full_basis.json")
    with open(out, "w") as fh:
        json.dump(tied12(), fh)
    print("wrote", out)
