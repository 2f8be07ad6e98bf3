"""Write oracle-computed reference values for the GPU tests.

Calls only the CPU oracle (``oracle/``) and the seeded input generators
(``workloads``); nothing here touches the CUDA path.  Run from the repository
root:

    python tests/golden/make_golden.py            # every file
    python tests/golden/make_golden.py tile16 tr8  # some of them

Column sums are split over a pool of spawned processes, one contiguous chunk
of columns each; the chunks' results (f, Riemannian gradient and HVPs, all
linear in the per-column summands at fixed gates) are added in chunk order.

Files:

* ``tied12_full_basis.json``: the tied parity n = 12 workload, f, gradient and
  one HVP over all 4096 columns.
* ``tile14_general.json``: n = 14 (7 sites, 7 layers, 44 general gates), f,
  gradient and one HVP over columns [0, 512): one 512-column tile.
* ``tile16_general.json``: the n = 16 benchmark instance (78 general gates),
  columns [0, 512): the first tile of the benchmark, one HVP direction.
* ``tile16_parity.json``: the same with parity gates, columns [0, 1024): the
  benchmark's first parity step, one even and one odd 512-column tile.
* ``tr12_trajectory.json``: three trust-region iterations (Alg. 10 with the
  truncated CG of Alg. 11) of the tied parity n = 12 workload over all 4096
  columns: per step f, f_new, rho, acceptance, inner iterations, tCG exit,
  the radius after the step and the gates after the step.
* ``tr8_trajectory.json``: general gates at n = 8 (4 sites, 7 layers,
  t = 1, seed 103), all 256 columns: thirty iterations from a start with
  noise 0.05 (radius 0.01, at most 0.04), and six from a start with noise 0.3
  and radius 1.5 (rejected steps, radius shrinks); the per-step scalars of
  every step and the gates after steps 1, 10 and 30 (1 and 6).
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as w  # noqa: E402
from oracle import model, statevector as sv, trust_region as tr  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

_TARGETS = {}


def _c(a):
    a = np.asarray(a)
    return {"shape": list(a.shape), "re": a.real.ravel().tolist(), "im": a.imag.ravel().tolist()}


def _target(p):
    key = (p.L, p.J, p.U, p.t, p.periodic, p.model)
    if key not in _TARGETS:
        _TARGETS[key] = model.SectorTarget(p.L, p.J, p.U, p.t, p.periodic, p.model)
    return _TARGETS[key]


def _partial(args):
    p, cols, Xraw, gates, chunk = args
    f, g, hv, _ = sv.cost_grad_hvp(p, _target(p), cols, Xraw, gates=gates, chunk=chunk)
    return f, g, hv


class Pooled:
    """Oracle sums over ``cols`` split into contiguous chunks on a pool."""

    def __init__(self, pool, p, cols, per_job, chunk):
        self.pool, self.p, self.chunk = pool, p, chunk
        cols = list(cols)
        self.jobs = [cols[i:i + per_job] for i in range(0, len(cols), per_job)]

    def __call__(self, gates, Xraw=None):
        res = self.pool.map(_partial, [(self.p, js, Xraw, gates, self.chunk) for js in self.jobs], chunksize=1)
        f = 0.0
        g = np.zeros_like(res[0][1])
        hv = None if Xraw is None else np.zeros_like(res[0][2])
        for fr, gr, hr in res:   # chunk order
            f += fr
            g += gr
            if hv is not None:
                hv += hr
        return f, g, hv


def tied12(pool):
    """n = 12, 9 layers, one parity gate per layer, every basis column."""
    p = w.config_problem("tied12")
    X = w.random_directions(p.n_params, 1, 202)
    st = model.SectorTarget(p.L, p.J, p.U, p.t, p.periodic)
    f, g, hv, _ = sv.cost_grad_hvp(p, st, range(1 << p.n), X, chunk=64)
    return {"workload": "tied12", "direction_seed": 202, "k": 1, "f": f,
            "rgrad": _c(g), "hvp": _c(hv)}


def _tile(pool, name, structure, c0, c1, dseed, per_job, chunk):
    p = w.config_problem(name, structure=structure)
    X = w.random_directions(p.n_params, 1, dseed)
    f, g, hv = Pooled(pool, p, range(c0, c1), per_job, chunk)(p.gates, X)
    return {"workload": name, "structure": structure, "columns": [c0, c1], "direction_seed": dseed, "k": 1,
            "f": f, "rgrad": _c(g), "hvp": _c(hv)}


def tile14(pool):
    return _tile(pool, "n14", 0, 0, 512, 402, 16, 8)


def tile16(pool):
    return _tile(pool, "n16", 0, 0, 512, 1602, 8, 4)


def tile16p(pool):
    return _tile(pool, "n16", 1, 0, 1024, 1602, 8, 4)


def _trajectory(pool, p, steps, keep, per_job, chunk, params):
    ev = Pooled(pool, p, range(1 << p.n), per_job, chunk)
    cost = lambda G: ev(G)[0]
    grad = lambda G: ev(G)[:2]
    hess = lambda G, X: ev(G, X[None])[2][0]
    G, radius = p.gates.copy(), params.radius
    out = []
    for it in range(steps):
        G, radius, info = tr.tr_step(cost, grad, hess, G, radius, params, p.structure)
        rec = {"step": it + 1, "f": info["f"], "f_new": info["f_new"], "rho": info["rho"],
               "accepted": bool(info["accepted"]), "n_inner": int(info["n_inner"]),
               "tcg_exit": int(info["tcg_exit"]), "radius": radius}
        if it + 1 in keep:
            rec["gates"] = _c(G)
        out.append(rec)
        print(f"  step {it + 1}: f {info['f']:.15e} rho {info['rho']:.6f} inner {info['n_inner']}", flush=True)
    return out


def tr12(pool):
    p = w.config_problem("tied12")
    params = tr.TRParams(radius=0.01, max_radius=0.1)
    steps = _trajectory(pool, p, 3, {1, 2, 3}, 64, 64, params)
    return {"workload": "tied12", "radius0": 0.01, "max_radius": 0.1, "steps": steps}


def tr8(pool):
    # n = 8 (4 sites), 7 layers, t = 1: far enough from its optimum that 30
    # steps with the radius capped at 0.04 neither converge nor reach the
    # rounding floor of f; a second start (noise 0.3, radius 1.5) rejects
    # steps and shrinks the radius within its first six iterations
    out = {}
    for key, sigma, r0, rmax, nsteps, keep in (("long", 0.05, 0.01, 0.04, 30, {1, 10, 30}),
                                                ("shrink", 0.3, 1.5, 1.5, 6, {1, 6})):
        p = w.make_problem(4, 7, 1.0, seed=103, sigma=sigma)
        params = tr.TRParams(radius=r0, max_radius=rmax)
        out[key] = {"L": 4, "depth": 7, "t": 1.0, "seed": 103, "sigma": sigma, "radius0": r0, "max_radius": rmax,
                    "steps": _trajectory(pool, p, nsteps, keep, 32, 32, params)}
    return out


FILES = {
    "tied12": ("tied12_full_basis.json", tied12),
    "tile14": ("tile14_general.json", tile14),
    "tile16": ("tile16_general.json", tile16),
    "tile16p": ("tile16_parity.json", tile16p),
    "tr12": ("tr12_trajectory.json", tr12),
    "tr8": ("tr8_trajectory.json", tr8),
}


if __name__ == "__main__":
    names = sys.argv[1:] or list(FILES)
    os.environ["OMP_NUM_THREADS"] = "1"     # inherited by the spawned workers
    ctx = mp.get_context("spawn")
    with ctx.Pool(os.cpu_count() or 1) as pool:
        for nm in names:
            fname, fn = FILES[nm]
            t0 = time.perf_counter()
            data = fn(pool)
            out = os.path.join(HERE, fname)
            with open(out, "w") as fh:
                json.dump(data, fh)
            print(f"wrote {out} ({time.perf_counter() - t0:.0f} s)", flush=True)
