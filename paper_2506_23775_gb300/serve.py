"""Continuous-batching request loop for cost / gradient / HVP requests.

Requests for problems of different sizes arrive over time.  The server admits
a request as soon as a slot and enough device memory are free (admission by
HBM footprint: the problem's target blocks plus its sweep workspace), queues
its evaluation at once on that request's own CUDA stream -- so requests that
arrive while others are on the GPU run concurrently with them -- and returns
each result when its completion event fires.  Target blocks and workspaces
stay on the device between requests for the same problem (a context cache),
so repeated requests skip the set-up; new contexts are built by host worker
threads while the loop keeps admitting and collecting work.

Every evaluation runs the library's kernels in the same order as the same
request evaluated alone on a context with the same tile size and sweep grid,
so a result in the mix equals the result alone bit for bit.  With a sweep
grid of m items per thread (rq_set_grid) each request's sweeps take fewer
CTAs, so more requests share the GPU at once and each pays its per-CTA
costs fewer times.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from math import comb
from typing import Dict, List, Optional

import numpy as np


@dataclass
class Request:
    rid: int
    kind: str                 # "cost" | "grad" | "hvp"
    problem: object           # workloads.Problem (topology, target parameters, gates)
    dirs: Optional[np.ndarray] = None
    arrival: float = 0.0      # seconds after the start of the stream
    # filled by the server
    admitted: float = float("nan")
    done: float = float("nan")
    f: float = float("nan")
    rgrad: Optional[np.ndarray] = None
    hvps: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def problem_key(p) -> tuple:
    return (p.L, p.periodic, p.J, p.U, p.t, p.structure, p.n_params,
            p.pairs.tobytes(), p.param_of.tobytes())


def work_flops(req: "Request") -> float:
    """FP64 flops of one request: 1 / 3 / 9 gate passes per gate for cost /
    gradient / HVP, 32 flops per amplitude and column (a quarter for parity
    gates), over the full basis."""
    p = req.problem
    units = {"cost": 1, "grad": 3, "hvp": 9}[req.kind]
    return units * p.n_gates * 32.0 * 4.0 ** p.n / (4.0 if p.structure == 1 else 1.0)


def admission_key(req: "Request", now: float, aging: float, fp64_flops_per_s: float) -> float:
    """Shortest-work-first order with aging: estimated seconds of work minus
    ``aging`` times the seconds the request has waited (smaller = sooner)."""
    return work_flops(req) / fp64_flops_per_s - aging * (now - req.arrival)


def gpu_width(p, tile: int, sms: int = 152, grid: int = 0) -> float:
    """Fraction of the GPU one sweep kernel of this problem fills (its items
    over two 256-thread CTAs per SM; with a sweep grid of ``grid`` items per
    thread, the threads of its CTAs)."""
    n_store = (1 << (p.n - 1)) if p.structure == 1 else (1 << p.n)
    items = n_store / 4 * tile
    if grid > 0:
        items = min(items, -(-items // (256 * grid)) * 256)
    return min(1.0, items / (sms * 2 * 256))


def footprint_bytes(p, tile: int, k: int = 1) -> int:
    """Device bytes of a problem's context: target blocks, tables, workspace."""
    n_store = (1 << (p.n - 1)) if p.structure == 1 else (1 << p.n)
    target = comb(2 * p.L, p.L) ** 2 * 16 + 3 * (1 << p.n) * 4
    sets = (1 + k) * (p.n_gates + 1) + 1 + k
    return int(target + tile * sets * n_store * 16)


class _Slot:
    def __init__(self, ctx, stream, key, tile, nbytes):
        self.ctx, self.stream, self.key, self.tile, self.nbytes = ctx, stream, key, tile, nbytes
        self.busy = False
        self.last_used = 0.0


class Server:
    """Continuous batching over per-problem device contexts.

    ``memory_budget``: bytes of device memory the server may hold;
    ``max_inflight``: evaluations on the GPU at once; ``tile``: columns per
    tile of every context (a power of two; smaller tiles lower the footprint);
    ``contexts_per_problem``: contexts one problem may hold at once (several
    requests for the same problem then run concurrently); ``setup_workers``:
    host threads that build new contexts (target blocks) while the loop keeps
    admitting and collecting work.  ``policy``: "fifo" (arrival order) or
    "sjf" (shortest estimated work first); ``aging``: with "sjf", seconds of
    estimated work forgiven per second a request has waited, so a large
    request cannot wait forever behind a stream of small ones (0: pure
    shortest-first).  ``grid``: sweep grid of every context (rq_set_grid:
    0 fills the GPU per sweep; m > 0 at most the CTAs that give each thread m
    items, so that concurrent requests share the GPU).
    """

    def __init__(self, device: int = 0, memory_budget: Optional[int] = None, max_inflight: int = 8,
                 tile: int = 128, contexts_per_problem: int = 2, setup_workers: int = 2,
                 policy: str = "sjf", aging: float = 0.0, fp64_flops_per_s: float = 1.2e12,
                 grid: int = 0):
        import concurrent.futures as cf

        import torch
        from . import rq
        self.torch, self.rq = torch, rq
        self.device = device
        self.dev = torch.device("cuda", device)
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            memory_budget = int(0.5 * free)
        self.budget = memory_budget
        self.max_inflight = max_inflight
        self.tile = tile
        self.grid = grid
        self.per_problem = contexts_per_problem
        self.slots: Dict[tuple, List[_Slot]] = collections.defaultdict(list)
        self.building: Dict[tuple, list] = collections.defaultdict(list)   # futures of contexts being set up
        self.held = 0
        self.stats = collections.Counter()
        self.pool = cf.ThreadPoolExecutor(max_workers=setup_workers)
        self.policy = policy
        self.aging = aging
        self.rate = fp64_flops_per_s   # converts work_flops into estimated seconds
        self.sms = torch.cuda.get_device_properties(self.dev).multi_processor_count

    # -- contexts ----------------------------------------------------------
    def _evict_idle(self, need: int) -> bool:
        idle = sorted((s.last_used, id(s), s) for lst in self.slots.values() for s in lst if not s.busy)
        for _, _, s in idle:
            if self.held + need <= self.budget:
                break
            s.ctx.close()
            self.held -= s.nbytes
            self.slots[s.key].remove(s)
            self.stats["evicted"] += 1
        return self.held + need <= self.budget

    def _build(self, p, key, tile, need):
        self.torch.cuda.set_device(self.dev)
        stream = self.torch.cuda.Stream(device=self.dev)
        ctx = self.rq.Context(self.device, stream=stream.cuda_stream).setup_problem(p)
        ctx.set_tile(tile, 1)
        if self.grid:
            ctx.set_grid(self.grid)
        return _Slot(ctx, stream, key, tile, need)

    def _harvest_builds(self):
        for key, futs in self.building.items():
            done = [fu for fu in futs if fu.done()]
            for fu in done:
                futs.remove(fu)
                self.slots[key].append(fu.result())   # re-raises a failed set-up
                self.stats["setups"] += 1

    def _slot_for(self, req: Request) -> Optional[_Slot]:
        p = req.problem
        key = problem_key(p)
        for s in self.slots[key]:
            if not s.busy:
                self.stats["reused"] += 1
                return s
        if len(self.slots[key]) + len(self.building[key]) >= self.per_problem:
            return None                       # wait for one of this problem's contexts
        if self.building[key]:
            return None                       # one set-up at a time per problem
        tile = min(self.tile, 1 << p.n)
        k = 0 if req.dirs is None else req.dirs.shape[0]
        need = footprint_bytes(p, tile, max(k, 1))
        if need > self.budget:
            raise MemoryError(f"request {req.rid} needs {need} bytes, the budget is {self.budget}")
        if not self._evict_idle(need):
            return None
        self.held += need
        self.building[key].append(self.pool.submit(self._build, p, key, tile, need))
        return None

    # -- one evaluation, queued on the slot's stream ------------------------
    def _launch(self, req: Request, s: _Slot):
        torch = self.torch
        p = req.problem
        with torch.cuda.stream(s.stream):
            g = torch.from_numpy(np.ascontiguousarray(p.gates)).to(self.dev, non_blocking=False)
            f = torch.zeros(1, dtype=torch.float64, device=self.dev)
            rg = torch.zeros_like(g)
            if req.kind == "hvp":
                d = torch.from_numpy(np.ascontiguousarray(req.dirs)).to(self.dev)
                hv = torch.zeros_like(d)
        # the library runs on the same stream, so the copies above precede its kernels
        if req.kind == "cost":
            s.ctx.cost_dev(g.data_ptr(), f.data_ptr())
            out = (f, None, None)
        elif req.kind == "grad":
            s.ctx.grad_dev(g.data_ptr(), f.data_ptr(), rg.data_ptr())
            out = (f, rg, None)
        else:
            s.ctx.hvp_dev(g.data_ptr(), d.data_ptr(), req.dirs.shape[0], f.data_ptr(), rg.data_ptr(),
                          hv.data_ptr())
            out = (f, rg, hv)
        ev = torch.cuda.Event()
        ev.record(s.stream)
        return ev, out

    def run(self, requests: List[Request], realtime: bool = True) -> Dict[str, float]:
        """Serve ``requests`` (sorted by arrival).  ``realtime``: honour the
        arrival times; otherwise every request is available at once."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        inflight = []
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        waiting: List[Request] = []
        while pending or waiting or inflight or any(self.building.values()):
            t = now()
            while pending and (not realtime or pending[0].arrival <= t):
                waiting.append(pending.popleft())
            self._harvest_builds()
            # admit as slots and memory allow.  "fifo": arrival order.  "sjf":
            # shortest work first, and a new request joins only while the
            # in-flight sweeps do not already fill the GPU (a saturated FP64
            # pipe gains nothing from overlap, and sharing it delays everyone).
            # A request whose problem has no free context does not block others.
            if self.policy == "sjf":
                waiting.sort(key=lambda r: admission_key(r, t, self.aging, self.rate))
            width = sum(gpu_width(r.problem, s.tile, self.sms, self.grid) for r, s, _, _ in inflight)
            still = []
            for req in waiting:
                if len(inflight) >= self.max_inflight or (self.policy == "sjf" and inflight and width >= 1.0):
                    still.append(req)
                    continue
                s = self._slot_for(req)
                if s is None:
                    still.append(req)
                    continue
                s.busy = True
                req.admitted = now()
                ev, out = self._launch(req, s)
                inflight.append((req, s, ev, out))
                width += gpu_width(req.problem, s.tile, self.sms, self.grid)
            waiting = still
            # collect finished work
            rest = []
            for item in inflight:
                req, s, ev, out = item
                if ev.query():
                    f, rg, hv = out
                    req.f = float(f.item())
                    req.rgrad = None if rg is None else rg.cpu().numpy()
                    req.hvps = None if hv is None else hv.cpu().numpy()
                    req.done = now()
                    s.busy = False
                    s.last_used = req.done
                else:
                    rest.append(item)
            inflight = rest
            if inflight or waiting or pending or any(self.building.values()):
                time.sleep(0.0005)
        wall = now()
        lat = np.array([r.latency for r in requests])
        return {"requests": len(requests), "wall_s": wall, "evals_per_s": len(requests) / wall,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "setups": self.stats["setups"], "reused": self.stats["reused"], "evicted": self.stats["evicted"]}

    def close(self):
        self.pool.shutdown(wait=True)
        self._harvest_builds()
        for lst in self.slots.values():
            for s in lst:
                s.ctx.close()
        self.slots.clear()
        self.held = 0


def poisson_stream(problems, kinds, rate_hz: float, seed: int, k: int = 1) -> List[Request]:
    """Requests over ``problems`` with exponential inter-arrival times."""
    import workloads as w
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i, (p, kind) in enumerate(zip(problems, kinds)):
        t += rng.exponential(1.0 / rate_hz)
        dirs = w.random_directions(p.n_params, k, seed * 1000 + i) if kind == "hvp" else None
        out.append(Request(rid=i, kind=kind, problem=p, dirs=dirs, arrival=t))
    return out
