"""Column shards on real device contexts: two gloo ranks, both on GPU 0.

Each rank evaluates its contiguous column range with its own context (its
own stream and workspace; no kernel of one rank waits on the other), the
packed partials are exchanged by one all-gather and summed in rank order on
the host.  Both the host-memory path (``sharded_eval``) and the
device-pointer path (``DeviceShard``: the library writes the partial straight
into the buffer the all-gather sends) must give the unsharded device result
to 1e-13.
"""
import os
import socket

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASES = {"small": ("small", 0, 3), "tied12": ("tied12", 1, 1)}


def _rank(rank, world, port, case, out_path):
    import torch.distributed as dist
    from paper_2506_23775_gb300 import rq, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    name, structure, k = CASES[case]
    prob = w.config_problem(name, structure=structure)
    X = w.random_directions(prob.n_params, k, 77)
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ctx = rq.Context(0, stream=stream.cuda_stream).setup_problem(prob)
    n_cols = 1 << prob.n
    host = shard.sharded_eval(shard.context_evaluator(ctx, prob.gates, X), n_cols, prob.n_params, k)
    # device pointers: the partial lands in the buffer that is gathered
    ds = shard.DeviceShard(ctx, prob.n_params, k, torch.device("cuda", 0))
    g_d = torch.from_numpy(prob.gates.copy()).cuda()
    x_d = torch.from_numpy(X.copy()).cuda()
    ctx.set_columns(*shard.column_shard(n_cols, rank, world))
    ds.evaluate(g_d.data_ptr(), x_d.data_ptr())
    dev = ds.total(stream=stream)
    if rank == 0:
        np.savez(out_path, hf=host[0], hg=host[1], hh=host[2], df=dev[0], dg=dev[1], dh=dev[2])
    dist.barrier()
    ctx.close()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", sorted(CASES))
def test_two_ranks_on_one_gpu_match_unsharded(rq, tmp_path, case):
    import torch.multiprocessing as mp
    out = str(tmp_path / "r.npz")
    mp.spawn(_rank, args=(2, _free_port(), case, out), nprocs=2, join=True)
    name, structure, k = CASES[case]
    prob = w.config_problem(name, structure=structure)
    X = w.random_directions(prob.n_params, k, 77)
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        f, g, hv = ctx.hvp(prob.gates, X)
    r = np.load(out)
    for tag in ("h", "d"):
        assert abs(float(r[tag + "f"]) - f) <= 1e-13 * abs(f), (tag, float(r[tag + "f"]), f)
        for got, ref in ((r[tag + "g"], g), (r[tag + "h"], hv)):
            assert np.linalg.norm(got - ref) <= 1e-13 * max(np.linalg.norm(ref), 1e-6 * 2 ** prob.n), tag
