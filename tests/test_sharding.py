"""Column sharding across ranks: world-size-2 gloo processes on the CPU.

Each rank evaluates its shard (here with the CPU oracle standing in for a
device context) and the partials are summed in rank order; the total must
match the unsharded sum."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2506_23775_gb300 import shard  # noqa: E402


def test_column_shard_partition():
    for n_cols in (1, 7, 256, 65536):
        for world in (1, 2, 3, 8):
            ranges = [shard.column_shard(n_cols, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n_cols
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.column_shard(10, 2, 2)


def test_pack_roundtrip(rng):
    g = rng.standard_normal((5, 4, 4)) + 1j * rng.standard_normal((5, 4, 4))
    h = rng.standard_normal((2, 5, 4, 4)) + 1j * rng.standard_normal((2, 5, 4, 4))
    f, g2, h2 = shard.unpack(shard.pack(1.5, g, h), 5, 2)
    assert f == 1.5 and np.array_equal(g, g2) and np.array_equal(h, h2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import workloads as w
    from tests._helpers import oracle_eval
    prob = w.make_problem(3, 5, 0.4, seed=55)
    X = w.random_directions(prob.n_params, 2, 56)

    def evaluate(c0, c1):
        f, g, hv, _ = oracle_eval(prob, range(c0, c1), X, chunk=64)
        return f, g, hv

    f, g, hv = shard.sharded_eval(evaluate, 1 << prob.n, prob.n_params, 2)
    if rank == 0:
        np.savez(out_path, f=f, g=g, hv=hv)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_sum_matches_unsharded(tmp_path):
    out = str(tmp_path / "res.npz")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    import workloads as w
    from tests._helpers import oracle_eval
    prob = w.make_problem(3, 5, 0.4, seed=55)
    X = w.random_directions(prob.n_params, 2, 56)
    f, g, hv, _ = oracle_eval(prob, range(1 << prob.n), X, chunk=64)
    r = np.load(out)
    assert abs(float(r["f"]) - f) <= 1e-13 * abs(f)
    np.testing.assert_allclose(r["g"], g, atol=1e-13 * np.abs(g).max())
    np.testing.assert_allclose(r["hv"], hv, atol=1e-13 * np.abs(hv).max())


def _exchange_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    part = torch.arange(7, dtype=torch.float64) * (rank + 1) + 0.1 * rank
    total = shard.exchange(part)
    if rank == 0:
        np.save(out_path, total)
    dist.barrier()
    dist.destroy_process_group()


def test_exchange_sums_partials_in_rank_order(tmp_path):
    out = str(tmp_path / "x.npy")
    mp.spawn(_exchange_worker, args=(3, _free_port(), out), nprocs=3, join=True)
    rows = [np.arange(7, dtype=np.float64) * (r + 1) + 0.1 * r for r in range(3)]
    assert np.array_equal(np.load(out), (rows[0] + rows[1]) + rows[2])


def _failing_worker(rank, world, port, out_path):
    import datetime
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    if rank == 1:
        # this rank fails on the host before the exchange (no device work in flight)
        os._exit(3)
    try:
        shard.sharded_eval(lambda c0, c1: (1.0, np.zeros((1, 4, 4), np.complex128), None), 16, 1, 0)
        status = "completed"
    except Exception as e:  # the surviving rank learns of the failure from the collective
        status = "error: " + type(e).__name__
    with open(out_path, "w") as fh:
        fh.write(status)
    os._exit(0)


def test_a_failed_rank_is_reported_not_hung(tmp_path):
    import subprocess
    import sys
    import time
    out = str(tmp_path / "status.txt")
    port = _free_port()
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from tests.test_sharding import _failing_worker\n"
        "import torch.multiprocessing as mp\n"
        "mp.start_processes(_failing_worker, args=(2, %d, %r), nprocs=2, join=False, start_method='spawn')\n"
        "import time; time.sleep(0.1)\n" % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))), port, out))
    t0 = time.time()
    proc = subprocess.Popen([sys.executable, "-c", code])
    deadline = t0 + 120
    while time.time() < deadline and not os.path.exists(out):
        time.sleep(0.2)
    proc.wait(timeout=30)
    assert os.path.exists(out), "the surviving rank neither finished nor reported the failure"
    assert open(out).read().startswith("error"), open(out).read()
