"""Admission order of the request server (host logic, no GPU)."""
import workloads as w
from paper_2506_23775_gb300 import serve


def _req(rid, L, depth, kind, arrival):
    return serve.Request(rid=rid, kind=kind, problem=w.make_problem(L, depth, 0.5, seed=rid), arrival=arrival)


def test_work_estimate_orders_kinds_and_sizes():
    small_cost = _req(0, 4, 3, "cost", 0.0)
    small_hvp = _req(1, 4, 3, "hvp", 0.0)
    big_cost = _req(2, 7, 3, "cost", 0.0)
    assert serve.work_flops(small_hvp) == 9 * serve.work_flops(small_cost)
    assert serve.work_flops(big_cost) == serve.work_flops(small_cost) * 4 ** 6 * \
        big_cost.problem.n_gates / small_cost.problem.n_gates


def test_shortest_first_without_aging():
    reqs = [_req(0, 7, 3, "hvp", 0.0), _req(1, 4, 3, "cost", 5.0), _req(2, 5, 3, "grad", 2.0)]
    order = sorted(reqs, key=lambda r: serve.admission_key(r, 10.0, 0.0, 1.2e12))
    assert [r.rid for r in order] == [1, 2, 0]


def test_aging_lets_a_long_waiting_large_request_through():
    big = _req(0, 7, 3, "hvp", 0.0)
    small = _req(1, 4, 3, "cost", 0.0)
    est = serve.work_flops(big) / 1.2e12
    # fresh: the small request goes first
    assert serve.admission_key(small, 0.0, 1.0, 1.2e12) < serve.admission_key(big, 0.0, 1.0, 1.2e12)
    # the big one has waited longer than its estimated work: it overtakes a new small one
    small_new = _req(2, 4, 3, "cost", 2.0 * est)
    t = 2.0 * est
    assert serve.admission_key(big, t, 1.0, 1.2e12) < serve.admission_key(small_new, t, 1.0, 1.2e12)
    # without aging it never does
    assert serve.admission_key(big, t, 0.0, 1.2e12) > serve.admission_key(small_new, t, 0.0, 1.2e12)


def test_gpu_width_with_a_sweep_grid():
    """Width = threads of the sweep's CTAs over two 256-thread CTAs per SM;
    a grid of m items per thread cuts the CTAs of a large sweep, not of a
    sweep that already has fewer items than threads."""
    p = w.make_problem(6, 3, 0.5, seed=1)      # n = 12: 1024 items per column
    full = serve.gpu_width(p, 128, sms=152)    # 131072 items: 1.68 GPUs of threads
    assert full == 1.0
    narrow = serve.gpu_width(p, 128, sms=152, grid=32)
    assert narrow == 16 * 256 / (152 * 2 * 256)  # ceil(131072 / (256 * 32)) = 16 CTAs
    small = w.make_problem(3, 3, 0.5, seed=2)  # n = 6: 16 items per column
    assert serve.gpu_width(small, 4, sms=152, grid=8) == serve.gpu_width(small, 4, sms=152) == 64 / (152 * 512)
