"""Every output entry is written: outputs poisoned with NaN before a call
come back finite and equal to the results into fresh buffers (host and
device-pointer entry points, general and parity gates, several tiles and
direction chunks, the sweep grid of a shared GPU)."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    from paper_2506_23775_gb300 import _build, rq
    _build.build()
    return rq


@pytest.mark.parametrize("structure,tile,dirs_per_sweep,grid", [
    (0, 0, 0, 0),      # automatic tile: one tile of all 256 columns
    (0, 64, 1, 0),     # four tiles, three direction chunks
    (1, 32, 2, 8),     # parity gates: even and odd tiles, two chunks, a narrow grid
])
def test_poisoned_outputs_are_overwritten(rq, structure, tile, dirs_per_sweep, grid):
    torch = pytest.importorskip("torch")
    prob = w.make_problem(4, 5, 0.25, seed=101, structure=structure)
    X = w.random_directions(prob.n_params, 3, 102)
    with rq.Context(0) as ctx:
        ctx.setup_problem(prob)
        ctx.set_tile(tile, dirs_per_sweep)
        ctx.set_grid(grid)
        f, g, hv = ctx.hvp(prob.gates, X)
        assert np.isfinite(f) and np.isfinite(g).all() and np.isfinite(hv).all()
        # host entry points into caller arrays full of NaN
        rg = np.full_like(g, np.nan)
        hvo = np.full_like(hv, np.nan)
        f1, rg, hvo = ctx.hvp(prob.gates, X, out=(rg, hvo))
        assert f1 == f and np.array_equal(rg, g) and np.array_equal(hvo, hv)
        # device-pointer entry points into device buffers full of NaN
        dev = torch.device("cuda:0")
        tg = torch.from_numpy(prob.gates.copy()).to(dev)
        tx = torch.from_numpy(X.copy()).to(dev)
        tf = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        trg = torch.full(tuple(g.shape), complex("nan+nanj"), dtype=torch.complex128, device=dev)
        thv = torch.full(tuple(hv.shape), complex("nan+nanj"), dtype=torch.complex128, device=dev)
        ctx.hvp_dev(tg.data_ptr(), tx.data_ptr(), 3, tf.data_ptr(), trg.data_ptr(), thv.data_ptr())
        torch.cuda.synchronize()
        assert tf.item() == f
        assert np.array_equal(trg.cpu().numpy(), g) and np.array_equal(thv.cpu().numpy(), hv)
        tf.fill_(float("nan"))
        trg.fill_(complex("nan+nanj"))
        ctx.grad_dev(tg.data_ptr(), tf.data_ptr(), trg.data_ptr())
        torch.cuda.synchronize()
        fg, gg = ctx.grad(prob.gates)
        assert tf.item() == fg and np.array_equal(trg.cpu().numpy(), gg)
        tf.fill_(float("nan"))
        ctx.cost_dev(tg.data_ptr(), tf.data_ptr())
        torch.cuda.synchronize()
        assert tf.item() == ctx.cost(prob.gates)
        if structure == 1:   # entries outside the parity pattern come back as exact zeros
            mask = ~w.parity_mask()
            assert not np.any(g[:, mask]) and not np.any(hv[:, :, mask])
