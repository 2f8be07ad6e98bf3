"""PyTorch autograd for the circuit cost, with the library's adjoint kernels.

``circuit_cost(gates, ctx)`` returns ``f(G) = -Re Tr[U^dagger C(G)]``
(Eq. f_target) for a complex128 CUDA tensor ``gates`` of shape
``[n_params, 4, 4]``; its backward is the device backward sweep (the paper's
backward pass with gate holes, Fig. backward_pass_gate_gradient) and its
double backward the device Hessian-vector product (Appendix "Evaluating
Hessian-vector products").

Gradients follow PyTorch's convention for a real loss of complex inputs,
``dL/dx + i dL/dy``, which is the paper's gradient convention (Eq. def_grad).
They are *Euclidean*: the cost is extended to all complex matrices, so
``gates.grad`` is ``gbar`` of Eq. grad_proj before the tangent projection
(a Riemannian optimiser projects it; the library's own Riemannian outputs
are those of ``rq_set_gradient_space(ctx, RQ_SPACE_RIEMANNIAN)``).
For parity-structured circuits the cost is restricted to the pattern of
Eq. paritygatematrix, so gradients and HVPs are masked to it.

Every evaluation is stream-ordered on the library context's stream; the
functions synchronise that stream with the current torch stream.
"""
from __future__ import annotations

import torch


def _euclidean(ctx):
    if getattr(ctx, "_space", None) != 1:
        ctx.set_gradient_space(1)


def _run(ctx, fn):
    cur = torch.cuda.current_stream()
    lib_stream = ctx.stream_handle()
    if lib_stream is not None and lib_stream != cur.cuda_stream:
        ev = torch.cuda.Event()
        ev.record(cur)
        ext = torch.cuda.ExternalStream(lib_stream)
        ext.wait_event(ev)
        fn()
        ev2 = torch.cuda.Event()
        ev2.record(ext)
        cur.wait_event(ev2)
    else:
        fn()


def _check(gates):
    if not (gates.is_cuda and gates.dtype == torch.complex128 and gates.dim() == 3 and gates.shape[1:] == (4, 4)):
        raise TypeError("gates must be a complex128 CUDA tensor of shape [n_params, 4, 4]")
    return gates.contiguous()


class _EuclidGrad(torch.autograd.Function):
    """``gates -> gbar(gates)``; its VJP with cotangent V is the Euclidean
    Hessian applied to V (the real Hessian is symmetric)."""

    @staticmethod
    def forward(actx, gates, ctx):
        gates = _check(gates)
        _euclidean(ctx)
        f = torch.zeros(1, dtype=torch.float64, device=gates.device)
        g = torch.empty_like(gates)
        _run(ctx, lambda: ctx.grad_dev(gates.data_ptr(), f.data_ptr(), g.data_ptr()))
        actx.save_for_backward(gates)
        actx.rq = ctx
        return g

    @staticmethod
    def backward(actx, v):
        (gates,) = actx.saved_tensors
        ctx = actx.rq
        _euclidean(ctx)
        v = v.contiguous().to(torch.complex128)
        f = torch.zeros(1, dtype=torch.float64, device=gates.device)
        g = torch.empty_like(gates)
        h = torch.empty_like(gates)
        _run(ctx, lambda: ctx.hvp_dev(gates.data_ptr(), v.data_ptr(), 1, f.data_ptr(), g.data_ptr(), h.data_ptr()))
        return h, None


class _Cost(torch.autograd.Function):
    @staticmethod
    def forward(actx, gates, ctx):
        gates = _check(gates)
        _euclidean(ctx)
        f = torch.zeros(1, dtype=torch.float64, device=gates.device)
        g = torch.empty_like(gates)
        _run(ctx, lambda: ctx.grad_dev(gates.data_ptr(), f.data_ptr(), g.data_ptr()))
        actx.save_for_backward(gates, g)
        actx.rq = ctx
        return f[0]

    @staticmethod
    def backward(actx, gf):
        gates, g = actx.saved_tensors
        if torch.is_grad_enabled():
            # double backward requested: a differentiable gradient
            g = _EuclidGrad.apply(gates, actx.rq)
        return gf * g, None


def circuit_cost(gates: torch.Tensor, ctx) -> torch.Tensor:
    """Differentiable ``f(G)`` over the context's column range (0-dim float64)."""
    return _Cost.apply(gates, ctx)
