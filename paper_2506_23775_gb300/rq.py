"""Thin ctypes binding of the ``rq`` C ABI (``include/rq.h``).

Argument marshalling only: every step of the cost, gradient, HVP and
trust-region computation runs inside ``librq.so`` on the GPU.  Importing this
module does not load the library; the first :class:`Context` does, and it
raises if the library is missing (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Tuple

import numpy as np

_LIB = None
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "librq.so")

RQ_OK, RQ_EINVAL, RQ_ENOMEM, RQ_ECUDA, RQ_ETIMEOUT, RQ_ESTATE = 0, -1, -2, -3, -4, -5

# Every symbol declared in include/rq.h.
EXPORTS = ("rq_create", "rq_destroy", "rq_setup_target", "rq_set_columns", "rq_set_tile", "rq_set_grid",
           "rq_cost", "rq_grad", "rq_hvp", "rq_cost_dev", "rq_grad_dev", "rq_hvp_dev",
           "rq_tr_step", "rq_target_column", "rq_get_info", "rq_profile_start", "rq_profile_stop",
           "rq_cost_static", "rq_set_gradient_space", "rq_batch_create", "rq_batch_destroy",
           "rq_batch_add", "rq_batch_set_tile", "rq_batch_set_grid", "rq_batch_grid_info", "rq_batch_hvp", "rq_batch_info", "rq_batch_last_error",
           "rq_batch_set_fusion", "rq_batch_fusion_info",
           "rq_set_arithmetic", "rq_set_translation", "rq_hessian", "rq_set_checkpointing",
           "rq_set_graphs", "rq_set_checks", "rq_set_first_layer", "rq_set_last_layer", "rq_set_fusion", "rq_fusion_info",
           "rq_last_error")


class RQCircuit(C.Structure):
    _fields_ = [("n_qubits", C.c_int), ("n_gates", C.c_int), ("n_params", C.c_int),
                ("structure", C.c_int), ("pairs", C.POINTER(C.c_int32)),
                ("param_of", C.POINTER(C.c_int32))]


class RQTarget(C.Structure):
    _fields_ = [("model", C.c_int), ("n_sites", C.c_int), ("periodic", C.c_int),
                ("J", C.c_double), ("U", C.c_double), ("t", C.c_double),
                ("dense_U", C.POINTER(C.c_double))]


class RQTRState(C.Structure):
    _fields_ = [("radius", C.c_double), ("max_radius", C.c_double), ("rho_accept", C.c_double),
                ("kappa", C.c_double), ("theta", C.c_double), ("max_inner", C.c_int),
                ("f", C.c_double), ("f_new", C.c_double), ("rho", C.c_double),
                ("grad_norm", C.c_double), ("step_norm", C.c_double), ("accepted", C.c_int),
                ("n_inner", C.c_int), ("tcg_exit", C.c_int), ("full_hessian", C.c_int)]


class RQInfo(C.Structure):
    _fields_ = [("n_qubits", C.c_int), ("n_gates", C.c_int), ("n_params", C.c_int),
                ("structure", C.c_int), ("amplitudes_per_column", C.c_int64),
                ("columns", C.c_int64), ("columns_per_tile", C.c_int), ("n_tiles", C.c_int),
                ("max_dirs", C.c_int), ("workspace_bytes", C.c_int64),
                ("target_entries", C.c_int64), ("kernel_launches", C.c_int64),
                ("ctas_per_sweep", C.c_int)]


class RQKernelStat(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_int64), ("total_ms", C.c_double),
                ("flops", C.c_double), ("bytes", C.c_double)]


class RQError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rq error {code}: {msg}")
        self.code = code


def load(path: Optional[str] = None) -> C.CDLL:
    """Load ``librq.so`` (raises ``OSError`` if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    vp, dp, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int64
    sig = {
        "rq_create": ([C.POINTER(vp), C.c_int, vp], C.c_int),
        "rq_destroy": ([vp], C.c_int),
        "rq_setup_target": ([vp, C.POINTER(RQTarget), C.POINTER(RQCircuit)], C.c_int),
        "rq_set_columns": ([vp, i64, i64], C.c_int),
        "rq_set_tile": ([vp, C.c_int, C.c_int], C.c_int),
        "rq_set_grid": ([vp, C.c_int], C.c_int),
        "rq_cost": ([vp, dp, dp], C.c_int),
        "rq_grad": ([vp, dp, dp, dp], C.c_int),
        "rq_hvp": ([vp, dp, dp, C.c_int, dp, dp, dp], C.c_int),
        "rq_cost_dev": ([vp, vp, vp], C.c_int),
        "rq_grad_dev": ([vp, vp, vp, vp], C.c_int),
        "rq_hvp_dev": ([vp, vp, vp, C.c_int, vp, vp, vp], C.c_int),
        "rq_tr_step": ([vp, dp, C.POINTER(RQTRState)], C.c_int),
        "rq_target_column": ([vp, i64, dp], C.c_int),
        "rq_get_info": ([vp, C.POINTER(RQInfo)], C.c_int),
        "rq_profile_start": ([vp], C.c_int),
        "rq_cost_static": ([vp, dp, dp], C.c_int),
        "rq_set_gradient_space": ([vp, C.c_int], C.c_int),
        "rq_set_arithmetic": ([vp, C.c_int], C.c_int),
        "rq_set_translation": ([vp, C.c_int], C.c_int),
        "rq_hessian": ([vp, dp, dp, dp, dp], C.c_int),
        "rq_set_checkpointing": ([vp, C.c_int], C.c_int),
        "rq_set_graphs": ([vp, C.c_int], C.c_int),
        "rq_set_checks": ([vp, C.c_int], C.c_int),
        "rq_set_first_layer": ([vp, C.c_int], C.c_int),
        "rq_set_last_layer": ([vp, C.c_int], C.c_int),
        "rq_set_fusion": ([vp, C.c_int], C.c_int),
        "rq_fusion_info": ([vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
        "rq_batch_create": ([C.POINTER(vp), C.c_int], C.c_int),
        "rq_batch_destroy": ([vp], C.c_int),
        "rq_batch_add": ([vp, C.POINTER(RQTarget), C.POINTER(RQCircuit), C.POINTER(C.c_int)], C.c_int),
        "rq_batch_set_tile": ([vp, C.c_int], C.c_int),
        "rq_batch_set_grid": ([vp, C.c_int], C.c_int),
        "rq_batch_grid_info": ([vp, C.POINTER(C.c_int), C.POINTER(C.c_double)], C.c_int),
        "rq_batch_hvp": ([vp, dp, dp, C.c_int, C.c_int, dp, dp, dp], C.c_int),
        "rq_batch_info": ([vp, C.POINTER(C.c_int), C.POINTER(C.c_int), dp], C.c_int),
        "rq_batch_last_error": ([vp], C.c_char_p),
        "rq_batch_set_fusion": ([vp, C.c_int], C.c_int),
        "rq_batch_fusion_info": ([vp, C.POINTER(C.c_int), dp], C.c_int),
        "rq_profile_stop": ([vp, C.POINTER(RQKernelStat), C.c_int, C.POINTER(C.c_int)], C.c_int),
        "rq_last_error": ([vp], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = lib
    return lib


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


class Context:
    """One device context: a target, a circuit and a column range."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        self._lib = load()
        h = C.c_void_p()
        st = self._lib.rq_create(C.byref(h), device, C.c_void_p(stream) if stream else None)
        if st != RQ_OK:
            raise RQError(st, self._lib.rq_last_error(None).decode())
        self._h = h
        self._stream = stream or None
        self._space = 0
        self.n_params = 0
        self.n_qubits = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rq_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int):
        if st != RQ_OK:
            raise RQError(st, self._lib.rq_last_error(self._h).decode())

    # --- set-up ---------------------------------------------------------
    def setup(self, n_sites: int, pairs, param_of=None, n_params: Optional[int] = None,
              structure: int = 0, J: float = 1.0, U: float = 4.0, t: float = 0.5,
              periodic: bool = False, model: int = 0, dense_U=None, n_qubits: Optional[int] = None):
        """Chain targets (model 0 spinful, 1 spinless) from (n_sites, J, U, t,
        periodic); model 2 takes a dense ``dense_U`` (2^n x 2^n complex) and
        ``n_qubits`` instead."""
        pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        self._pairs = pairs
        if param_of is not None:
            self._param_of = np.ascontiguousarray(param_of, dtype=np.int32)
            npar = int(n_params if n_params is not None else self._param_of.max() + 1)
            pp = self._param_of.ctypes.data_as(C.POINTER(C.c_int32))
        else:
            self._param_of = None
            npar = pairs.shape[0]
            pp = None
        dptr = None
        if model == 2:
            dense = np.ascontiguousarray(dense_U, dtype=np.complex128)
            nq = int(n_qubits) if n_qubits is not None else int(round(np.log2(dense.shape[0])))
            if dense.shape != (1 << nq, 1 << nq):
                raise ValueError(f"dense_U must be {1 << nq} x {1 << nq}, got {dense.shape}")
            dptr = dense.ctypes.data_as(C.POINTER(C.c_double))
        else:
            nq = (2 if model == 0 else 1) * n_sites
        circ = RQCircuit(nq, pairs.shape[0], npar, structure,
                         pairs.ctypes.data_as(C.POINTER(C.c_int32)), pp)
        tgt = RQTarget(model, n_sites, 1 if periodic else 0, J, U, t, dptr)
        self._check(self._lib.rq_setup_target(self._h, C.byref(tgt), C.byref(circ)))
        self.n_params, self.n_qubits, self.structure = npar, nq, structure
        return self

    def setup_problem(self, prob):
        """Set up from a ``workloads.Problem``."""
        return self.setup(prob.L, prob.pairs, prob.param_of, prob.n_params, prob.structure,
                          prob.J, prob.U, prob.t, prob.periodic, getattr(prob, "model", 0))

    def set_gradient_space(self, space: int):
        """0: Riemannian outputs (default); 1: Euclidean gradient and Hessian."""
        self._check(self._lib.rq_set_gradient_space(self._h, int(space)))
        self._space = int(space)

    def set_arithmetic(self, arith: int):
        """0: FP64 sweeps (default); 1: double-float sweeps on the FP32 pipe."""
        self._check(self._lib.rq_set_arithmetic(self._h, int(arith)))

    def set_checkpointing(self, interval: int):
        """Keep the forward state every ``interval`` gates (1: every gate) and
        recompute the rest in the backward pass."""
        self._check(self._lib.rq_set_checkpointing(self._h, int(interval)))

    def set_first_layer(self, enable: bool):
        """Sweep only the nonzero items of the first layer's gates (default on)."""
        self._check(self._lib.rq_set_first_layer(self._h, 1 if enable else 0))

    def set_last_layer(self, enable: bool):
        """Skip the zero-adjoint items of the last layer's gates in the backward sweep (default on)."""
        self._check(self._lib.rq_set_last_layer(self._h, 1 if enable else 0))

    def set_fusion(self, max_window_qubits: int):
        self._check(self._lib.rq_set_fusion(self._h, int(max_window_qubits)))
        return self

    def fusion_info(self) -> dict:
        n, fg, mx = C.c_int(), C.c_int(), C.c_int()
        self._check(self._lib.rq_fusion_info(self._h, C.byref(n), C.byref(fg), C.byref(mx)))
        return {"passes": n.value, "fused_gates": fg.value, "max_pass_gates": mx.value}

    def set_checks(self, enable: bool):
        """Validate the gates of every call (unitarity, parity pattern)."""
        self._check(self._lib.rq_set_checks(self._h, 1 if enable else 0))

    def set_graphs(self, enable: bool):
        """Capture host-memory evaluations into CUDA graphs (default on)."""
        self._check(self._lib.rq_set_graphs(self._h, 1 if enable else 0))

    def set_translation(self, shift_sites: int):
        """Sum over translation-orbit representatives (0: plain basis sums)."""
        self._check(self._lib.rq_set_translation(self._h, int(shift_sites)))

    def stream_handle(self):
        """The cudaStream_t given at creation (None: a library-owned stream)."""
        return self._stream

    def set_columns(self, begin: int, end: int):
        self._check(self._lib.rq_set_columns(self._h, int(begin), int(end)))

    def set_tile(self, columns_per_tile: int = 0, max_dirs: int = 0):
        self._check(self._lib.rq_set_tile(self._h, int(columns_per_tile), int(max_dirs)))

    def set_grid(self, min_items_per_thread: int):
        """0: sweeps fill the GPU; m > 0: at most the CTAs that give each thread m items."""
        self._check(self._lib.rq_set_grid(self._h, int(min_items_per_thread)))

    def info(self) -> dict:
        i = RQInfo()
        self._check(self._lib.rq_get_info(self._h, C.byref(i)))
        return {name: getattr(i, name) for name, _ in RQInfo._fields_}

    # --- evaluations (host memory) ---------------------------------------
    def cost(self, gates) -> float:
        g = _c128(gates)
        f = C.c_double()
        self._check(self._lib.rq_cost(self._h, _dptr(g.view(np.float64)), C.byref(f)))
        return f.value

    def grad(self, gates) -> Tuple[float, np.ndarray]:
        g = _c128(gates)
        out = np.empty_like(g)
        f = C.c_double()
        self._check(self._lib.rq_grad(self._h, _dptr(g.view(np.float64)), C.byref(f),
                                      _dptr(out.view(np.float64))))
        return f.value, out

    def hvp(self, gates, dirs, out: Optional[Tuple[np.ndarray, np.ndarray]] = None
            ) -> Tuple[float, np.ndarray, np.ndarray]:
        """f, Riemannian gradient and HVPs; ``out=(rgrad, hvps)`` reuses
        caller arrays (for example pinned host memory)."""
        g = _c128(gates)
        d = _c128(dirs).reshape((-1,) + g.shape)
        if out is None:
            rg = np.empty_like(g)
            hv = np.empty_like(d)
        else:
            rg, hv = out
            assert rg.dtype == np.complex128 and rg.shape == g.shape and rg.flags.c_contiguous
            assert hv.dtype == np.complex128 and hv.shape == d.shape and hv.flags.c_contiguous
        f = C.c_double()
        self._check(self._lib.rq_hvp(self._h, _dptr(g.view(np.float64)), _dptr(d.view(np.float64)),
                                     d.shape[0], C.byref(f), _dptr(rg.view(np.float64)),
                                     _dptr(hv.view(np.float64))))
        return f.value, rg, hv

    def cost_static(self, gates) -> float:
        """``f`` like :meth:`cost`, with no device allocation in the call
        (scratch in the library's fixed static device array)."""
        g = _c128(gates)
        f = C.c_double()
        self._check(self._lib.rq_cost_static(self._h, _dptr(g.view(np.float64)), C.byref(f)))
        return f.value

    # --- evaluations (device pointers, stream ordered) ---------------------
    def cost_dev(self, gates_ptr: int, f_ptr: int):
        self._check(self._lib.rq_cost_dev(self._h, C.c_void_p(gates_ptr), C.c_void_p(f_ptr)))

    def grad_dev(self, gates_ptr: int, f_ptr: int, rgrad_ptr: int):
        self._check(self._lib.rq_grad_dev(self._h, C.c_void_p(gates_ptr), C.c_void_p(f_ptr),
                                          C.c_void_p(rgrad_ptr)))

    def hvp_dev(self, gates_ptr: int, dirs_ptr: int, k: int, f_ptr: int, rgrad_ptr: int, hvps_ptr: int):
        self._check(self._lib.rq_hvp_dev(self._h, C.c_void_p(gates_ptr), C.c_void_p(dirs_ptr), int(k),
                                         C.c_void_p(f_ptr), C.c_void_p(rgrad_ptr), C.c_void_p(hvps_ptr)))

    # --- trust region ---------------------------------------------------
    def tr_step(self, gates: np.ndarray, state: RQTRState) -> np.ndarray:
        """One trust-region iteration; returns the (possibly updated) gates."""
        g = _c128(gates).copy()
        self._check(self._lib.rq_tr_step(self._h, _dptr(g.view(np.float64)), C.byref(state)))
        return g

    def profile_start(self):
        self._check(self._lib.rq_profile_start(self._h))

    def profile_stop(self) -> dict:
        """Per-kernel-family launches, device ms, algorithmic flops and bytes."""
        arr = (RQKernelStat * 16)()
        n = C.c_int()
        self._check(self._lib.rq_profile_stop(self._h, arr, 16, C.byref(n)))
        return {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].total_ms,
                                           flops=arr[i].flops, bytes=arr[i].bytes)
                for i in range(min(n.value, 16))}

    def hessian(self, gates):
        """``(f, egrad, H)``: Euclidean gradient and the tied holomorphic
        second derivatives ``H[(p,a,b), (q,c,d)]`` as a ``[16P, 16P]`` array."""
        g = _c128(gates)
        eg = np.empty_like(g)
        D = g.shape[0] * 16
        H = np.empty((D, D), dtype=np.complex128)
        f = C.c_double()
        self._check(self._lib.rq_hessian(self._h, _dptr(g.view(np.float64)), C.byref(f),
                                         _dptr(eg.view(np.float64)), _dptr(H.view(np.float64))))
        return f.value, eg, H

    def target_column(self, j: int) -> np.ndarray:
        out = np.empty(1 << self.n_qubits, dtype=np.complex128)
        self._check(self._lib.rq_target_column(self._h, int(j), _dptr(out.view(np.float64))))
        return out


def tr_state(radius=0.01, max_radius=0.1, rho_accept=0.125, kappa=0.1, theta=1.0, max_inner=0,
             full_hessian=False) -> RQTRState:
    s = RQTRState()
    s.full_hessian = 1 if full_hessian else 0
    s.radius, s.max_radius, s.rho_accept = radius, max_radius, rho_accept
    s.kappa, s.theta, s.max_inner = kappa, theta, max_inner
    return s


class Batch:
    """Independent problems evaluated together (one CUDA-graph launch)."""

    def __init__(self, device: int = 0):
        self._lib = load()
        h = C.c_void_p()
        st = self._lib.rq_batch_create(C.byref(h), device)
        if st != RQ_OK:
            raise RQError(st, "rq_batch_create failed")
        self._h = h
        self.n_params = []
        self._keep = []

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rq_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != RQ_OK:
            raise RQError(st, self._lib.rq_batch_last_error(self._h).decode())

    def add_problem(self, prob) -> int:
        pairs = np.ascontiguousarray(prob.pairs, dtype=np.int32)
        pof = np.ascontiguousarray(prob.param_of, dtype=np.int32)
        circ = RQCircuit(prob.n, pairs.shape[0], prob.n_params, prob.structure,
                         pairs.ctypes.data_as(C.POINTER(C.c_int32)), pof.ctypes.data_as(C.POINTER(C.c_int32)))
        tgt = RQTarget(getattr(prob, "model", 0), prob.L, 1 if prob.periodic else 0, prob.J, prob.U, prob.t)
        idx = C.c_int()
        self._check(self._lib.rq_batch_add(self._h, C.byref(tgt), C.byref(circ), C.byref(idx)))
        self.n_params.append(prob.n_params)
        return idx.value

    def set_tile(self, columns_per_tile: int):
        self._check(self._lib.rq_batch_set_tile(self._h, int(columns_per_tile)))

    def info(self) -> dict:
        n, t = C.c_int(), C.c_int()
        ms = (C.c_double * 4)()
        self._check(self._lib.rq_batch_info(self._h, C.byref(n), C.byref(t), ms))
        q = C.c_int()
        fms = (C.c_double * 4)()
        self._check(self._lib.rq_batch_fusion_info(self._h, C.byref(q), fms))
        m = C.c_int()
        gms = (C.c_double * 5)()
        self._check(self._lib.rq_batch_grid_info(self._h, C.byref(m), gms))
        return {"n_problems": n.value, "columns_per_tile": t.value,
                "tune_ms": dict(zip((64, 128, 256, 512), list(ms))),
                "fusion_window": q.value, "fusion_tune_ms": dict(zip((0, 4, 5, 6), list(fms))),
                "grid_items": m.value, "grid_tune_ms": dict(zip((0, 8, 16, 32, 64), list(gms)))}

    def set_grid(self, min_items_per_thread: int):
        """Sweep grid of every problem (rq_set_grid): -1 autotune at the next
        evaluation, 0 each problem fills the GPU as if alone, m > 0 fixed."""
        self._check(self._lib.rq_batch_set_grid(self._h, int(min_items_per_thread)))

    def set_fusion(self, max_window_qubits: int):
        """-1: autotune the fusion window at the next evaluation; 0: off; 3..6."""
        self._check(self._lib.rq_batch_set_fusion(self._h, int(max_window_qubits)))

    def hvp(self, gates_list, dirs_list, plain: bool = False):
        """Per-problem lists in, per-problem (f, rgrad, hvps) lists out."""
        k = dirs_list[0].shape[0] if dirs_list else 0
        g = np.ascontiguousarray(np.concatenate([np.asarray(x, np.complex128).ravel() for x in gates_list]))
        d = np.ascontiguousarray(np.concatenate([np.asarray(x, np.complex128).ravel() for x in dirs_list])) \
            if k else np.zeros(1, np.complex128)
        f = np.empty(len(gates_list))
        rg = np.empty_like(g)
        hv = np.empty_like(d)
        self._check(self._lib.rq_batch_hvp(self._h, _dptr(g.view(np.float64)), _dptr(d.view(np.float64)), k,
                                           1 if plain else 0, _dptr(f), _dptr(rg.view(np.float64)),
                                           _dptr(hv.view(np.float64)) if k else None))
        out, go, do = [], 0, 0
        for P in self.n_params:
            r = rg[go:go + P * 16].reshape(P, 4, 4)
            h = hv[do:do + k * P * 16].reshape(k, P, 4, 4) if k else None
            out.append((r, h))
            go += P * 16
            do += k * P * 16
        return f, [o[0] for o in out], [o[1] for o in out]
