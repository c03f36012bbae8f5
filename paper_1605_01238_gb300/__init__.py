"""GB300 weighted-quadrature (WQ) assembly of 3D isogeometric stiffness and mass
matrices (Calabro, Sangalli, Tani, "Fast formation of isogeometric Galerkin
matrices by weighted quadrature").

A thin Python binding over the C ABI of libwq.so (include/wq.h): it marshals
arguments and wraps device memory in torch tensors. Every step of the method
runs in the library's CUDA kernels; there is no CPU path. PyTorch provides
device memory, streams and sparse CSR tensors.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import ALLOC_FN, FREE_FN, Options, WqError, check, load

__all__ = ["Plan", "Batch", "bilinear", "WqError", "launch_count", "load", "TorchAllocator", "HostBuffer", "VALUES_F64",
           "VALUES_F32", "PREC_FP64", "PREC_FP32"]

VALUES_F64, VALUES_F32 = 0, 1
PREC_FP64, PREC_FP32, PREC_MIXED, PREC_F32X2, PREC_TF32X3 = 0, 1, 2, 3, 4
_PREC = {"fp64": PREC_FP64, "fp32": PREC_FP32, "mixed": PREC_MIXED, "f32x2": PREC_F32X2, "tf32x3": PREC_TF32X3}
_ALGO = {"fused": 0, "staged": 1, "auto": 2}


def _torch():
    import torch
    return torch


def _stream(stream=None) -> ctypes.c_void_p:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype, numel: int, name: str) -> int:
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of {numel} elements")
    return t.data_ptr()


class _DeviceView:
    """__cuda_array_interface__ over plan-owned memory; keeps the plan alive."""

    def __init__(self, ptr: int, shape: tuple, typestr: str, owner):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


class HostBuffer:
    """Page-locked host memory of exactly `count` elements of `dtype` (wq_host_alloc),
    viewed as a numpy array (`.array`); released by close() or when collected."""

    def __init__(self, count: int, dtype=np.float64):
        self.dtype = np.dtype(dtype)
        ptr = ctypes.c_void_p()
        check(load().wq_host_alloc(int(count) * self.dtype.itemsize, ctypes.byref(ptr)))
        self._ptr = ptr
        buf = (ctypes.c_char * (int(count) * self.dtype.itemsize)).from_address(ptr.value)
        self.array = np.frombuffer(buf, dtype=self.dtype, count=int(count))

    def close(self) -> None:
        if getattr(self, "_ptr", None) is not None and self._ptr.value:
            self.array = None
            load().wq_host_free(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count() -> int:
    """Kernels launched by libwq in this process."""
    return int(load().wq_launch_count())


class TorchAllocator:
    """Plan-owned device memory from torch's caching allocator (the wq_options
    allocator callbacks), so that a plan draws on the same pool as the rest of a
    torch program. `live` maps each outstanding pointer to its size."""

    def __init__(self):
        torch = _torch()
        self.live = {}

        def _alloc(size, stream, ctx):
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(size), stream=int(stream or 0))
            except Exception:
                return None
            self.live[ptr] = int(size)
            return ptr

        def _free(ptr, stream, ctx):
            try:
                self.live.pop(ptr, None)
                torch.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass

        self.alloc_fn = ALLOC_FN(_alloc)
        self.free_fn = FREE_FN(_free)


class Plan:
    """Mesh- and geometry-dependent data of one 3D patch (wq_plan_create).

    p: degree (2..8); knots: three full open knot vectors; ctrl: (N_DOF, 3)
    control points with direction 1 fastest. Options (wq_options): algorithm
    ("auto", "staged", "fused"), precision and dtype (the defaults of the
    assembly calls), tiles ((t1, t2) of the fused kernel), checked (range-checked
    buffers and finite values, synchronising), tune_cache (a "p t1 t2" text file),
    allocator (a TorchAllocator, or any object with alloc_fn / free_fn ctypes
    callbacks; None = cudaMalloc) and scratch_limit (bytes of staged scratch held
    at once; 0 = the whole mesh).
    """

    def __init__(self, p: int, knots, ctrl, stream=None, *, algorithm=None, precision=None, dtype=None,
                 tiles=None, checked: bool = False, tune_cache=None, allocator=None, scratch_limit: int = 0):
        lib = load()
        self._knots = [np.ascontiguousarray(k, dtype=np.float64) for k in knots]
        if len(self._knots) != 3:
            raise ValueError("three knot vectors are required")
        ctrl = np.ascontiguousarray(ctrl, dtype=np.float64).reshape(-1, 3)
        n_knots = (ctypes.c_int64 * 3)(*[len(k) for k in self._knots])
        kptrs = (ctypes.c_void_p * 3)(*[k.ctypes.data for k in self._knots])
        opt = Options()
        check(lib.wq_options_init(ctypes.byref(opt)))
        if algorithm is not None:
            opt.algorithm = _ALGO[algorithm]
        if precision is not None:
            opt.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        if dtype is not None:
            opt.value_dtype = VALUES_F32 if dtype == _torch().float32 else VALUES_F64
        if tiles is not None:
            opt.tile[0], opt.tile[1] = int(tiles[0]), int(tiles[1])
        opt.checked = 1 if checked else 0
        opt.scratch_limit = int(scratch_limit)
        if tune_cache is not None:
            opt.tune_cache = str(tune_cache).encode()
        self._allocator = allocator
        if allocator is not None:
            opt.alloc, opt.free = allocator.alloc_fn, allocator.free_fn
        self.value_dtype = opt.value_dtype
        self.precision = opt.precision
        h = ctypes.c_void_p()
        check(lib.wq_plan_create(ctypes.byref(h), 3, int(p), n_knots, kptrs,
                                 ctypes.c_void_p(ctrl.ctypes.data), ctypes.byref(opt), _stream(stream)))
        self._h = h
        pp = ctypes.c_int()
        n = (ctypes.c_int64 * 3)()
        nqp = (ctypes.c_int64 * 3)()
        rows, nnz = ctypes.c_int64(), ctypes.c_int64()
        check(lib.wq_plan_info(h, ctypes.byref(pp), n, nqp, ctypes.byref(rows), ctypes.byref(nnz)))
        self.p = pp.value
        self.n = tuple(n)
        self.n_qp = tuple(nqp)
        self.n_rows = rows.value
        self.nnz = nnz.value
        nqm = ctypes.c_int()
        check(lib.wq_get_nq_max(h, ctypes.byref(nqm)))
        self.nq_max = nqm.value

    # -- lifetime
    def close(self) -> None:
        if getattr(self, "_h", None):
            load().wq_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    # -- pattern
    def pattern(self):
        """(row_ptr int64[N+1], col int32[nnz]) as zero-copy CUDA tensors."""
        torch = _torch()
        rp, cl = ctypes.c_void_p(), ctypes.c_void_p()
        check(load().wq_plan_pattern(self._h, ctypes.byref(rp), ctypes.byref(cl)))
        row_ptr = torch.as_tensor(_DeviceView(rp.value, (self.n_rows + 1,), "<i8", self), device="cuda")
        col = torch.as_tensor(_DeviceView(cl.value, (self.nnz,), "<i4", self), device="cuda")
        return row_ptr, col

    def csr(self, values):
        """torch.sparse_csr_tensor over the plan's pattern and the given values."""
        torch = _torch()
        row_ptr, col = self.pattern()
        return torch.sparse_csr_tensor(row_ptr, col, values, size=(self.n_rows, self.n_rows))

    # -- geometry
    def set_geometry(self, ctrl, stream=None) -> None:
        """New control points (CUDA tensor or host array); recomputes coefficients."""
        torch = _torch()
        if isinstance(ctrl, torch.Tensor) and ctrl.is_cuda:
            ptr, on_dev = _dev_ptr(ctrl, torch.float64, 3 * self.n_rows, "ctrl"), 1
        else:
            arr = np.ascontiguousarray(ctrl, dtype=np.float64).reshape(-1)
            self._host_ctrl = arr
            ptr, on_dev = arr.ctypes.data, 0
        check(load().wq_plan_set_geometry(self._h, ctypes.c_void_p(ptr), on_dev, _stream(stream)))

    def set_weights(self, weights=None, nurbs_basis: bool = False, stream=None) -> None:
        """NURBS weights of the control points (wq_plan_set_weights): a rational map
        F = sum w C B / sum w B; nurbs_basis=True also makes the basis functions NURBS
        (mass matrix only). weights: (N_DOF,) host array or CUDA float64 tensor, or None."""
        torch = _torch()
        ptr, on_dev = None, 0
        if weights is not None:
            if isinstance(weights, torch.Tensor) and weights.is_cuda:
                ptr, on_dev = _dev_ptr(weights, torch.float64, self.n_rows, "weights"), 1
            else:
                arr = np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
                if arr.size != self.n_rows:
                    raise ValueError("weights must hold N_DOF values")
                self._host_w = arr
                ptr = arr.ctypes.data
        check(load().wq_plan_set_weights(self._h, ctypes.c_void_p(ptr), on_dev, 1 if nurbs_basis else 0,
                                         _stream(stream)))

    def set_tensor(self, K=None, stream=None) -> None:
        """Coefficient tensor field (wq_plan_set_tensor): CUDA float64 (6, N_QP) tensor
        of K11 K12 K13 K22 K23 K33 at the points (q1 fastest), or None for K = I."""
        torch = _torch()
        ptr = None
        if K is not None:
            ptr = _dev_ptr(K, torch.float64, 6 * int(np.prod(self.n_qp)), "K")
        check(load().wq_plan_set_tensor(self._h, ctypes.c_void_p(ptr), _stream(stream)))

    def refresh(self, ctrl=None, stream=None) -> None:
        """Re-run every set-up kernel in place (optionally with new control points)."""
        torch = _torch()
        ptr, on_dev = None, 1
        if ctrl is not None:
            if isinstance(ctrl, torch.Tensor) and ctrl.is_cuda:
                ptr = _dev_ptr(ctrl, torch.float64, 3 * self.n_rows, "ctrl")
            else:
                arr = np.ascontiguousarray(ctrl, dtype=np.float64).reshape(-1)
                self._host_ctrl = arr
                ptr, on_dev = arr.ctypes.data, 0
        check(load().wq_plan_refresh(self._h, ctypes.c_void_p(ptr), on_dev, _stream(stream)))

    def set_algorithm(self, algorithm: str) -> None:
        """"fused" (one kernel, tiles in shared memory), "staged" (three kernels,
        intermediates in device memory) or "auto" (the default: staged)."""
        check(load().wq_plan_set_algorithm(self._h, _ALGO[algorithm]))

    def reserve(self, precision=None, dtype=None, adjoint: bool = False, stream=None) -> None:
        """Allocate now the scratch that the first assembly in (precision, dtype), and
        with adjoint=True the first adjoint, would allocate (wq_plan_reserve)."""
        torch = _torch()
        vdt = -1 if dtype is None else (VALUES_F32 if dtype == torch.float32 else VALUES_F64)
        prec = -1 if precision is None else (_PREC[precision] if isinstance(precision, str) else int(precision))
        check(load().wq_plan_reserve(self._h, prec, vdt, 1 if adjoint else 0, _stream(stream)))

    def set_tiles(self, t1: int = 0, t2: int = 0) -> None:
        """Assembly tile extents in directions 1 and 2 (0, 0 = defaults)."""
        check(load().wq_plan_set_tiles(self._h, int(t1), int(t2)))

    def tiles(self) -> tuple:
        """The plan's tile extents (0, 0 = defaults)."""
        a, b = ctypes.c_int(), ctypes.c_int()
        check(load().wq_plan_get_tiles(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    # -- assembly
    def _assemble(self, fn, kappa, out, dtype, precision, stream):
        torch = _torch()
        if dtype is None:
            dtype = torch.float32 if self.value_dtype == VALUES_F32 else torch.float64
        vdt = VALUES_F64 if dtype == torch.float64 else VALUES_F32 if dtype == torch.float32 else None
        if vdt is None:
            raise ValueError("dtype must be torch.float64 or torch.float32")
        if precision is None:
            prec = self.precision
        else:
            prec = _PREC[precision] if isinstance(precision, str) else int(precision)
        if out is None:
            out = torch.empty(self.nnz, dtype=dtype, device="cuda")
        vp = _dev_ptr(out, dtype, self.nnz, "out")
        kp = None
        if kappa is not None:
            kp = _dev_ptr(kappa, torch.float64, int(np.prod(self.n_qp)), "kappa")
        check(fn(self._h, ctypes.c_void_p(kp), ctypes.c_void_p(vp), vdt, prec, _stream(stream)))
        return out

    def stiffness(self, kappa=None, out=None, dtype=None, precision=None, stream=None):
        """CSR values of the WQ stiffness matrix (Eq. (stiff)) in the plan's order."""
        return self._assemble(load().wq_assemble_stiffness, kappa, out, dtype, precision, stream)

    def mass(self, kappa=None, out=None, dtype=None, precision=None, stream=None):
        """CSR values of the WQ mass matrix (Eq. (Mass_approx))."""
        return self._assemble(load().wq_assemble_mass, kappa, out, dtype, precision, stream)

    def load(self, f, out=None, stream=None):
        """WQ load vector b_i = Q_i(f det DF) (wq_assemble_load); f: CUDA float64 source
        at the points (q1 fastest), N_QP values."""
        torch = _torch()
        fp = _dev_ptr(f, torch.float64, int(np.prod(self.n_qp)), "f")
        if out is None:
            out = torch.empty(self.n_rows, dtype=torch.float64, device="cuda")
        bp = _dev_ptr(out, torch.float64, self.n_rows, "out")
        check(load().wq_assemble_load(self._h, ctypes.c_void_p(fp), ctypes.c_void_p(bp), _stream(stream)))
        return out

    def assemble_host(self, which: str, h_ctrl, d_vals, h_vals, stream=None) -> None:
        """End-to-end call with host buffers (wq_assemble_host): h_ctrl host float64
        control points or None, d_vals a CUDA float64 staging tensor of nnz
        elements (None when h_vals is a HostBuffer, which the last mode product
        writes directly), h_vals a host float64 tensor/array of nnz elements."""
        torch = _torch()
        vp = None if d_vals is None else _dev_ptr(d_vals, torch.float64, self.nnz, "d_vals")
        if isinstance(h_vals, torch.Tensor):
            if h_vals.is_cuda or h_vals.dtype != torch.float64 or h_vals.numel() != self.nnz:
                raise ValueError("h_vals must be a host float64 tensor of nnz elements")
            hp = h_vals.data_ptr()
        else:
            hp = h_vals.ctypes.data
        cp = None
        if h_ctrl is not None:
            if isinstance(h_ctrl, torch.Tensor):
                cp = h_ctrl.data_ptr()
            else:
                cp = h_ctrl.ctypes.data
        check(load().wq_assemble_host(self._h, 1 if which == "mass" else 0, ctypes.c_void_p(cp),
                                      ctypes.c_void_p(vp), ctypes.c_void_p(hp), _stream(stream)))

    def adjoint(self, lam, u, kappa=None, which: str = "stiffness", grad_kappa: bool = True,
                grad_ctrl: bool = True, stream=None):
        """(J, dJ/dkappa or None, dJ/dC or None) for J = lam^T A u, A = S, M or S+M
        (which = "stiffness", "mass", "both"); wq_adjoint."""
        torch = _torch()
        w = {"stiffness": 1, "mass": 2, "both": 3}[which]
        lp = _dev_ptr(lam, torch.float64, self.n_rows, "lam")
        up = _dev_ptr(u, torch.float64, self.n_rows, "u")
        nqp = int(np.prod(self.n_qp))
        kp = None if kappa is None else _dev_ptr(kappa, torch.float64, nqp, "kappa")
        gk = torch.empty(nqp, dtype=torch.float64, device="cuda") if grad_kappa else None
        gc = torch.empty(self.n_rows * 3, dtype=torch.float64, device="cuda") if grad_ctrl else None
        J = ctypes.c_double()
        check(load().wq_adjoint(self._h, w, ctypes.c_void_p(kp), ctypes.c_void_p(lp), ctypes.c_void_p(up),
                                ctypes.byref(J), ctypes.c_void_p(None if gk is None else gk.data_ptr()),
                                ctypes.c_void_p(None if gc is None else gc.data_ptr()), _stream(stream)))
        return J.value, gk, (None if gc is None else gc.view(self.n_rows, 3))

    def sync_check(self, stream=None) -> None:
        check(load().wq_sync_check(self._h, _stream(stream)))

    # -- inspection (synchronous copies)
    def points(self, direction: int) -> np.ndarray:
        out = np.empty(self.n_qp[direction])
        check(load().wq_get_points(self._h, direction, ctypes.c_void_p(out.ctypes.data)))
        return out

    def rules(self, direction: int, a: int, b: int):
        """(w[n, nq_max], q0[n], nq[n]): rule of kind (a, b) for every test function."""
        n = self.n[direction]
        w = np.empty((n, self.nq_max))
        q0 = np.empty(n, dtype=np.int32)
        nq = np.empty(n, dtype=np.int32)
        check(load().wq_get_rules(self._h, direction, a, b, ctypes.c_void_p(w.ctypes.data),
                                  ctypes.c_void_p(q0.ctypes.data), ctypes.c_void_p(nq.ctypes.data)))
        return w, q0, nq

    def coefficients(self) -> np.ndarray:
        """(7, nqp3, nqp2, nqp1): c_11 c_12 c_13 c_22 c_23 c_33 and det DF."""
        out = np.empty((7, self.n_qp[2], self.n_qp[1], self.n_qp[0]))
        check(load().wq_get_coefficients(self._h, ctypes.c_void_p(out.ctypes.data)))
        return out


class Batch:
    """Many plans assembled by one persistent, graph-captured launch (wq_batch_create).

    stiffness / mass: None, or one CUDA float64 tensor (nnz of that plan) or None
    per plan. The plans and tensors must stay alive as long as the batch."""

    def __init__(self, plans, stiffness=None, mass=None, stream=None):
        torch = _torch()
        self.plans = list(plans)
        count = len(self.plans)
        self._keep = []

        def ptrs(outs):
            if outs is None:
                return None
            arr = (ctypes.c_void_p * count)()
            for k, (pl, t) in enumerate(zip(self.plans, outs)):
                arr[k] = None if t is None else _dev_ptr(t, torch.float64, pl.nnz, "batch output")
            self._keep.append(outs)
            return arr

        handles = (ctypes.c_void_p * count)(*[pl.handle.value for pl in self.plans])
        s_arr, m_arr = ptrs(stiffness), ptrs(mass)
        h = ctypes.c_void_p()
        check(load().wq_batch_create(ctypes.byref(h), count, ctypes.cast(handles, ctypes.c_void_p),
                                     ctypes.cast(s_arr, ctypes.c_void_p) if s_arr is not None else None,
                                     ctypes.cast(m_arr, ctypes.c_void_p) if m_arr is not None else None,
                                     _stream(stream)))
        self._h = h
        n_items, nnz, grid = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        check(load().wq_batch_info(h, ctypes.byref(n_items), ctypes.byref(nnz), ctypes.byref(grid)))
        self.n_items, self.nnz_total, self.grid = n_items.value, nnz.value, grid.value

    def launch(self, stream=None) -> None:
        check(load().wq_batch_assemble(self._h, _stream(stream)))

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().wq_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bilinear_function():
    torch = _torch()

    class _Bilinear(torch.autograd.Function):
        """J = lam^T A(ctrl, kappa) u with the hand-written adjoint as backward."""

        @staticmethod
        def forward(ctx, ctrl, kappa, plan, lam, u, which):
            plan.set_geometry(ctrl.detach().reshape(-1).contiguous())
            want_k = kappa is not None and ctx.needs_input_grad[1]
            J, gk, gc = plan.adjoint(lam, u, None if kappa is None else kappa.detach().contiguous(), which,
                                     grad_kappa=want_k, grad_ctrl=ctx.needs_input_grad[0])
            ctx.save_for_backward(gc if gc is not None else torch.empty(0), gk if gk is not None else torch.empty(0))
            ctx.has = (gc is not None, gk is not None)
            return torch.tensor(J, dtype=torch.float64, device=ctrl.device)

        @staticmethod
        def backward(ctx, grad_out):
            gc, gk = ctx.saved_tensors
            g_ctrl = grad_out * gc if ctx.has[0] else None
            g_kappa = grad_out * gk if ctx.has[1] else None
            return g_ctrl, g_kappa, None, None, None, None

    return _Bilinear


_BILINEAR = None


def bilinear(plan, ctrl, lam, u, kappa=None, which: str = "stiffness"):
    """Differentiable J = lam^T A u for the plan's mesh with control points `ctrl`
    ((N_DOF, 3) CUDA float64) and coefficient field `kappa` (CUDA float64 over the
    points, or None); gradients flow to ctrl and kappa through wq_adjoint."""
    global _BILINEAR
    if _BILINEAR is None:
        _BILINEAR = _bilinear_function()
    return _BILINEAR.apply(ctrl, kappa, plan, lam, u, which)
