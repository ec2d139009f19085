"""Python binding of libnufft: plan objects over torch CUDA tensors, and autograd.

PyTorch provides device memory and streams only; every step of the transform runs
in the library's CUDA kernels.  All calls are enqueued on the current torch stream
of the tensors' device.
"""

from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import (NUFFT_BATCH_GRAPH, NUFFT_BATCH_PER_PROBLEM, NUFFT_BATCH_PERSISTENT, NUFFT_F32, NUFFT_F64,
                   NUFFT_PLAN_AUTOTUNE,
                   NUFFT_PLAN_HALF_TILE, NUFFT_RESERVE_STEP_HOST, NUFFT_PLAN_LONG_COLUMNS,
                   NUFFT_PLAN_TIMING, NUFFT_PLAN_UNFUSED, NufftError, check)

_CDTYPE = {NUFFT_F32: torch.complex64, NUFFT_F64: torch.complex128}
_RDTYPE = {NUFFT_F32: torch.float32, NUFFT_F64: torch.float64}


def _prec(precision):
    if precision in ("f32", "float32", torch.float32, torch.complex64, NUFFT_F32):
        return NUFFT_F32
    if precision in ("f64", "float64", torch.float64, torch.complex128, NUFFT_F64):
        return NUFFT_F64
    raise ValueError("precision must be 'f32' or 'f64'")


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A planned NUFFT-II on a fixed set of samples x (the planning stage, section 2.3).

    Parameters
    ----------
    N : number of frequencies k = 0..N-1
    x : samples, a 1-D tensor or array (moved to the current CUDA device as float64)
    eps : working accuracy
    precision : 'f32' (complex64 exec) or 'f64' (complex128 exec)
    L : grid size (0 = smallest power of two >= max(N, 1024); L > N oversamples)
    unfused : also build the materialised factors for :meth:`forward_unfused`
    timing : record per-kernel device times (:meth:`kernel_times`)
    autotune : with L = 0, time the grid L0 against 2 L0 and both four-step splits, keep the fastest
    long_columns : for odd log2 L, put the longer FFT of the four-step split on the columns
    half_tile : the column pass takes half as many columns per CTA
    """

    def __init__(self, N, x, eps, precision="f32", L=0, unfused=False, timing=False, device=None,
                 autotune=False, long_columns=False, half_tile=False):
        lib = _lib.load()
        device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if not isinstance(x, torch.Tensor):
            x = torch.as_tensor(x)
        x = x.detach().to(device=device, dtype=torch.float64).contiguous()
        self.device = device
        self.N, self.M = int(N), int(x.numel())
        self.prec = _prec(precision)
        self.cdtype, self.rdtype = _CDTYPE[self.prec], _RDTYPE[self.prec]
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            rc = lib.nufft2_plan(ctypes.byref(h), self.N, self.M, _ptr(x) if self.M else None,
                                 float(eps), self.prec, int(L),
                                 (NUFFT_PLAN_UNFUSED if unfused else 0) | (NUFFT_PLAN_TIMING if timing else 0)
                                 | (NUFFT_PLAN_AUTOTUNE if autotune else 0)
                                 | (NUFFT_PLAN_LONG_COLUMNS if long_columns else 0)
                                 | (NUFFT_PLAN_HALF_TILE if half_tile else 0),
                                 _stream(device))
        check(rc, "nufft2_plan")
        self._h = h
        self.eps = float(eps)
        # the samples the plan was built on: nufft2(..., plan=...) checks that it is given these
        self._x = x
        self._x_seen = set()
        K, g, Lo, wb = ctypes.c_int(), ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        check(lib.nufft2_plan_info(h, ctypes.byref(K), ctypes.byref(g), ctypes.byref(Lo), ctypes.byref(wb)),
              "nufft2_plan_info")
        self.K, self.gamma, self.L, self.work_bytes = K.value, g.value, Lo.value, wb.value

    # -- lifetime -----------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            torch.cuda.synchronize(self.device)
            _lib.load().nufft_destroy(self._h)
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

    # -- helpers ----------------------------------------------------------------------
    def _cx(self, t, n, name):
        if t.device != self.device or t.dtype != self.cdtype or not t.is_contiguous() or t.numel() != n:
            raise ValueError("%s must be a contiguous %s tensor of %d elements on %s"
                             % (name, self.cdtype, n, self.device))
        return t

    def export(self):
        """(t, d, alpha): grid indices, scaled perturbations (FP64) and a_pr = i^r alpha_pr."""
        t = torch.empty(self.M, dtype=torch.int32, device=self.device)
        d = torch.empty(self.M, dtype=torch.float64, device=self.device)
        alpha = (ctypes.c_double * (self.K * self.K))()
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_plan_export(self._h, _ptr(t) if self.M else None,
                                                 _ptr(d) if self.M else None, alpha, _stream(self.device)),
                  "nufft2_plan_export")
        import numpy as np
        return t, d, np.array(alpha[:], dtype=np.float64).reshape(self.K, self.K)

    def check(self):
        """Synchronise and raise NufftError(NUFFT_ETIMEOUT) if a device-side wait gave up."""
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_check(self._h, _stream(self.device)), "nufft2_check")

    def kernel_times(self):
        """Device milliseconds of each kernel of the last exec call (plan built with timing=True)."""
        buf = (ctypes.c_float * 8)()
        n = ctypes.c_int()
        check(_lib.load().nufft_kernel_times(self._h, buf, 8, ctypes.byref(n)), "nufft_kernel_times")
        return list(buf[: n.value])

    # -- online stage -------------------------------------------------------------------
    def forward(self, c, out=None):
        """f = A c (the NUFFT-II, eq. (2.11))."""
        self._cx(c, self.N, "c")
        f = out if out is not None else torch.empty(self.M, dtype=self.cdtype, device=self.device)
        self._cx(f, self.M, "f")
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_exec(self._h, _ptr(c), _ptr(f), _stream(self.device)), "nufft2_exec")
        return f

    def inverse(self, f, tol=1e-12, maxit=1000, out=None):
        """Solve A c = f by CG on the normal equations (section 3.3).

        Returns (c, iterations, relative residual of the normal equations)."""
        self._cx(f, self.M, "f")
        c = out if out is not None else torch.empty(self.N, dtype=self.cdtype, device=self.device)
        self._cx(c, self.N, "c")
        it, rr = ctypes.c_int(), ctypes.c_double()
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_inverse(self._h, _ptr(f), _ptr(c), float(tol), int(maxit), ctypes.byref(it),
                                             ctypes.byref(rr), _stream(self.device)), "nufft2_inverse")
        return c, it.value, rr.value

    def adjoint(self, g, out=None):
        """c = A^H g (the conjugate transpose of forward)."""
        self._cx(g, self.M, "g")
        c = out if out is not None else torch.empty(self.N, dtype=self.cdtype, device=self.device)
        self._cx(c, self.N, "c")
        with torch.cuda.device(self.device):
            check(_lib.load().nufft1_exec(self._h, _ptr(g), _ptr(c), _stream(self.device)), "nufft1_exec")
        return c

    def transpose(self, g):
        """The paper's NUFFT-I (section 3.1): A^T g = conj(A^H conj(g))."""
        return torch.conj(self.adjoint(torch.conj(g).resolve_conj().contiguous())).resolve_conj()

    def dx(self, c, g, out=None, accumulate=False):
        """gx_j (+)= Re(conj(g_j) d f_j / d x_j)."""
        self._cx(c, self.N, "c")
        self._cx(g, self.M, "g")
        gx = out if out is not None else torch.empty(self.M, dtype=self.rdtype, device=self.device)
        if gx.dtype != self.rdtype or gx.numel() != self.M or not gx.is_contiguous():
            raise ValueError("gx must be a contiguous %s tensor of %d elements" % (self.rdtype, self.M))
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_exec_dx(self._h, _ptr(c), _ptr(g), _ptr(gx), int(bool(accumulate)),
                                             _stream(self.device)), "nufft2_exec_dx")
        return gx

    def forward_deriv(self, c, out=None, out_deriv=None):
        """(f, f') with f = A c and f'_j = d f_j / d x_j, from K + 1 FFTs in one exec."""
        self._cx(c, self.N, "c")
        f = out if out is not None else torch.empty(self.M, dtype=self.cdtype, device=self.device)
        fp = out_deriv if out_deriv is not None else torch.empty(self.M, dtype=self.cdtype, device=self.device)
        self._cx(f, self.M, "f")
        self._cx(fp, self.M, "fprime")
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_exec_deriv(self._h, _ptr(c), _ptr(f), _ptr(fp), _stream(self.device)),
                  "nufft2_exec_deriv")
        return f, fp

    def grad_x(self, g, fprime, out=None, accumulate=False):
        """gx_j (+)= Re(conj(g_j) fprime_j)."""
        self._cx(g, self.M, "g")
        self._cx(fprime, self.M, "fprime")
        gx = out if out is not None else torch.empty(self.M, dtype=self.rdtype, device=self.device)
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_grad_x(self._h, _ptr(g), _ptr(fprime), _ptr(gx), int(bool(accumulate)),
                                            _stream(self.device)), "nufft2_grad_x")
        return gx

    def reserve(self, B=0, step_host=False):
        """The plan stage of the batch calls and of :meth:`step_host`
        (nufft2_plan_reserve): a workspace and kernel arguments for batches of up to B
        members, and with ``step_host`` the device buffers of the host-buffer step.  The
        exec calls themselves then allocate nothing and do not synchronise, so they can be
        captured in a CUDA graph.  Synchronises; call it outside any stream capture."""
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_plan_reserve(self._h, int(B), NUFFT_RESERVE_STEP_HOST if step_host else 0,
                                                  _stream(self.device)), "nufft2_plan_reserve")
        cap, sh = ctypes.c_int64(), ctypes.c_int()
        check(_lib.load().nufft2_plan_reserved(self._h, ctypes.byref(cap), ctypes.byref(sh)), "nufft2_plan_reserved")
        self._bcap, self._step_host = cap.value, bool(sh.value)

    def _need_batch(self, B):
        """Reserve for B members first, unless a stream is being captured: there the
        exec call must find its workspace already made (else it raises NUFFT_ESTATE)."""
        if B > getattr(self, "_bcap", 1) and not torch.cuda.is_current_stream_capturing():
            self.reserve(max(B, 2), getattr(self, "_step_host", False))

    def forward_batch(self, c, out=None):
        """f[b] = A c[b] for a (B, N) batch."""
        if c.dim() != 2 or c.shape[1] != self.N or c.dtype != self.cdtype or c.stride(1) != 1:
            raise ValueError("c must be (B, N) %s with unit inner stride" % self.cdtype)
        B = c.shape[0]
        self._need_batch(B)
        f = out if out is not None else torch.empty(B, self.M, dtype=self.cdtype, device=self.device)
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_exec_batch(self._h, B, _ptr(c), c.stride(0), _ptr(f), f.stride(0),
                                                _stream(self.device)), "nufft2_exec_batch")
        return f

    def _batch2(self, t, n, name):
        if t.dim() != 2 or t.shape[1] != n or t.dtype != self.cdtype or t.stride(1) != 1 or t.device != self.device:
            raise ValueError("%s must be (B, %d) %s with unit inner stride on %s" % (name, n, self.cdtype, self.device))
        return t

    def adjoint_batch(self, g, out=None):
        """c[b] = A^H g[b] for a (B, M) batch."""
        self._batch2(g, self.M, "g")
        B = g.shape[0]
        self._need_batch(B)
        c = out if out is not None else torch.empty(B, self.N, dtype=self.cdtype, device=self.device)
        self._batch2(c, self.N, "c")
        with torch.cuda.device(self.device):
            check(_lib.load().nufft1_exec_batch(self._h, B, _ptr(g), g.stride(0), _ptr(c), c.stride(0),
                                                _stream(self.device)), "nufft1_exec_batch")
        return c

    def forward_deriv_batch(self, c, out=None, out_deriv=None):
        """(f[b], f'[b]) for a (B, N) batch: the forward and df/dx of every member."""
        self._batch2(c, self.N, "c")
        B = c.shape[0]
        self._need_batch(B)
        f = out if out is not None else torch.empty(B, self.M, dtype=self.cdtype, device=self.device)
        fp = out_deriv if out_deriv is not None else torch.empty(B, self.M, dtype=self.cdtype, device=self.device)
        self._batch2(f, self.M, "f")
        self._batch2(fp, self.M, "fprime")
        if f.stride(0) != fp.stride(0):
            raise ValueError("f and fprime must have the same row stride")
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_exec_deriv_batch(self._h, B, _ptr(c), c.stride(0), _ptr(f), _ptr(fp),
                                                      f.stride(0), _stream(self.device)), "nufft2_exec_deriv_batch")
        return f, fp

    def grad_x_batch(self, g, fprime, out=None, accumulate=False):
        """gx (+)= sum_b Re(conj(g[b]) fprime[b]) for (B, M) batches."""
        self._batch2(g, self.M, "g")
        self._batch2(fprime, self.M, "fprime")
        if g.stride(0) != fprime.stride(0) or g.shape[0] != fprime.shape[0]:
            raise ValueError("g and fprime must have the same shape and row stride")
        gx = out if out is not None else torch.empty(self.M, dtype=self.rdtype, device=self.device)
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_grad_x_batch(self._h, g.shape[0], _ptr(g), _ptr(fprime), g.stride(0), _ptr(gx),
                                                  1 if accumulate else 0, _stream(self.device)), "nufft2_grad_x_batch")
        return gx

    def step_host(self, c_host, g_host, f_host, gc_host, gx_host):
        """One training step with host (ideally pinned) tensors: f = A c, A^H g into gc_host
        and dL/dx = Re(conj(g) f') into gx_host, copies overlapped with the transforms.
        Asynchronous: the host tensors hold the results once the current stream has
        completed."""
        for t, n, dt in ((c_host, self.N, self.cdtype), (g_host, self.M, self.cdtype), (f_host, self.M, self.cdtype),
                         (gc_host, self.N, self.cdtype), (gx_host, self.M, self.rdtype)):
            if t.device.type != "cpu" or t.dtype != dt or not t.is_contiguous() or t.numel() != n:
                raise ValueError("host tensors must be contiguous CPU tensors of the plan's sizes and types")
        if not getattr(self, "_step_host", False) and not torch.cuda.is_current_stream_capturing():
            self.reserve(getattr(self, "_bcap", 0), step_host=True)
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_step_host(self._h, _ptr(c_host), _ptr(g_host), _ptr(f_host), _ptr(gc_host),
                                               _ptr(gx_host), _stream(self.device)), "nufft2_step_host")

    def forward_host(self, c_host, f_host):
        """f_host = A c_host with host (ideally pinned) tensors; synchronises."""
        if c_host.device.type != "cpu" or f_host.device.type != "cpu":
            raise ValueError("forward_host takes CPU tensors")
        if c_host.dtype != self.cdtype or f_host.dtype != self.cdtype:
            raise ValueError("dtype must be %s" % self.cdtype)
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_exec_host(self._h, _ptr(c_host), _ptr(f_host), _stream(self.device)),
                  "nufft2_exec_host")
        return f_host

    def forward_unfused(self, c, out=None):
        """The unfused comparator (plan must be built with unfused=True)."""
        self._cx(c, self.N, "c")
        f = out if out is not None else torch.empty(self.M, dtype=self.cdtype, device=self.device)
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_exec_unfused(self._h, _ptr(c), _ptr(f), _stream(self.device)),
                  "nufft2_exec_unfused")
        return f


def rank(eps, gamma):
    """The planner's rank for accuracy eps and perturbation gamma = max |delta_j| (host)."""
    K = ctypes.c_int()
    check(_lib.load().nufft_rank(float(eps), float(gamma), ctypes.byref(K)), "nufft_rank")
    return K.value


def tune_save(path):
    """Write the autotuner's choices of this process to ``path``; returns the entry count."""
    n = ctypes.c_int64()
    check(_lib.load().nufft_tune_save(str(path).encode(), ctypes.byref(n)), "nufft_tune_save")
    return n.value


def tune_load(path):
    """Merge a table written by :func:`tune_save`; later autotuned plans reuse it.
    Returns the number of entries read."""
    n = ctypes.c_int64()
    check(_lib.load().nufft_tune_load(str(path).encode(), ctypes.byref(n)), "nufft_tune_load")
    return n.value


def tune_clear():
    """Empty the autotuner's table; returns the number of entries it held."""
    n = ctypes.c_int64()
    check(_lib.load().nufft_tune_clear(ctypes.byref(n)), "nufft_tune_clear")
    return n.value


class _Nufft2(torch.autograd.Function):
    """f = A(x) c with a hand-written backward: dL/dc = A^H g, dL/dx = Re(conj(g) f').

    When x needs a gradient the forward also forms f' = df/dx (nufft2_exec_deriv: the
    same pass with one more rank) and keeps it for the backward."""

    @staticmethod
    def forward(ctx, c, x, plan):
        ctx.plan = plan
        cc = c.detach().contiguous()
        batched = cc.dim() == 2
        want_dx = ctx.needs_input_grad[1]
        fp = None
        if not want_dx:
            f = plan.forward_batch(cc) if batched else plan.forward(cc)
        elif batched:
            f, fp = plan.forward_deriv_batch(cc)
        else:
            f, fp = plan.forward_deriv(cc)
        ctx.save_for_backward(fp if fp is not None else torch.empty(0, device=plan.device))
        ctx.batched = batched
        return f

    @staticmethod
    def backward(ctx, g):
        (fp,) = ctx.saved_tensors
        plan = ctx.plan
        g = g.contiguous()
        gc = gx = None
        if ctx.needs_input_grad[0]:
            if ctx.batched:
                gc = plan.adjoint_batch(g)
            else:
                gc = plan.adjoint(g)
        if ctx.needs_input_grad[1]:
            gx = torch.empty(plan.M, dtype=plan.rdtype, device=plan.device)
            if ctx.batched:
                plan.grad_x_batch(g, fp, gx)
            else:
                plan.grad_x(g, fp, gx)
            gx = gx.to(torch.float64)
        return gc, gx, None


def _check_plan_samples(plan, x):
    """Raise ValueError unless x holds the samples `plan` was built on.  A stale plan would
    give wrong values and gradients silently.  A tensor already found equal is remembered
    by (storage address, version counter), so a training loop that passes the same x pays
    for one comparison (a device sync) and not one per step."""
    if x.numel() != plan.M:
        raise ValueError("x has %d samples, the plan was built on %d" % (x.numel(), plan.M))
    key = (x.data_ptr(), x._version, str(x.device))
    if key in plan._x_seen:
        return
    xs = x.detach().to(device=plan.device, dtype=torch.float64).reshape(-1)
    if not torch.equal(xs, plan._x):
        raise ValueError("the plan was built on other samples than x: build a new plan for these x")
    plan._x_seen.add(key)


def nufft2(c, x, eps=1e-9, plan=None, L=0):
    """Differentiable NUFFT-II: f_j = sum_k c_k exp(-2 pi i x_j k) for c of shape (N,)
    or (B, N) (complex64 -> FP32 exec, complex128 -> FP64 exec) and samples x (float64).
    Gradients flow to c and x.  Pass a prebuilt ``plan`` to reuse it; it must have been
    built on the same x (checked: ValueError otherwise)."""
    if plan is None:
        plan = Plan(c.shape[-1], x.detach(), eps, precision=c.dtype, L=L, device=c.device)
    else:
        _check_plan_samples(plan, x)
    return _Nufft2.apply(c, x, plan)


__all__ = ["Plan", "nufft2", "NufftError", "NUFFT_F32", "NUFFT_F64"]


class Plan2D:
    """A planned 2D NUFFT-II (section 4, eq. (4.4)) on samples (x_j, y_j).

    f_j = sum_{k1<m, k2<n} C[k1, k2] exp(-2 pi i (k1 x_j + k2 y_j)), C an m x n complex64
    (precision "f32") or complex128 ("f64") tensor (row-major).  Each direction runs the 1D
    method at eps / 2.
    """

    def __init__(self, m, n, x, y, eps, precision="f32", timing=False, device=None):
        lib = _lib.load()
        device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        x = torch.as_tensor(x).detach().to(device=device, dtype=torch.float64).contiguous().reshape(-1)
        y = torch.as_tensor(y).detach().to(device=device, dtype=torch.float64).contiguous().reshape(-1)
        if x.numel() != y.numel():
            raise ValueError("x and y must have the same length")
        self.device = device
        self.m, self.n, self.M = int(m), int(n), int(x.numel())
        self.prec = _prec(precision)
        self.cdtype = _CDTYPE[self.prec]
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            rc = lib.nufft2d_plan(ctypes.byref(h), self.m, self.n, self.M, _ptr(x) if self.M else None,
                                  _ptr(y) if self.M else None, float(eps), self.prec,
                                  NUFFT_PLAN_TIMING if timing else 0, _stream(device))
        check(rc, "nufft2d_plan")
        self._h = h
        Kx, Ky, gx, gy = ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        Lx, Ly = ctypes.c_int64(), ctypes.c_int64()
        check(lib.nufft2d_plan_info(h, ctypes.byref(Kx), ctypes.byref(Ky), ctypes.byref(gx), ctypes.byref(gy),
                                    ctypes.byref(Lx), ctypes.byref(Ly)), "nufft2d_plan_info")
        self.Kx, self.Ky, self.gamma_x, self.gamma_y = Kx.value, Ky.value, gx.value, gy.value
        self.Lx, self.Ly = Lx.value, Ly.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            torch.cuda.synchronize(self.device)
            _lib.load().nufft_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, C, out=None):
        """f = the 2D NUFFT-II of the m x n matrix C."""
        if C.device != self.device or C.dtype != self.cdtype or not C.is_contiguous() or C.numel() != self.m * self.n:
            raise ValueError("C must be a contiguous %s tensor of %d x %d elements on %s"
                             % (self.cdtype, self.m, self.n, self.device))
        f = out if out is not None else torch.empty(self.M, dtype=self.cdtype, device=self.device)
        if f.device != self.device or f.dtype != self.cdtype or not f.is_contiguous() or f.numel() != self.M:
            raise ValueError("f must be a contiguous %s tensor of %d elements" % (self.cdtype, self.M))
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_exec(self._h, _ptr(C), _ptr(f), _stream(self.device)), "nufft2_exec")
        return f

    def adjoint(self, g, out=None):
        """C = A^H g: C[k1, k2] = sum_j g_j exp(+2 pi i (k1 x_j + k2 y_j)), an m x n tensor."""
        if g.device != self.device or g.dtype != self.cdtype or not g.is_contiguous() or g.numel() != self.M:
            raise ValueError("g must be a contiguous %s tensor of %d elements on %s"
                             % (self.cdtype, self.M, self.device))
        C = out if out is not None else torch.empty((self.m, self.n), dtype=self.cdtype, device=self.device)
        if C.device != self.device or C.dtype != self.cdtype or not C.is_contiguous() or C.numel() != self.m * self.n:
            raise ValueError("C must be a contiguous %s tensor of %d x %d elements" % (self.cdtype, self.m, self.n))
        with torch.cuda.device(self.device):
            check(_lib.load().nufft1_exec(self._h, _ptr(g), _ptr(C), _stream(self.device)), "nufft1_exec")
        return C

    def check(self):
        """Synchronise and raise NufftError if a device-side wait gave up or a check failed."""
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_check(self._h, _stream(self.device)), "nufft2_check")

    def kernel_times(self):
        """Device milliseconds of the column and row pass of the last forward, or of the row
        and column pass of the last adjoint (timing=True)."""
        buf = (ctypes.c_float * 8)()
        k = ctypes.c_int()
        check(_lib.load().nufft_kernel_times(self._h, buf, 8, ctypes.byref(k)), "nufft_kernel_times")
        return list(buf[: k.value])


class Batch:
    """Many independent NUFFT-II problems of uneven sizes, run together.

    Problem i has N[i] frequencies, the samples ``xs[i]`` and accuracy ``eps[i]``; each
    is planned as by :class:`Plan`.  Problems sharing a grid length and rank bound run
    in one launch per pass.  Data is packed: coefficients are one tensor of sum(N)
    values, problem i's at ``offN[i]:offN[i+1]``; samples, values and cotangents one of
    sum(M), problem i's at ``offM[i]:offM[i+1]``.

    graph : replay a CUDA graph of the launches when called again with the same tensors
    per_problem : each problem runs its own plan's launches (no batched launches)
    persistent : every batched class of a direction in one persistent launch
    autotune : tune each problem's grid and split (see :class:`Plan`)
    L : optional per-problem grid sizes (0 = default)
    """

    def __init__(self, Ns, xs, eps, precision="f32", graph=False, autotune=False, L=None, device=None,
                 per_problem=False, persistent=False):
        import numpy as np
        lib = _lib.load()
        device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = device
        self.count = len(Ns)
        xs = [torch.as_tensor(x).detach().to(device=device, dtype=torch.float64).reshape(-1) for x in xs]
        if len(xs) != self.count:
            raise ValueError("one sample vector per problem")
        epsv = np.broadcast_to(np.asarray(eps, dtype=np.float64), (self.count,)).copy()
        self.N = np.asarray(Ns, dtype=np.int64)
        self.M = np.asarray([x.numel() for x in xs], dtype=np.int64)
        self.offN = np.concatenate([[0], np.cumsum(self.N)])
        self.offM = np.concatenate([[0], np.cumsum(self.M)])
        self.prec = _prec(precision)
        self.cdtype = _CDTYPE[self.prec]
        xp = torch.cat(xs) if self.count else torch.empty(0, dtype=torch.float64, device=device)
        Lv = np.zeros(self.count, dtype=np.int64) if L is None else np.asarray(L, dtype=np.int64)
        flags = ((NUFFT_BATCH_GRAPH if graph else 0) | (NUFFT_PLAN_AUTOTUNE if autotune else 0)
                 | (NUFFT_BATCH_PER_PROBLEM if per_problem else 0) | (NUFFT_BATCH_PERSISTENT if persistent else 0))
        h = ctypes.c_void_p()
        with torch.cuda.device(device):
            rc = lib.nufft2_plan_many(ctypes.byref(h), self.count, self.N.ctypes.data, self.M.ctypes.data,
                                      Lv.ctypes.data, _ptr(xp) if xp.numel() else None, epsv.ctypes.data,
                                      self.prec, flags, _stream(device))
        check(rc, "nufft2_plan_many")
        self._h = h
        ncls, tn, tm = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        K = np.zeros(self.count, dtype=np.int32)
        Lo = np.zeros(self.count, dtype=np.int64)
        check(lib.nufft_batch_info(h, ctypes.byref(ncls), ctypes.byref(tn), ctypes.byref(tm), K.ctypes.data,
                                   Lo.ctypes.data), "nufft_batch_info")
        self.classes, self.total_N, self.total_M = ncls.value, tn.value, tm.value
        self.K, self.L = K, Lo
        nl = ctypes.c_int64()
        check(lib.nufft_batch_launches(h, ctypes.byref(nl)), "nufft_batch_launches")
        self.launches_per_direction = nl.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            torch.cuda.synchronize(self.device)
            _lib.load().nufft_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _cx(self, t, n, name):
        if t.device != self.device or t.dtype != self.cdtype or not t.is_contiguous() or t.numel() != n:
            raise ValueError("%s must be a contiguous %s tensor of %d elements on %s"
                             % (name, self.cdtype, n, self.device))
        return t

    def _run(self, fn, a, na, b, nb, what):
        self._cx(a, na, "input")
        self._cx(b, nb, "output")
        with torch.cuda.device(self.device):
            check(fn(self._h, _ptr(a), _ptr(b), _stream(self.device)), what)
        return b

    def forward(self, c, out=None):
        """f_i = A_i c_i for every problem (packed)."""
        f = out if out is not None else torch.empty(self.total_M, dtype=self.cdtype, device=self.device)
        return self._run(_lib.load().nufft2_exec_many, c, self.total_N, f, self.total_M, "nufft2_exec_many")

    def adjoint(self, g, out=None):
        """c_i = A_i^H g_i for every problem (packed)."""
        c = out if out is not None else torch.empty(self.total_N, dtype=self.cdtype, device=self.device)
        return self._run(_lib.load().nufft1_exec_many, g, self.total_M, c, self.total_N, "nufft1_exec_many")

    def forward_each(self, c, out=None):
        """The forward with one single-plan exec per problem (the per-problem comparator)."""
        f = out if out is not None else torch.empty(self.total_M, dtype=self.cdtype, device=self.device)
        self._cx(c, self.total_N, "c")
        self._cx(f, self.total_M, "f")
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_exec_each(self._h, _ptr(c), _ptr(f), 0, _stream(self.device)),
                  "nufft2_exec_each")
        return f

    def adjoint_each(self, g, out=None):
        """The adjoint with one single-plan exec per problem."""
        c = out if out is not None else torch.empty(self.total_N, dtype=self.cdtype, device=self.device)
        self._cx(g, self.total_M, "g")
        self._cx(c, self.total_N, "c")
        with torch.cuda.device(self.device):
            check(_lib.load().nufft2_exec_each(self._h, _ptr(c), _ptr(g), 1, _stream(self.device)),
                  "nufft2_exec_each")
        return c

    def check(self):
        """Synchronise and raise NufftError(NUFFT_ETIMEOUT) if a device-side wait gave up."""
        with torch.cuda.device(self.device):
            check(_lib.load().nufft_batch_check(self._h, _stream(self.device)), "nufft_batch_check")
