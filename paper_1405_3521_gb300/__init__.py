"""GB300-native semi-Lagrangian value iteration for Hamilton-Jacobi-Bellman
equations and the independent sub-domain method of Festa (arXiv:1405.3521).

Python surface over the C ABI of include/hjb.h (marshalling only; the work
runs in the sm_103a CUDA library, which must be built first):

    Problem(...)                    hjb_create / hjb_destroy
    solve(p, ...)                   hjb_solve            (Sec. 3, value iteration)
    subdomains(p, ...)              hjb_subdomains       (RA, Sec. 3; ISA steps 1-2)
    solve_decomposed(p, mask, ...)  hjb_solve_decomposed (ISA steps 3-4, Sec. 4)
    solve_batch([p, ...], ...)      hjb_solve_batch
    backward(p, v, grad_v, wrt)     hjb_backward         (adjoint, pi frozen)
    point_values(p, v, pts)         hjb_point_values
    solve_static(p, ...)            hjb_solve_static     (no device allocation)
    HJBSolve.apply(theta, spec)     autograd: V(theta) for s = exp(theta)

Arrays may be CUDA torch tensors or host numpy arrays.  Outputs follow the
labels array: torch on the GPU when the labels are a CUDA tensor, numpy
otherwise.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _capi
from ._capi import (HJB_DYN_DUBINS, HJB_DYN_SPEED_CURRENT, HJB_WEIGHTS_EXP, HJB_WEIGHTS_IMPLICIT,
                    HJB_INTERP_Q1, HJB_INTERP_P1, HJB_SUBDOMAIN_TARGETS_ALL,
                    HJB_SUBDOMAIN_TARGETS_OWN, HJBError, NotConverged, check,
                    hjb_ra_opts, hjb_solve_opts, hjb_stats)

__all__ = ["Problem", "solve", "subdomains", "solve_decomposed", "solve_batch", "backward",
           "point_values", "solve_static", "HJBSolve", "point_loss", "HJBError", "NotConverged", "library_path",
           "version", "pinned_empty", "pinned_copy"]


def library_path():
    return _capi.LIB_PATH


def version():
    return _capi.lib().hjb_version().decode()


def _is_torch(x):
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(x, torch.Tensor)


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        assert x.is_contiguous(), "tensors must be contiguous"
        return x.data_ptr()
    assert x.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
    return x.ctypes.data


def _as_dtype(x, dtype):
    """Contiguous view/copy of x with the requested element type."""
    if x is None:
        return None
    if _is_torch(x):
        import torch
        tdt = {np.float32: torch.float32, np.uint8: torch.uint8, np.uint32: torch.int32}[dtype]
        return x.to(tdt).contiguous()
    return np.ascontiguousarray(x, dtype=dtype)


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:  # pragma: no cover
        pass
    return None


def _opts(tol=0.0, max_iters=0, use_w_form=-1, v_init=None, sweeps_per_check=0, local_iters=0,
          subdomain_targets=0, n_subdomains=0, warm_start=0):
    o = hjb_solve_opts()
    o.n_subdomains = int(n_subdomains)
    o.warm_start = int(warm_start)
    o.tol = float(tol)
    o.max_iters = int(max_iters)
    o.use_w_form = int(use_w_form)
    o.v_init = _ptr(v_init)
    o.sweeps_per_check = int(sweeps_per_check)
    o.local_iters = int(local_iters)
    o.subdomain_targets = int(subdomain_targets)
    return o


class Problem:
    """A discrete HJB problem (Sec. 2-3 of the paper) on a structured grid.

    shape: nodes per dimension (x first); lo/hi: the box (period for the
    periodic heading of the Dubins car); controls: [A, 2] vectors (speed /
    current dynamics) or [A, 1] turn rates (Dubins); labels: target labels
    per node (0 free, k target component k); speed / log_speed / scale
    (per-axis factors [N, 2]) / current / cost: optional node fields; h, lam:
    time step and discount rate; weights: 0 = exp(-lam h) step weights, 1 = the
    1 / (1 + lam h) weights of the printed scheme; interp: 0 = Q1, 1 = P1 on
    the Kuhn triangles of each cell (2D); controls_b: the second
    player's set of a differential game ([B, 2], f = D (a - b) + c).
    Node arrays are in (z,) y, x order with x fastest.
    """

    def __init__(self, shape, lo, hi, controls, labels, h, lam=1.0, n_targets=None,
                 dyn=HJB_DYN_SPEED_CURRENT, speed=None, current=None, log_speed=None,
                 dubins_v=1.0, cost=None, cost_const=1.0, value_out=1.0, periodic=None,
                 scale=None, controls_b=None, weights=0, interp=0):
        L = _capi.lib()
        nd = len(shape)
        self.shape = tuple(int(s) for s in shape)
        self.ndim = nd
        self.N = int(np.prod(self.shape))
        self.labels = _as_dtype(labels, np.uint8).reshape(-1)
        self.speed = None if speed is None else _as_dtype(speed, np.float32).reshape(-1)
        self.current = None if current is None else _as_dtype(current, np.float32).reshape(-1)
        self.log_speed = None if log_speed is None else _as_dtype(log_speed, np.float32).reshape(-1)
        self.cost = None if cost is None else _as_dtype(cost, np.float32).reshape(-1)
        self.scale = None if scale is None else _as_dtype(scale, np.float32).reshape(-1)
        self.controls_b = None if controls_b is None else np.ascontiguousarray(
            np.asarray(controls_b, dtype=np.float32).reshape(len(controls_b), -1))
        self.controls = np.ascontiguousarray(np.asarray(controls, dtype=np.float32).reshape(
            len(controls), -1))
        self.on_gpu = _is_torch(self.labels) and self.labels.is_cuda
        if n_targets is None:
            lab = self.labels.cpu().numpy() if _is_torch(self.labels) else self.labels
            n_targets = int(lab.max())
        self.n_targets = int(n_targets)
        self.h, self.lam, self.value_out = float(h), float(lam), float(value_out)
        self.lo, self.hi = list(lo), list(hi)
        per = [0, 0, 0] if periodic is None else list(periodic) + [0] * (3 - len(periodic))
        g = _capi.hjb_grid()
        g.ndim = nd
        for d in range(3):
            g.n[d] = self.shape[d] if d < nd else 1
            g.lo[d] = float(lo[d]) if d < nd else 0.0
            g.hi[d] = float(hi[d]) if d < nd else 1.0
            g.periodic[d] = int(per[d])
        dy = _capi.hjb_dynamics()
        dy.kind = int(dyn)
        dy.speed = _ptr(self.speed)
        dy.current = _ptr(self.current)
        dy.log_speed = _ptr(self.log_speed)
        dy.dubins_v = float(dubins_v)
        dy.scale = _ptr(self.scale)
        co = _capi.hjb_cost()
        co.l = _ptr(self.cost)
        co.l_const = float(cost_const)
        di = _capi.hjb_discount()
        di.h = float(h)
        di.lam = float(lam)
        di.weights = int(weights)
        di.interp = int(interp)
        ct = _capi.hjb_controls()
        ct.count = self.controls.shape[0]
        ct.dim = self.controls.shape[1]
        ct.a = self.controls.ctypes.data
        if self.controls_b is not None:
            ct.count_b = self.controls_b.shape[0]
            ct.b = self.controls_b.ctypes.data
        tg = _capi.hjb_target()
        tg.labels = _ptr(self.labels)
        tg.n_targets = self.n_targets
        tg.value_out = float(value_out)
        self._grid = g
        self._desc = (g, dy, co, di, ct, tg)  # kept for hjb_solve_static
        self._handle = C.c_void_p()
        check(L.hjb_create(C.byref(g), C.byref(dy), C.byref(co), C.byref(di), C.byref(ct),
                           C.byref(tg), C.byref(self._handle)))

    @property
    def handle(self):
        return self._handle

    def close(self):
        if getattr(self, "_handle", None) and self._handle.value:
            _capi.lib().hjb_destroy(self._handle)
            self._handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self, n, dtype=np.float32):
        """Output array of n elements on the problem's side: a CUDA tensor, or
        for host problems a numpy array in page-locked memory (so that the
        library's device-to-host copies run at full speed) when torch can
        allocate it, else an ordinary numpy array."""
        if self.on_gpu:
            import torch
            tdt = {np.float32: torch.float32, np.uint32: torch.int32}[dtype]
            return torch.empty(n, dtype=tdt, device=self.labels.device)
        return pinned_empty(n, dtype)


def pinned_empty(n, dtype=np.float32):
    """numpy array of n elements in page-locked host memory (ordinary memory
    when CUDA is not available)."""
    try:
        import torch
        if torch.cuda.is_available():
            tdt = {np.float32: torch.float32, np.uint32: torch.int32, np.uint8: torch.uint8}[dtype]
            return torch.empty(n, dtype=tdt, pin_memory=True).numpy().view(dtype)
    except (ImportError, RuntimeError, KeyError):
        pass
    return np.empty(n, dtype=dtype)


def pinned_copy(a, dtype=np.float32):
    """Copy of an array in page-locked host memory (see pinned_empty)."""
    a = np.ascontiguousarray(np.asarray(a), dtype=dtype)
    out = pinned_empty(a.size, dtype).reshape(a.shape)
    out[...] = a
    return out


def solve(p: Problem, tol=0.0, max_iters=0, use_w_form=-1, v_init=None, sweeps_per_check=0,
          out=None, stream=None, allow_not_converged=False, local_iters=0):
    """Value iteration (Sec. 3).  Returns (V, stats dict).  local_iters:
    applications of T per staged tile and sweep (1 = plain Jacobi value
    iteration, 0 = library default)."""
    out = p.empty(p.N) if out is None else out
    st = hjb_stats()
    o = _opts(tol, max_iters, use_w_form, v_init, sweeps_per_check, local_iters)
    rc = _capi.lib().hjb_solve(p.handle, C.byref(o), _ptr(out), C.byref(st), _stream(stream))
    check(rc, allow_not_converged)
    return out, st.as_dict()


def solve_static(p: Problem, tol=0.0, max_iters=0, v_init=None, out=None, stream=None,
                 local_iters=0):
    """hjb_solve_static on the problem's descriptors: the full-domain solve
    without any device allocation (device arrays only, bounded grid size).
    Returns (V, stats dict)."""
    out = p.empty(p.N) if out is None else out
    st = hjb_stats()
    o = _opts(tol, max_iters, -1, v_init, 0, local_iters)
    g, dy, co, di, ct, tg = p._desc
    check(_capi.lib().hjb_solve_static(C.byref(g), C.byref(dy), C.byref(co), C.byref(di),
                                       C.byref(ct), C.byref(tg), C.byref(o), _ptr(out),
                                       C.byref(st), _stream(stream)))
    return out, st.as_dict()


def subdomains(p: Problem, stride, delta=-1.0, C_=0.0, M=-1.0, q=1.0, h_coarse=0.0, tol=0.0,
               max_iters=0, want_aux=False, stream=None, max_splits=0, split_gain=0.0,
               split_labels=None):
    """RA (Sec. 3) + projection (ISA step 2).  Returns (fine_mask, coarse_labels,
    v_aux or None, stats).  delta < 0: 2 (C dx_K^q + M dx_K), M < 0 estimated
    from the coarse solution.  max_splits > 0 re-splits the target components
    recursively (split_labels, optional [N] uint8 output: the final division;
    stats["subdomains"] its component count)."""
    ra = hjb_ra_opts()
    ra.max_splits = int(max_splits)
    ra.split_gain = float(split_gain)
    ra.split_labels = _ptr(split_labels)
    for d in range(3):
        ra.coarse_stride[d] = int(stride[d]) if d < len(stride) else 1
    ra.h_coarse = float(h_coarse)
    ra.delta = float(delta)
    ra.C, ra.M, ra.q = float(C_), float(M), float(q)
    ra.tol = float(tol)
    ra.max_iters = int(max_iters)
    nk = []
    for d in range(p.ndim):
        r = int(stride[d])
        per = p._grid.periodic[d]
        nk.append(p.shape[d] // r if per else (p.shape[d] - 1) // r + 1)
    NK = int(np.prod(nk))
    fine = p.empty(p.N, np.uint32)
    coarse = p.empty(NK, np.uint32)
    aux = p.empty(p.n_targets * NK) if want_aux else None
    st = hjb_stats()
    check(_capi.lib().hjb_subdomains(p.handle, C.byref(ra), _ptr(fine), _ptr(coarse), _ptr(aux),
                                     C.byref(st), _stream(stream)))
    return fine, coarse, aux, st.as_dict()


def solve_decomposed(p: Problem, fine_mask, tol=0.0, max_iters=0, use_w_form=-1,
                     sweeps_per_check=0, out=None, stream=None, local_iters=0,
                     subdomain_targets=0, n_subdomains=0, v_init=None, warm_start=0):
    """ISA steps 3-4 (Sec. 4).  Returns (Vbar, per-sub-domain stats, total stats).
    subdomain_targets: 0 = every target node inside a sub-domain is its
    target (Sec. 4 step 3 as written), 1 = only its own component (the
    target choice of RA step 1, Sec. 3).  n_subdomains: bits of fine_mask
    (0: n_targets; more after re-splitting).  v_init: warm start of every
    sub-domain; warm_start=1: start from the last reconstruction's coarse
    auxiliary solutions interpolated onto the fine grid."""
    out = p.empty(p.N) if out is None else out
    per = (hjb_stats * max(p.n_targets, int(n_subdomains)))()
    tot = hjb_stats()
    o = _opts(tol, max_iters, use_w_form, v_init, sweeps_per_check, local_iters, subdomain_targets,
              n_subdomains, warm_start)
    check(_capi.lib().hjb_solve_decomposed(p.handle, _ptr(fine_mask), C.byref(o), _ptr(out), per,
                                           C.byref(tot), _stream(stream)))
    return out, [s.as_dict() for s in per], tot.as_dict()


def solve_batch(problems, tol=0.0, max_iters=0, use_w_form=-1, sweeps_per_check=0, outs=None,
                stream=None, local_iters=0):
    """Many problems in one persistent launch.  Returns (list of V, list of stats)."""
    n = len(problems)
    outs = [p.empty(p.N) for p in problems] if outs is None else outs
    hs = (C.c_void_p * n)(*[p.handle.value for p in problems])
    os_ = (C.c_void_p * n)(*[_ptr(o) for o in outs])
    per = (hjb_stats * n)()
    o = _opts(tol, max_iters, use_w_form, None, sweeps_per_check, local_iters)
    check(_capi.lib().hjb_solve_batch(hs, n, C.byref(o), os_, per, _stream(stream)))
    return outs, [s.as_dict() for s in per]


def backward(p: Problem, v, grad_v, wrt=0, tol=0.0, max_iters=0, out=None, stream=None):
    """Adjoint of the converged solve: dL/dtheta (wrt=0) or dL/dl (wrt=1)."""
    out = p.empty(p.N) if out is None else out
    st = hjb_stats()
    o = _opts(tol, max_iters)
    check(_capi.lib().hjb_backward(p.handle, _ptr(v), _ptr(grad_v), int(wrt), C.byref(o),
                                   _ptr(out), C.byref(st), _stream(stream)))
    return out, st.as_dict()


def point_values(p: Problem, v, points, with_grad=True, stream=None):
    """I[V] at points [P, 2] and the gradient of their mean w.r.t. V."""
    npts = int(points.shape[0])
    vals = p.empty(npts)
    grad = p.empty(p.N) if with_grad else None
    check(_capi.lib().hjb_point_values(p.handle, _ptr(v), _ptr(points), npts, _ptr(vals),
                                       _ptr(grad), _stream(stream)))
    return vals, grad


try:
    import torch

    class HJBSolve(torch.autograd.Function):
        """V(theta) for f = exp(theta) a (+ c): forward = hjb_solve, backward =
        hjb_backward(wrt=0) with the optimal policy recomputed from V.

        spec: dict with the Problem keyword arguments other than log_speed."""

        @staticmethod
        def forward(ctx, theta, spec, tol=0.0):
            th = theta.detach().contiguous().to(torch.float32)
            p = Problem(log_speed=th, **spec)
            v, _ = solve(p, tol=tol)
            ctx.problem = p
            ctx.theta = th
            ctx.save_for_backward(v)
            return v

        @staticmethod
        def backward(ctx, grad_v):
            (v,) = ctx.saved_tensors
            g, _ = backward(ctx.problem, v, grad_v.contiguous().to(torch.float32), wrt=0)
            return g.view_as(ctx.theta), None, None

    class _PointLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v, problem, points):
            vals, grad = point_values(problem, v.detach().contiguous(), points)
            ctx.save_for_backward(grad)
            return vals.mean()

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            return grad * gout, None, None

    def point_loss(v, problem, points):
        """L = mean_p I[V](points_p) with its gradient computed by the library."""
        return _PointLoss.apply(v, problem, points)

except ImportError:  # pragma: no cover
    HJBSolve = None
    point_loss = None
