"""FP64 CPU oracle for semi-Lagrangian value iteration and the independent
sub-domain method (Festa, arXiv:1405.3521, Sec. 3-4).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg, never by the library.  The arithmetic lives
in ``hjb_oracle.c`` (plain C, FP64); this module compiles it with gcc and
marshals numpy arrays through ctypes.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hjb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (OpenMP when gcc has it)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Prob(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("periodic", C.c_int * 3), ("dyn", C.c_int),
        ("speed", C.c_void_p), ("current", C.c_void_p), ("dubins_v", C.c_double),
        ("cost", C.c_void_p), ("cost_const", C.c_double),
        ("h", C.c_double), ("lam", C.c_double),
        ("ncontrols", C.c_int), ("cdim", C.c_int), ("controls", C.c_void_p),
        ("target", C.c_void_p), ("ntargets", C.c_int), ("v_out", C.c_double),
        ("scale", C.c_void_p), ("nb", C.c_int), ("controls_b", C.c_void_p),
        ("weights", C.c_int), ("interp", C.c_int),
    ]


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.POINTER(_Prob)
            vp, d, i = C.c_void_p, C.c_double, C.c_int
            lib.ohjb_interp.argtypes = [P, vp, vp]
            lib.ohjb_interp.restype = d
            lib.ohjb_apply.argtypes = [P, vp, vp, vp, vp, i, i, i]
            lib.ohjb_apply.restype = d
            lib.ohjb_initial.argtypes = [P, vp, vp, i, i]
            lib.ohjb_solve.argtypes = [P, d, i, vp, vp, i, i, i, C.POINTER(d)]
            lib.ohjb_solve.restype = i
            lib.ohjb_solve_gs.argtypes = [P, d, i, vp, vp, i, i, C.POINTER(d)]
            lib.ohjb_solve_gs.restype = i
            lib.ohjb_coarse_shape.argtypes = [P, vp, vp]
            lib.ohjb_coarse_shape.restype = i
            lib.ohjb_label.argtypes = [C.c_longlong, i, vp, vp, d, d, vp, vp]
            lib.ohjb_label.restype = C.c_longlong
            lib.ohjb_delta.argtypes = [P, vp, vp, d, d, d, C.POINTER(d)]
            lib.ohjb_delta.restype = d
            lib.ohjb_ra.argtypes = [P, vp, d, d, d, i, vp, vp, i]
            lib.ohjb_ra.restype = C.c_longlong
            lib.ohjb_project.argtypes = [P, vp, vp, vp]
            lib.ohjb_ra_split.argtypes = [P, vp, d, d, d, i, i, d, i, vp, vp, C.POINTER(i)]
            lib.ohjb_ra_split.restype = C.c_longlong
            lib.ohjb_isa.argtypes = [P, vp, d, i, i, vp, vp, vp, i, i]
            lib.ohjb_isa.restype = C.c_longlong
            lib.ohjb_policy.argtypes = [P, vp, vp, i]
            lib.ohjb_policy.restype = d
            lib.ohjb_adjoint.argtypes = [P, vp, vp, d, i, vp, C.POINTER(d)]
            lib.ohjb_adjoint.restype = i
            lib.ohjb_grad.argtypes = [P, vp, vp, vp, vp, vp]
            lib.ohjb_points.argtypes = [P, vp, vp, i, vp, vp]
            lib.ohjb_tie_influence.argtypes = [P, vp, vp, d, d, i, vp, vp]
            lib.ohjb_tie_influence.restype = C.c_longlong
            lib.ohjb_max_threads.restype = i
            _lib = lib
    return _lib


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


class Problem:
    """A discretised problem in the notation of Sec. 2-3 of the paper.

    shape: nodes per dimension (x first).  lo/hi: box (period for periodic
    dims).  dyn: 0 for f = s a + c, 1 for the Dubins car.  controls: [A, cdim].
    target: int labels per node (0 free, k >= 1 component k), shaped like the
    grid in (z, y, x) order or flat.  Fields are node arrays in the same order.
    """

    def __init__(self, shape, lo, hi, controls, target, h, lam=1.0, periodic=None,
                 dyn=0, speed=None, current=None, dubins_v=1.0, cost=None,
                 cost_const=1.0, v_out=1.0, ntargets=None, scale=None, controls_b=None,
                 weights=0, interp=0):
        self.ndim = len(shape)
        self.shape = tuple(int(s) for s in shape)
        self.N = int(np.prod(self.shape))
        self.controls = _f64(np.asarray(controls, dtype=np.float64).reshape(len(controls), -1))
        self.target = np.ascontiguousarray(np.asarray(target).reshape(-1), dtype=np.int32)
        assert self.target.size == self.N
        self.speed = _f64(None if speed is None else np.asarray(speed).reshape(-1))
        self.current = _f64(None if current is None else np.asarray(current).reshape(-1, 2))
        self.cost = _f64(None if cost is None else np.asarray(cost).reshape(-1))
        self.scale = _f64(None if scale is None else np.asarray(scale).reshape(-1, 2))
        self.controls_b = None if controls_b is None else _f64(
            np.asarray(controls_b, dtype=np.float64).reshape(len(controls_b), -1))
        self.ntargets = int(self.target.max()) if ntargets is None else int(ntargets)
        per = [0, 0, 0] if periodic is None else list(periodic) + [0] * (3 - len(periodic))
        s = _Prob()
        s.ndim = self.ndim
        for d in range(3):
            s.n[d] = self.shape[d] if d < self.ndim else 1
            s.lo[d] = float(lo[d]) if d < self.ndim else 0.0
            s.hi[d] = float(hi[d]) if d < self.ndim else 1.0
            s.periodic[d] = int(per[d])
        s.dyn = int(dyn)
        s.speed = _ptr(self.speed)
        s.current = _ptr(self.current)
        s.dubins_v = float(dubins_v)
        s.cost = _ptr(self.cost)
        s.cost_const = float(cost_const)
        s.h = float(h)
        s.lam = float(lam)
        s.ncontrols = self.controls.shape[0]
        s.cdim = self.controls.shape[1]
        s.controls = _ptr(self.controls)
        s.target = _ptr(self.target)
        s.ntargets = self.ntargets
        s.v_out = float(v_out)
        s.scale = _ptr(self.scale)
        s.nb = 0 if self.controls_b is None else self.controls_b.shape[0]
        s.controls_b = _ptr(self.controls_b)
        s.weights = int(weights)
        s.interp = int(interp)
        self._s = s
        self.h, self.lam, self.v_out = float(h), float(lam), float(v_out)
        self.lo, self.hi, self.periodic = list(lo), list(hi), per[: self.ndim]

    @property
    def beta(self):
        if self._s.weights == 1:
            return 1.0 / (1.0 + self.lam * self.h)
        return float(np.exp(-self.lam * self.h))

    def spacing(self, d):
        n = self.shape[d]
        return (self.hi[d] - self.lo[d]) / (n if self.periodic[d] else n - 1)

    def _ref(self):
        return C.byref(self._s)


def _mask_args(mask, bit):
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint32).reshape(-1)
    return m, int(bit)


def initial(p: Problem, mask=None, bit=0, only_target=0):
    V = np.empty(p.N)
    m, b = _mask_args(mask, bit)
    _lib_handle().ohjb_initial(p._ref(), V.ctypes.data, _ptr(m), b, int(only_target))
    return V


def apply(p: Problem, V, mask=None, bit=0, only_target=0, nthreads=1, with_policy=False):
    """One application of T (Sec. 3, eq. Tdef).  Returns (T(V), residual[, policy])."""
    V = _f64(V).reshape(-1)
    out = np.empty(p.N)
    pol = np.empty(p.N, dtype=np.int32) if with_policy else None
    m, b = _mask_args(mask, bit)
    r = _lib_handle().ohjb_apply(p._ref(), V.ctypes.data, out.ctypes.data, _ptr(pol),
                                 _ptr(m), b, int(only_target), int(nthreads))
    return (out, r, pol) if with_policy else (out, r)


def solve(p: Problem, tol=1e-12, max_iters=1_000_000, V0=None, mask=None, bit=0,
          only_target=0, nthreads=1, gs=False):
    """Value iteration to ||V^{n+1}-V^n||_inf <= tol.  Returns (V, iterations, residual)."""
    m, b = _mask_args(mask, bit)
    V = initial(p, mask, bit, only_target) if V0 is None else _f64(V0).reshape(-1).copy()
    r = C.c_double(0.0)
    lib = _lib_handle()
    if gs:
        it = lib.ohjb_solve_gs(p._ref(), float(tol), int(max_iters), V.ctypes.data, _ptr(m), b,
                               int(only_target), C.byref(r))
    else:
        it = lib.ohjb_solve(p._ref(), float(tol), int(max_iters), V.ctypes.data, _ptr(m), b,
                            int(only_target), int(nthreads), C.byref(r))
    return V, int(it), float(r.value)


def coarse_shape(p: Problem, stride):
    st = (C.c_int * 3)(*(list(stride) + [1] * (3 - len(stride))))
    nk = (C.c_int * 3)()
    if _lib_handle().ohjb_coarse_shape(p._ref(), st, nk) != 0:
        raise ValueError("stride does not divide the grid")
    return tuple(nk[d] for d in range(p.ndim))


def label(Vaux, target_coarse, delta, tie_eps=1e-6):
    """RA steps 2-3 on given auxiliary solutions Vaux[m, NK]."""
    Vaux = _f64(Vaux)
    m, NK = Vaux.shape
    t = np.ascontiguousarray(target_coarse, dtype=np.int32).reshape(-1)
    vmin = np.empty(NK)
    lab = np.empty(NK, dtype=np.uint32)
    ties = _lib_handle().ohjb_label(NK, m, Vaux.ctypes.data, t.ctypes.data, float(delta),
                                    float(tie_eps), vmin.ctypes.data, lab.ctypes.data)
    return vmin, lab, int(ties)


def ra(p: Problem, stride, delta, h_coarse=None, tol=1e-12, max_iters=1_000_000, nthreads=1):
    """RA (Sec. 3): auxiliary coarse solves, min, labels.  Returns (Vaux[m,NK], labels[NK], ties)."""
    nk = coarse_shape(p, stride)
    NK = int(np.prod(nk))
    st = (C.c_int * 3)(*(list(stride) + [1] * (3 - len(stride))))
    hc = p.h * stride[0] if h_coarse is None else float(h_coarse)
    Vaux = np.empty((p.ntargets, NK))
    lab = np.empty(NK, dtype=np.uint32)
    ties = _lib_handle().ohjb_ra(p._ref(), st, hc, float(delta), float(tol), int(max_iters),
                                 Vaux.ctypes.data, lab.ctypes.data, int(nthreads))
    if ties < 0:
        raise ValueError("bad stride")
    return Vaux, lab, int(ties)


def delta(p: Problem, stride, Vaux, C_=0.0, q=1.0, M=-1.0):
    """Threshold of RA step 3, 2 (C dx_K^q + M dx_K) (eq. rep, Prop. 3.1); M < 0
    estimates M by the largest discrete gradient norm of min_k V_k on the
    coarse grid (reading R5).  Returns (delta, M)."""
    st = (C.c_int * 3)(*(list(stride) + [1] * (3 - len(stride))))
    Va = _f64(Vaux)
    if Va.shape != (p.ntargets, int(np.prod(coarse_shape(p, stride)))):
        raise ValueError("Vaux must be [ntargets, coarse nodes]")
    Mo = C.c_double(0.0)
    dl = _lib_handle().ohjb_delta(p._ref(), st, Va.ctypes.data, float(C_), float(q), float(M),
                                  C.byref(Mo))
    if dl < 0:
        raise ValueError("stride does not divide the grid")
    return float(dl), float(Mo.value)


def project(p: Problem, stride, coarse_labels):
    """ISA step 2 (Sec. 4), reading R4.  Returns the fine bitmask [N]."""
    st = (C.c_int * 3)(*(list(stride) + [1] * (3 - len(stride))))
    cl = np.ascontiguousarray(coarse_labels, dtype=np.uint32).reshape(-1)
    out = np.empty(p.N, dtype=np.uint32)
    _lib_handle().ohjb_project(p._ref(), st, cl.ctypes.data, out.ctypes.data)
    return out


def ra_split(p: Problem, stride, delta, max_splits, min_gain=0.05, h_coarse=None, tol=1e-12,
             max_iters=1_000_000, nthreads=1):
    """Recursive re-splitting of the target components (Conclusions; reading
    R22): the component with the largest sub-domain is split in two, and the
    split is kept when both parts' sub-domains are smaller than (1 -
    min_gain) times its own.  Returns (components [N] int32, fine mask [N],
    m, largest)."""
    st = (C.c_int * 3)(*(list(stride) + [1] * (3 - len(stride))))
    hc = p.h * stride[0] if h_coarse is None else float(h_coarse)
    comp = np.empty(p.N, dtype=np.int32)
    fine = np.empty(p.N, dtype=np.uint32)
    m = C.c_int(0)
    largest = _lib_handle().ohjb_ra_split(p._ref(), st, hc, float(delta), float(tol),
                                          int(max_iters), int(max_splits), float(min_gain),
                                          int(nthreads),
                                          comp.ctypes.data, fine.ctypes.data, C.byref(m))
    if largest < 0:
        raise ValueError("bad stride")
    return comp, fine, int(m.value), int(largest)


def isa(p: Problem, fine_mask, tol=1e-12, max_iters=1_000_000, gs=False, keep_vk=False,
        nthreads=1, own_targets=False):
    """ISA steps 3-4 (Sec. 4).  Returns (Vbar, uncovered, iters[m], Vk or None).
    own_targets: sub-problem k keeps only target component k (the target
    choice of RA step 1, Sec. 3) instead of every target node inside it."""
    fm = np.ascontiguousarray(fine_mask, dtype=np.uint32).reshape(-1)
    Vbar = np.empty(p.N)
    Vk = np.empty((p.ntargets, p.N)) if keep_vk else None
    its = np.zeros(p.ntargets, dtype=np.int32)
    unc = _lib_handle().ohjb_isa(p._ref(), fm.ctypes.data, float(tol), int(max_iters), int(gs),
                                 _ptr(Vk), Vbar.ctypes.data, its.ctypes.data, int(nthreads),
                                 int(bool(own_targets)))
    return Vbar, int(unc), its, Vk


def policy(p: Problem, V, nthreads=1):
    V = _f64(V).reshape(-1)
    pol = np.empty(p.N, dtype=np.int32)
    r = _lib_handle().ohjb_policy(p._ref(), V.ctypes.data, pol.ctypes.data, int(nthreads))
    return pol, r


def adjoint(p: Problem, pol, g, tol=1e-13, max_iters=1_000_000):
    pol = np.ascontiguousarray(pol, dtype=np.int32).reshape(-1)
    g = _f64(g).reshape(-1)
    lam = np.empty(p.N)
    r = C.c_double(0.0)
    it = _lib_handle().ohjb_adjoint(p._ref(), pol.ctypes.data, g.ctypes.data, float(tol),
                                    int(max_iters), lam.ctypes.data, C.byref(r))
    return lam, int(it), float(r.value)


def grad(p: Problem, V, pol, lam):
    """(dL/dtheta for s = exp(theta), dL/dl)."""
    V = _f64(V).reshape(-1)
    pol = np.ascontiguousarray(pol, dtype=np.int32).reshape(-1)
    lam = _f64(lam).reshape(-1)
    gt = np.empty(p.N)
    gc = np.empty(p.N)
    _lib_handle().ohjb_grad(p._ref(), V.ctypes.data, pol.ctypes.data, lam.ctypes.data,
                            gt.ctypes.data, gc.ctypes.data)
    return gt, gc


def points(p: Problem, V, pts, with_grad=True):
    """Loss L = mean_p I[V](pts_p): (values[P], dL/dV[N] or None)."""
    V = _f64(V).reshape(-1)
    pts = _f64(pts).reshape(-1, p.ndim)
    P = pts.shape[0]
    vals = np.empty(P)
    g = np.empty(p.N) if with_grad else None
    _lib_handle().ohjb_points(p._ref(), V.ctypes.data, pts.ctypes.data, int(P), vals.ctypes.data,
                              _ptr(g))
    return vals, g


def tie_influence(p: Problem, V, pol, eps=1e-6, face_eps=1e-5, closure=True,
                  with_second=False):
    """Nodes whose policy or interpolant gradient is not unique (the two best
    controls within eps, or the chosen foot within face_eps cells of a cell
    face) and, with closure, everything downstream of them along the
    transposed policy map.  Returns a bool mask [N] (and, with_second, the
    runner-up control of every free node)."""
    V = _f64(V).reshape(-1)
    pol = np.ascontiguousarray(pol, dtype=np.int32).reshape(-1)
    out = np.empty(p.N, dtype=np.uint8)
    sec = np.empty(p.N, dtype=np.int32) if with_second else None
    _lib_handle().ohjb_tie_influence(p._ref(), V.ctypes.data, pol.ctypes.data, float(eps),
                                     float(face_eps), int(bool(closure)), out.ctypes.data,
                                     _ptr(sec))
    return (out.astype(bool), sec) if with_second else out.astype(bool)


def interp(p: Problem, V, y):
    V = _f64(V).reshape(-1)
    y = _f64(y).reshape(-1)
    return float(_lib_handle().ohjb_interp(p._ref(), V.ctypes.data, y.ctypes.data))


def max_threads():
    return int(_lib_handle().ohjb_max_threads())
