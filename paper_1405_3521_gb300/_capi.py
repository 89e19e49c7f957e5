"""ctypes binding of the C ABI declared in include/hjb.h.

Argument marshalling only: every step of every solve runs in the CUDA
library libhjb.so.  The binding refuses to run when the library is missing
(there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HJB_LIBRARY may point at another build of the same library (for A/B
# comparisons of compile-time tuning); the default is the in-tree build.
LIB_PATH = os.environ.get("HJB_LIBRARY") or os.path.join(_HERE, "_build", "libhjb.so")

HJB_OK = 0
HJB_ERR_INVALID_ARG = -1
HJB_ERR_CUDA = -2
HJB_ERR_OOM = -3
HJB_ERR_NOT_CONVERGED = -4
HJB_ERR_UNSUPPORTED = -5
HJB_ERR_TIMEOUT = -6
HJB_DYN_SPEED_CURRENT = 0
HJB_DYN_DUBINS = 1
HJB_WEIGHTS_EXP = 0
HJB_WEIGHTS_IMPLICIT = 1
HJB_INTERP_Q1 = 0
HJB_INTERP_P1 = 1
HJB_SUBDOMAIN_TARGETS_ALL = 0
HJB_SUBDOMAIN_TARGETS_OWN = 1

EXPORTS = ["hjb_create", "hjb_destroy", "hjb_solve", "hjb_subdomains", "hjb_solve_decomposed",
           "hjb_solve_batch", "hjb_backward", "hjb_point_values", "hjb_solve_static",
           "hjb_tune_get", "hjb_tune_set", "hjb_tune_load", "hjb_tune_save", "hjb_tune_clear",
           "hjb_last_error", "hjb_version"]


class HJBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hjb error %d: %s" % (code, msg))
        self.code = code


class NotConverged(HJBError):
    pass


class hjb_grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("periodic", C.c_int * 3)]


class hjb_dynamics(C.Structure):
    _fields_ = [("kind", C.c_int), ("speed", C.c_void_p), ("current", C.c_void_p),
                ("log_speed", C.c_void_p), ("dubins_v", C.c_double), ("scale", C.c_void_p)]


class hjb_cost(C.Structure):
    _fields_ = [("l", C.c_void_p), ("l_const", C.c_double)]


class hjb_discount(C.Structure):
    _fields_ = [("h", C.c_double), ("lam", C.c_double), ("weights", C.c_int), ("interp", C.c_int)]


class hjb_controls(C.Structure):
    _fields_ = [("count", C.c_int), ("dim", C.c_int), ("a", C.c_void_p), ("count_b", C.c_int),
                ("b", C.c_void_p)]


class hjb_target(C.Structure):
    _fields_ = [("labels", C.c_void_p), ("n_targets", C.c_int), ("value_out", C.c_double)]


class hjb_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iters", C.c_int), ("use_w_form", C.c_int),
                ("v_init", C.c_void_p), ("sweeps_per_check", C.c_int),
                ("local_iters", C.c_int), ("subdomain_targets", C.c_int),
                ("n_subdomains", C.c_int), ("warm_start", C.c_int)]


class hjb_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("node_updates", C.c_longlong),
                ("final_residual", C.c_double), ("ms", C.c_double), ("ties", C.c_longlong),
                ("labelled", C.c_longlong), ("launches", C.c_longlong), ("tile_rows", C.c_int),
                ("tile_lanes", C.c_int),
                ("delta", C.c_double), ("lipschitz", C.c_double), ("local_iters", C.c_int),
                ("subdomains", C.c_int), ("largest", C.c_longlong), ("tile_visits", C.c_longlong),
                ("tile_layers", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hjb_tune_choice(C.Structure):
    _fields_ = [("tile_rows", C.c_int), ("lanes", C.c_int), ("local_iters", C.c_int),
                ("ms", C.c_double), ("layers", C.c_int)]


class hjb_ra_opts(C.Structure):
    _fields_ = [("coarse_stride", C.c_int * 3), ("h_coarse", C.c_double), ("delta", C.c_double),
                ("C", C.c_double), ("M", C.c_double), ("q", C.c_double), ("tol", C.c_double),
                ("max_iters", C.c_int), ("max_splits", C.c_int), ("split_gain", C.c_double),
                ("split_labels", C.c_void_p)]


_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libhjb.so is not built: run `python -c \"import __graft_entry__ as g; "
                              "g.build()\"` or `python -m paper_1405_3521_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i = C.c_void_p, C.c_int
        P = C.c_void_p
        L.hjb_create.argtypes = [C.POINTER(hjb_grid), C.POINTER(hjb_dynamics), C.POINTER(hjb_cost),
                                 C.POINTER(hjb_discount), C.POINTER(hjb_controls),
                                 C.POINTER(hjb_target), C.POINTER(C.c_void_p)]
        L.hjb_destroy.argtypes = [P]
        L.hjb_solve.argtypes = [P, C.POINTER(hjb_solve_opts), vp, C.POINTER(hjb_stats), vp]
        L.hjb_subdomains.argtypes = [P, C.POINTER(hjb_ra_opts), vp, vp, vp, C.POINTER(hjb_stats), vp]
        L.hjb_solve_decomposed.argtypes = [P, vp, C.POINTER(hjb_solve_opts), vp,
                                           C.POINTER(hjb_stats), C.POINTER(hjb_stats), vp]
        L.hjb_solve_batch.argtypes = [C.POINTER(C.c_void_p), i, C.POINTER(hjb_solve_opts),
                                      C.POINTER(C.c_void_p), C.POINTER(hjb_stats), vp]
        L.hjb_backward.argtypes = [P, vp, vp, i, C.POINTER(hjb_solve_opts), vp,
                                   C.POINTER(hjb_stats), vp]
        L.hjb_point_values.argtypes = [P, vp, vp, i, vp, vp, vp]
        L.hjb_solve_static.argtypes = [C.POINTER(hjb_grid), C.POINTER(hjb_dynamics),
                                       C.POINTER(hjb_cost), C.POINTER(hjb_discount),
                                       C.POINTER(hjb_controls), C.POINTER(hjb_target),
                                       C.POINTER(hjb_solve_opts), vp, C.POINTER(hjb_stats), vp]
        L.hjb_tune_get.argtypes = [C.c_char_p, C.POINTER(hjb_tune_choice)]
        L.hjb_tune_set.argtypes = [C.c_char_p, C.POINTER(hjb_tune_choice)]
        L.hjb_tune_load.argtypes = [C.c_char_p, C.POINTER(C.c_int)]
        L.hjb_tune_save.argtypes = [C.c_char_p]
        L.hjb_tune_clear.argtypes = []
        L.hjb_last_error.restype = C.c_char_p
        L.hjb_version.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("hjb_last_error", "hjb_version"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def check(rc, allow_not_converged=False):
    if rc == HJB_OK:
        return
    msg = lib().hjb_last_error().decode()
    if rc == HJB_ERR_NOT_CONVERGED:
        if allow_not_converged:
            return
        raise NotConverged(rc, msg)
    raise HJBError(rc, msg)
