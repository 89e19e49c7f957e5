"""The allocation-free solve (hjb_solve_static) against the ordinary solve.

Some callers cannot allocate device memory while they run: real-time
control loops that forbid cudaMalloc/cudaFree after start-up (both may
synchronise the device), and plug-ins whose host application owns every
device allocation.  They use hjb_solve_static, which keeps its working
memory in one static device array.  This file is collected last so that a
run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import synthetic as S
from _cases import gpu_problem, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hjb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1405_3521_gb300 as h
    h._capi.lib()
    return h


def _static_call(hjb, p, out):
    """hjb_solve_static through the C ABI with the problem's descriptors."""
    from paper_1405_3521_gb300 import _capi
    g, dy, co, di, ct, tg = p._desc
    o = _capi.hjb_solve_opts()
    o.tol, o.max_iters, o.use_w_form, o.v_init, o.sweeps_per_check = 0.0, 0, -1, None, 0
    st = _capi.hjb_stats()
    import torch
    rc = _capi.lib().hjb_solve_static(C.byref(g), C.byref(dy), C.byref(co), C.byref(di),
                                      C.byref(ct), C.byref(tg), C.byref(o), out.data_ptr(),
                                      C.byref(st), torch.cuda.current_stream().cuda_stream)
    return rc, st


def test_static_solve_matches_solve_twice(hjb):
    import torch
    d1 = S.c2(n=257, A=64, ntargets=6)
    d2 = S.c1(n=101)
    for d in (d1, d2, d1):  # consecutive calls share the static array
        p = gpu_problem(hjb, d)
        ref, _ = hjb.solve(p)
        out = torch.full((p.N,), float("nan"), device="cuda")
        rc, st = _static_call(hjb, p, out)
        assert rc == 0, hjb._capi.lib().hjb_last_error()
        assert st.converged in (1, 2)
        assert np.abs(to_np(out) - to_np(ref)).max() < 1e-4


def test_static_solve_rejects_what_it_cannot_hold(hjb):
    import torch
    from paper_1405_3521_gb300 import _capi
    d = S.c2(n=1025, A=16, ntargets=4)  # over the node limit
    p = gpu_problem(hjb, d)
    out = torch.empty(p.N, device="cuda")
    rc, _ = _static_call(hjb, p, out)
    assert rc == _capi.HJB_ERR_INVALID_ARG
    assert b"maximum" in _capi.lib().hjb_last_error()
    ph = gpu_problem(hjb, S.c1(n=41), host=True)  # host arrays would need staging
    rc, _ = _static_call(hjb, ph, torch.empty(ph.N, device="cuda"))
    assert rc == _capi.HJB_ERR_INVALID_ARG
