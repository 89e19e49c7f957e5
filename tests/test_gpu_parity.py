"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Tolerance: 1e-4 in L-infinity on V (the Kruzhkov
value); labels bit-exact except decisions within 1e-6 of the threshold;
gradients 1e-3 relative."""
import numpy as np
import pytest

import synthetic as S
from _cases import gpu_problem, oracle_problem, projection_reads, to_np

pytestmark = pytest.mark.gpu

TOL_V = 1e-4


@pytest.fixture(scope="module")
def hjb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1405_3521_gb300 as h
    h._capi.lib()  # fails loudly when the library is missing
    return h


def _ref(orc, d, tol=1e-12, **kw):
    p = oracle_problem(orc, d)
    V, it, r = orc.solve(p, tol=tol, nthreads=8, **kw)
    return p, V


@pytest.mark.parametrize("wform", [1, 0])
def test_c1_full_solve(hjb, orc, wform):
    d = S.c1()
    _, Vo = _ref(orc, d, tol=1e-10)
    p = gpu_problem(hjb, d)
    V, st = hjb.solve(p, use_w_form=wform)
    err = np.abs(to_np(V) - Vo).max()
    assert st["converged"] == 1
    assert err < TOL_V, err
    # quiescent tiles are skipped (exactly), so at most every free node per
    # application, with 6 applications per staged tile and sweep by default
    nfree = int((d["labels"] == 0).sum())
    assert 0 < st["node_updates"] <= st["iterations"] * nfree * 6


@pytest.mark.parametrize("nx,ny,A,cur", [(67, 45, 16, True), (33, 97, 7, False),
                                          (130, 9, 32, True), (257, 129, 64, True)])
def test_ragged_speed_current(hjb, orc, nx, ny, A, cur):
    """Grids that are not multiples of the 32 x 8 tile, generic and
    specialised control counts, speed and current fields."""
    X, Y = S.mesh2(nx, ny)
    g = S.rng("misc", nx * 1000 + ny)
    cen = S.disk_centers(g, 3, 0.12)
    lab = S.disk_labels(X, Y, cen, 0.12)
    d = dict(shape=(nx, ny), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
             controls=S.f32(S.circle_controls(A)), labels=lab, ntargets=3,
             speed=S.f32(S.speed_field(g, X, Y)),
             current=S.f32(S.current_field(g, X, Y)) if cur else None,
             h=min(2.0 / (nx - 1), 2.0 / (ny - 1)), lam=1.0, v_out=1.0)
    _, Vo = _ref(orc, d, tol=1e-11)
    p = gpu_problem(hjb, d)
    V, st = hjb.solve(p)
    assert np.abs(to_np(V) - Vo).max() < TOL_V


def test_halo4_long_steps(hjb, orc):
    """Feet travelling 2-4 cells per step select the wider-halo kernel."""
    n = 61
    X, Y = S.mesh2(n, n)
    g = S.rng("misc", 77)
    lab = S.disk_labels(X, Y, S.disk_centers(g, 2, 0.15), 0.15)
    d = dict(shape=(n, n), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
             controls=S.f32(S.circle_controls(32)), labels=lab, ntargets=2,
             speed=S.f32(S.speed_field(g, X, Y)), current=None, h=2.3 * 2.0 / (n - 1), lam=1.0,
             v_out=1.0)
    _, Vo = _ref(orc, d, tol=1e-11)
    V, st = hjb.solve(gpu_problem(hjb, d))
    assert np.abs(to_np(V) - Vo).max() < TOL_V


def test_cost_field_vform(hjb, orc):
    """A running-cost field forces the V (min) form; lambda != 1."""
    n = 73
    X, Y = S.mesh2(n, n)
    g = S.rng("misc", 5)
    lab = S.disk_labels(X, Y, S.disk_centers(g, 2, 0.1), 0.1)
    cost = S.f32(0.5 + X * X + Y * Y)
    d = dict(shape=(n, n), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
             controls=S.f32(S.circle_controls(32)), labels=lab, ntargets=2, speed=None,
             current=None, cost=cost, h=2.0 / (n - 1), lam=0.7, v_out=2.5 / 0.7)
    _, Vo = _ref(orc, d, tol=1e-11)
    V, st = hjb.solve(gpu_problem(hjb, d))
    assert np.abs(to_np(V) - Vo).max() < TOL_V


def test_host_buffers_match_device(hjb, orc):
    d = S.c2(n=129, ntargets=5)
    pd = gpu_problem(hjb, d)
    ph = gpu_problem(hjb, d, host=True)
    Vd, _ = hjb.solve(pd)
    Vh, _ = hjb.solve(ph)
    assert isinstance(Vh, np.ndarray)
    assert np.array_equal(to_np(Vd), Vh)


def test_warm_start_and_degenerate(hjb, orc):
    d = S.c1(n=41)
    p = gpu_problem(hjb, d)
    V, st = hjb.solve(p)
    V2, st2 = hjb.solve(p, v_init=V)
    assert st2["iterations"] <= 2
    assert np.abs(to_np(V2) - to_np(V)).max() < 1e-6
    # no target node at all: every node keeps the "never arrives" value
    d0 = dict(d)
    d0["labels"] = np.zeros_like(d["labels"])
    V0, st0 = hjb.solve(gpu_problem(hjb, d0))
    assert np.abs(to_np(V0) - 1.0).max() < 1e-6
    # every node a target: nothing to iterate
    d1 = dict(d)
    d1["labels"] = np.ones_like(d["labels"])
    d1["ntargets"] = 1
    V1, st1 = hjb.solve(gpu_problem(hjb, d1))
    assert np.abs(to_np(V1)).max() == 0.0 and st1["node_updates"] == 0
    # smallest grid: 2 x 2
    d2 = dict(shape=(2, 2), lo=(0.0, 0.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
              controls=S.f32(S.axis_controls()), labels=np.array([[1, 0], [0, 0]], np.uint8),
              ntargets=1, speed=None, current=None, h=1.0, lam=1.0, v_out=1.0)
    _, Vo = _ref(orc, d2)
    V2, _ = hjb.solve(gpu_problem(hjb, d2))
    assert np.abs(to_np(V2) - Vo).max() < 1e-6


def test_not_converged_reports(hjb):
    d = S.c1(n=61)
    p = gpu_problem(hjb, d)
    with pytest.raises(hjb.NotConverged):
        hjb.solve(p, max_iters=3)
    V, st = hjb.solve(p, max_iters=3, allow_not_converged=True)
    assert st["iterations"] == 3 and st["converged"] == 0


def test_dubins_3d(hjb, orc):
    d = S.c3(nxy=41, nth=16, ntargets=3, stride=(5, 5, 4))
    _, Vo = _ref(orc, d, tol=1e-11)
    V, st = hjb.solve(gpu_problem(hjb, d))
    assert np.abs(to_np(V) - Vo).max() < TOL_V


def test_ra_labels_and_projection(hjb, orc):
    """RA on the coarse grid (Sec. 3) and the projection (Sec. 4): coarse
    labels bit-exact except near-threshold decisions; the fine mask is the
    projection of the coarse labels (integer, exact)."""
    d = S.c2(n=129, ntargets=6, stride=8)
    po = oracle_problem(orc, d)
    stride = (8, 8)
    delta = 0.12
    Vaux_o, lab_o, _ = orc.ra(po, stride, delta, tol=1e-11)
    p = gpu_problem(hjb, d)
    fine, coarse, aux, st = hjb.subdomains(p, stride, delta=delta, want_aux=True)
    coarse = to_np(coarse).astype(np.uint32)
    fine = to_np(fine).astype(np.uint32)
    aux = to_np(aux).reshape(Vaux_o.shape)
    assert np.abs(aux - Vaux_o).max() < TOL_V
    vmin = Vaux_o.min(0)
    diff = coarse ^ lab_o
    near = np.zeros_like(diff, dtype=bool)
    for k in range(d["ntargets"]):
        close = np.abs(np.abs(Vaux_o[k] - vmin) - delta) <= TOL_V
        near |= close & (((diff >> k) & 1) == 1)
    bad = (diff != 0) & ~near
    assert bad.sum() == 0
    # the projection agrees bit for bit wherever it reads only coarse labels
    # both sides agree on (everywhere when they all agree)
    reads = projection_reads(orc.coarse_shape(po, stride), stride[0], diff != 0, d["shape"])
    fine_o = orc.project(po, stride, lab_o)
    assert np.array_equal(fine[~reads], fine_o[~reads])
    assert st["labelled"] == sum(int(((fine >> k) & 1).sum()) for k in range(6))


def _ra_case(which):
    """Workloads for the two RA paths: bands of the on-chip coarse solve of
    several heights (8 bands of 2-3 rows; 5 bands of 2 rows; halo 4 with long
    steps), a V-form cost field with a drift, a ragged coarse grid."""
    if which == "c2":
        return S.c2(n=257, ntargets=8, stride=16), (16, 16), 0.12, {}
    if which == "c1":
        return S.c1(n=41), (4, 4), 0.2, {}
    if which == "vdp":
        return S.vdp(n=97, slices=4, stride=8), (8, 8), 0.1, {}
    if which == "halo4":
        n = 97
        X, Y = S.mesh2(n, n)
        g = S.rng("misc", 78)
        lab = S.disk_labels(X, Y, S.disk_centers(g, 3, 0.15), 0.15)
        d = dict(shape=(n, n), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
                 controls=S.f32(S.circle_controls(32)), labels=lab, ntargets=3,
                 speed=S.f32(S.speed_field(g, X, Y)), current=None, h=2.3 * 2.0 / (n - 1),
                 lam=1.0, v_out=1.0)
        return d, (4, 4), 0.15, {}
    nx, ny = 161, 73  # ragged: coarse 21 x 10
    X, Y = S.mesh2(nx, ny)
    g = S.rng("misc", 79)
    lab = S.disk_labels(X, Y, S.disk_centers(g, 4, 0.12), 0.12)
    d = dict(shape=(nx, ny), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
             controls=S.f32(S.circle_controls(16)), labels=lab, ntargets=4,
             speed=S.f32(S.speed_field(g, X, Y)), current=S.f32(S.current_field(g, X, Y)),
             h=2.0 / (nx - 1), lam=1.0, v_out=1.0)
    return d, (8, 8), 0.12, {}


@pytest.mark.parametrize("path", ["on_chip", "tiles"])
@pytest.mark.parametrize("which", ["c2", "c1", "vdp", "halo4", "ragged"])
def test_ra_paths_against_oracle(hjb, orc, monkeypatch, path, which):
    """RA step 1 (Sec. 3) by the on-chip cluster solve (HJB_RA=chip) and by
    the tile-queue sweep (HJB_RA=tiles), the two paths the tuner chooses
    between for 2D coarse grids: the auxiliary solutions against the
    oracle's at 1e-4, the labels bit for bit except near-threshold
    decisions."""
    monkeypatch.setenv("HJB_RA", "tiles" if path == "tiles" else "chip")
    d, stride, delta, _ = _ra_case(which)
    po = oracle_problem(orc, d)
    Vaux_o, lab_o, _ = orc.ra(po, stride, delta, tol=1e-11, nthreads=8)
    p = gpu_problem(hjb, d)
    fine, coarse, aux, st = hjb.subdomains(p, stride, delta=delta, want_aux=True)
    assert st["converged"] == 1
    assert np.abs(to_np(aux).reshape(Vaux_o.shape) - Vaux_o).max() < TOL_V
    diff = to_np(coarse).astype(np.uint32) ^ lab_o
    vmin = Vaux_o.min(0)
    for k in range(d["ntargets"]):
        bad = ((diff >> k) & 1) == 1
        assert np.all(np.abs(np.abs(Vaux_o[k][bad] - vmin[bad]) - delta) <= TOL_V)
    # the on-chip solve is one application per iteration; the tile sweep
    # applies T several times per staged tile
    assert (st["local_iters"] == 1) == (path == "on_chip")


@pytest.mark.parametrize("which", ["c1", "c2"])
def test_decomposed_matches_oracle_isa(hjb, orc, which):
    if which == "c1":
        d = S.c1(n=81)
        stride = (4, 4)
    else:
        d = S.c2(n=129, ntargets=6, stride=8)
        stride = (8, 8)
    po = oracle_problem(orc, d)
    _, lab_o, _ = orc.ra(po, stride, 0.15, tol=1e-11)
    fine = orc.project(po, stride, lab_o)
    Vbar_o, unc, _, _ = orc.isa(po, fine, tol=1e-11, nthreads=8)
    p = gpu_problem(hjb, d)
    import torch
    fm = torch.as_tensor(fine.astype(np.int32)).cuda()
    Vbar, per, tot = hjb.solve_decomposed(p, fm)
    assert np.abs(to_np(Vbar) - Vbar_o).max() < TOL_V
    assert tot["converged"] == 1
    # host mask path
    Vbar_h, _, _ = hjb.solve_decomposed(p, fine)
    assert np.array_equal(to_np(Vbar_h), to_np(Vbar))


def test_decomposed_equal_subdomains_solved_once(hjb, orc):
    """Sub-domains with equal node sets share one solve (their V_k is the same
    function of the node set); Vbar still matches the oracle's ISA, which
    solves every copy."""
    d = S.c1(n=81)
    stride = (4, 4)
    po = oracle_problem(orc, d)
    _, lab_o, _ = orc.ra(po, stride, 0.15, tol=1e-11)
    fine = orc.project(po, stride, lab_o).astype(np.uint32)
    b0 = fine & np.uint32(1)
    fine = (fine & ~np.uint32(0b1100)) | (b0 << np.uint32(2)) | (b0 << np.uint32(3))
    Vbar_o, _, its_o, _ = orc.isa(po, fine, tol=1e-11, nthreads=8)
    p = gpu_problem(hjb, d)
    Vbar, per, tot = hjb.solve_decomposed(p, fine)
    assert np.abs(to_np(Vbar) - Vbar_o).max() < TOL_V
    assert tot["converged"] == 1
    assert per[2]["node_updates"] == 0 and per[3]["node_updates"] == 0
    assert per[2]["iterations"] == per[0]["iterations"] == per[3]["iterations"]
    assert per[0]["node_updates"] > 0 and per[1]["node_updates"] > 0
    assert all(s["converged"] == 1 for s in per)


def test_dubins_whole_domain_subdomains(hjb, orc):
    """3D Dubins with every node in every sub-domain (the safe threshold of a
    discontinuous value function): one solve, equal to the full solve."""
    d = S.c3(nxy=40, nth=16, stride=(3, 3, 4))
    po = oracle_problem(orc, d)
    Vo, _, _ = orc.solve(po, tol=1e-11, nthreads=8)
    p = gpu_problem(hjb, d)
    fine, _, _, rst = hjb.subdomains(p, d["stride"], delta=4.0)
    assert rst["labelled"] == d["ntargets"] * d["labels"].size
    Vbar, per, tot = hjb.solve_decomposed(p, fine)
    assert np.abs(to_np(Vbar) - Vo).max() < TOL_V
    assert sum(s["node_updates"] > 0 for s in per) == 1
    V, st = hjb.solve(p)
    # the two calls may run differently tuned tiles (shape, applications per
    # tile), whose FP32 roundings differ within the stopping tolerance
    assert np.abs(to_np(V) - to_np(Vbar)).max() < 1e-5


def test_batch_uneven(hjb, orc):
    sides = [64, 97, 130, 71]
    ds = [S.c4_problem(i, n) for i, n in enumerate(sides)]
    ps = [gpu_problem(hjb, d) for d in ds]
    Vs, sts = hjb.solve_batch(ps)
    for d, V, st in zip(ds, Vs, sts):
        _, Vo = _ref(orc, d, tol=1e-11)
        assert np.abs(to_np(V) - Vo).max() < TOL_V
        assert st["converged"] == 1
    # batch result equals the single solves
    V0, _ = hjb.solve(ps[1])
    assert np.abs(to_np(V0) - to_np(Vs[1])).max() < 1e-6


def test_point_values(hjb, orc):
    d = S.c1(n=51)
    po, Vo = _ref(orc, d)
    p = gpu_problem(hjb, d)
    import torch
    g = np.random.default_rng(3)
    pts = S.f32(g.uniform(-1, 1, size=(300, 2)))
    vals_o, gr_o = orc.points(po, Vo, pts)
    vals, gr = hjb.point_values(p, torch.as_tensor(Vo.astype(np.float32)).cuda(),
                                torch.as_tensor(pts.astype(np.float32)).cuda())
    assert np.abs(to_np(vals) - vals_o).max() < 1e-5
    assert np.abs(to_np(gr) - gr_o).max() < 1e-6


def test_adjoint_gradient(hjb, orc):
    """hjb_backward against the FP64 adjoint of the oracle (1e-3 relative),
    with both solves from the same seeded inputs."""
    n, A = 65, 16
    d = S.c5(n=n, A=A, ntargets=3, P=256)
    po = oracle_problem(orc, d)
    Vo, _, _ = orc.solve(po, tol=1e-14, nthreads=8)
    pol, _ = orc.policy(po, Vo)
    vals, gV = orc.points(po, Vo, d["points"])
    lam, _, _ = orc.adjoint(po, pol, gV, tol=1e-14)
    gt_o, gc_o = orc.grad(po, Vo, pol, lam)
    import torch
    p = gpu_problem(hjb, d)
    V, _ = hjb.solve(p)
    pts = torch.as_tensor(d["points"].astype(np.float32)).cuda()
    _, gV_gpu = hjb.point_values(p, V, pts)
    gt, st = hjb.backward(p, V, gV_gpu, wrt=0, tol=1e-9)
    gc, _ = hjb.backward(p, V, gV_gpu, wrt=1, tol=1e-9)
    rel_t = np.abs(to_np(gt) - gt_o).max() / np.abs(gt_o).max()
    rel_c = np.abs(to_np(gc) - gc_o).max() / np.abs(gc_o).max()
    assert rel_c < 1e-3, rel_c
    assert rel_t < 1e-3, rel_t


def test_adjoint_policy_refinement(hjb, orc, monkeypatch):
    """The backward decides the optimal policy in FP64 on values refined from
    the FP32 solution (the FP64 residual of the policy-frozen system, an FP32
    correction).  With a current and a running-cost field, both of which
    enter that residual, the gradients match the oracle's FP64 adjoint within
    1e-3 relative, no worse (beyond the FP32 accumulation noise) than without
    the refinement (HJB_ADJ_REFINE=0), and the statistics show the
    refinement's iterations."""
    import torch
    n, A = 129, 32
    d = S.c5(n=n, A=A, ntargets=3, P=512)
    X, Y = S.mesh2(n, n)
    g = S.rng("misc", 41)
    d["current"] = S.f32(0.5 * S.current_field(g, X, Y))
    d["cost"] = S.f32(S.speed_field(g, X, Y))
    po = oracle_problem(orc, d)
    Vo, _, _ = orc.solve(po, tol=1e-14, nthreads=orc.max_threads())
    pol, _ = orc.policy(po, Vo)
    _, gV = orc.points(po, Vo, d["points"])
    lam, _, _ = orc.adjoint(po, pol, gV, tol=1e-14)
    gt_o, gc_o = orc.grad(po, Vo, pol, lam)
    p = gpu_problem(hjb, d)
    V, _ = hjb.solve(p)
    pts = torch.as_tensor(d["points"].astype(np.float32)).cuda()
    _, gV_gpu = hjb.point_values(p, V, pts)
    errs = {}
    for refine in ("1", "0"):
        monkeypatch.setenv("HJB_ADJ_REFINE", refine)
        gt, st = hjb.backward(p, V, gV_gpu, wrt=0)
        gc, _ = hjb.backward(p, V, gV_gpu, wrt=1)
        assert (st["local_iters"] > 0) == (refine == "1"), st
        errs[refine] = (np.abs(to_np(gt) - gt_o).max() / np.abs(gt_o).max(),
                        np.abs(to_np(gc) - gc_o).max() / np.abs(gc_o).max())
    assert errs["1"][0] < 1e-3 and errs["1"][1] < 1e-3, errs
    assert errs["1"][0] <= errs["0"][0] + 1e-4 and errs["1"][1] <= errs["0"][1] + 1e-4, errs


def test_autograd_function(hjb, orc):
    import torch
    n, A = 49, 16
    d = S.c5(n=n, A=A, ntargets=2, P=128)
    spec = dict(shape=d["shape"], lo=d["lo"], hi=d["hi"], controls=d["controls"],
                labels=torch.as_tensor(d["labels"]).cuda(), h=d["h"], n_targets=2)
    theta = torch.as_tensor(d["log_speed"].astype(np.float32)).cuda().requires_grad_(True)
    v = hjb.HJBSolve.apply(theta, spec)
    prob = hjb.Problem(log_speed=theta.detach(), **spec)
    loss = hjb.point_loss(v, prob, torch.as_tensor(d["points"].astype(np.float32)).cuda())
    loss.backward()
    po = oracle_problem(orc, d)
    Vo, _, _ = orc.solve(po, tol=1e-14)
    pol, _ = orc.policy(po, Vo)
    _, gV = orc.points(po, Vo, d["points"])
    lam, _, _ = orc.adjoint(po, pol, gV, tol=1e-14)
    gt_o, _ = orc.grad(po, Vo, pol, lam)
    g = theta.grad.detach().cpu().numpy().reshape(-1)
    assert np.abs(g - gt_o).max() / np.abs(gt_o).max() < 1e-3


def test_tile_shapes_agree_bitwise(hjb, orc, monkeypatch):
    """Every tile shape (32 x 8 / 4 / 2 nodes with 1 / 2 / 4 control groups)
    computes the same Jacobi iteration; tile-local foot coordinates round at
    the last ulp differently per shape, so results agree to FP32 rounding.
    The grid holds more tiles than resident CTAs, so every CTA stages several
    items through both shared-memory buffers."""
    n, A = 577, 16
    X, Y = S.mesh2(n, n)
    g = S.rng("misc", 31)
    lab = S.disk_labels(X, Y, S.disk_centers(g, 5, 0.1), 0.1)
    d = dict(shape=(n, n), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
             controls=S.f32(S.circle_controls(A)), labels=lab, ntargets=5,
             speed=S.f32(S.speed_field(g, X, Y)), current=S.f32(S.current_field(g, X, Y)),
             h=2.0 / (n - 1), lam=1.0, v_out=1.0)
    p = gpu_problem(hjb, d)
    outs = []
    for loop in ("coop", "graph"):
        monkeypatch.setenv("HJB_LOOP", loop)
        for rows in ("8", "4", "2"):
            monkeypatch.setenv("HJB_TILE_ROWS", rows)
            V, st = hjb.solve(p, local_iters=1)
            outs.append(to_np(V))
            fine, _, _, _ = hjb.subdomains(p, (16, 16), delta=0.2)
            Vb, _, _ = hjb.solve_decomposed(p, fine, local_iters=1)
            outs.append(to_np(Vb))
    for k in range(2, len(outs), 2):
        assert np.abs(outs[0] - outs[k]).max() < 1e-5
        assert np.abs(outs[1] - outs[k + 1]).max() < 1e-5
    # the same shape in both loop modes runs the identical iteration
    assert np.array_equal(outs[0], outs[6]) and np.array_equal(outs[1], outs[7])
    # and against the oracle's own fixed point at this size
    po = oracle_problem(orc, d)
    Vo, _, _ = orc.solve(po, tol=1e-11, nthreads=orc.max_threads())
    assert np.abs(outs[0] - Vo).max() < TOL_V


@pytest.mark.parametrize("A", [32, 64])
def test_lane_split_agrees_bitwise(hjb, monkeypatch, A):
    """The lane split of 32 x 4 tiles (lanes n and n + 16 of a warp take a_j
    and -a_j of node n) evaluates the same foot products as the two control
    groups (a_{j + A/2} = -a_j exactly, and negation is exact), and the
    extremum does not depend on the order: V, the sweep counts and the
    node-update counts are identical, with one and with six applications
    per staged tile, for the full and the decomposed solve."""
    n = 577
    X, Y = S.mesh2(n, n)
    g = S.rng("misc", 37)
    lab = S.disk_labels(X, Y, S.disk_centers(g, 5, 0.1), 0.1)
    ctrl = S.f32(S.circle_controls(A))
    assert np.array_equal(ctrl[A // 2:], -ctrl[:A // 2])
    d = dict(shape=(n, n), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
             controls=ctrl, labels=lab, ntargets=5,
             speed=S.f32(S.speed_field(g, X, Y)), current=S.f32(S.current_field(g, X, Y)),
             h=2.0 / (n - 1), lam=1.0, v_out=1.0)
    p = gpu_problem(hjb, d)
    monkeypatch.setenv("HJB_TUNE", "off")
    monkeypatch.setenv("HJB_TILE_ROWS", "4")
    fine, _, _, _ = hjb.subdomains(p, (16, 16), delta=0.2)
    runs = {}
    for lanes in ("1", "2"):
        monkeypatch.setenv("HJB_TILE_LANES", lanes)
        for li in (1, 6):
            V, st = hjb.solve(p, local_iters=li)
            Vb, _, tot = hjb.solve_decomposed(p, fine, local_iters=li)
            assert st["tile_lanes"] == int(lanes) and tot["tile_lanes"] == int(lanes)
            runs[lanes, li] = (to_np(V), st["iterations"], st["node_updates"],
                               to_np(Vb), tot["iterations"], tot["node_updates"])
    for li in (1, 6):
        a, b = runs["1", li], runs["2", li]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[3], b[3])
        assert a[1:3] == b[1:3] and a[4:6] == b[4:6]


@pytest.mark.parametrize("loop", ["graph", "coop"])
def test_queue_schedules_agree_bitwise(hjb, monkeypatch, loop):
    """Static and dynamic sharing of a sweep's tile queue among the CTAs run
    the identical iteration: a tile's new values depend only on the previous
    sweep's values and its own staged tile, so V, the sweep count and the
    node-update count agree bitwise.  2D full, decomposed and batched solves
    with four applications per tile (more tiles than resident CTAs, items of
    unequal cost), and the 3D Dubins solve."""
    monkeypatch.setenv("HJB_LOOP", loop)
    n, A = 577, 16
    X, Y = S.mesh2(n, n)
    g = S.rng("misc", 31)
    lab = S.disk_labels(X, Y, S.disk_centers(g, 5, 0.1), 0.1)
    d = dict(shape=(n, n), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
             controls=S.f32(S.circle_controls(A)), labels=lab, ntargets=5,
             speed=S.f32(S.speed_field(g, X, Y)), current=S.f32(S.current_field(g, X, Y)),
             h=2.0 / (n - 1), lam=1.0, v_out=1.0)
    p = gpu_problem(hjb, d)
    batch = [gpu_problem(hjb, S.c4_problem(i, m)) for i, m in ((0, 200), (1, 333), (2, 150))]
    p3 = gpu_problem(hjb, S.c3(nxy=64, nth=32, ntargets=3, stride=(3, 3, 4)))
    runs = {}
    for mode in ("static", "dynamic"):
        monkeypatch.setenv("HJB_QUEUE", mode)
        out = []
        V, st = hjb.solve(p, local_iters=4)
        out.append((to_np(V), st["iterations"], st["node_updates"]))
        fine, _, _, _ = hjb.subdomains(p, (16, 16), delta=0.2)
        Vb, _, tot = hjb.solve_decomposed(p, fine, local_iters=4)
        out.append((to_np(Vb), tot["iterations"], tot["node_updates"]))
        Vs, sts = hjb.solve_batch(batch, local_iters=4)
        out += [(to_np(v), s["iterations"], s["node_updates"]) for v, s in zip(Vs, sts)]
        V3, st3 = hjb.solve(p3)
        out.append((to_np(V3), st3["iterations"], st3["node_updates"]))
        runs[mode] = out
    for (va, ia, ua), (vb, ib, ub) in zip(runs["static"], runs["dynamic"]):
        assert np.array_equal(va, vb)
        assert (ia, ua) == (ib, ub)


def test_decomposed_own_targets_against_oracle(hjb, orc):
    """ISA with sub-problems that keep only their own target component (the
    target choice of RA step 1, Sec. 3, as the alternative reading of Sec. 4
    step 3): the GPU decomposed solve on the oracle's own decomposition
    against the oracle's ISA with the same choice, node by node.  At this
    threshold sub-domains reach into other components, where the two
    readings differ by more than the tolerance."""
    d = S.c2(n=129, A=16, ntargets=4, stride=4)
    nt = orc.max_threads()
    po = oracle_problem(orc, d)
    _, lab_o, _ = orc.ra(po, (4, 4), 0.5, tol=1e-11, nthreads=nt)
    fine = orc.project(po, (4, 4), lab_o)
    lab = np.asarray(d["labels"]).reshape(-1)
    assert sum(int(np.sum(((fine >> k) & 1)[(lab != 0) & (lab != k + 1)])) for k in range(4)) > 0
    Vo, unc, _, _ = orc.isa(po, fine, tol=1e-11, nthreads=nt, own_targets=True)
    Vr, _, _, _ = orc.isa(po, fine, tol=1e-11, nthreads=nt)
    assert unc == 0 and np.abs(Vo - Vr).max() > 10 * TOL_V
    p = gpu_problem(hjb, d)
    Vb, per, tot = hjb.solve_decomposed(p, fine, subdomain_targets=hjb.HJB_SUBDOMAIN_TARGETS_OWN)
    assert tot["converged"] == 1
    assert np.abs(to_np(Vb).astype(np.float64) - Vo).max() < TOL_V
    Vb3, _, _ = hjb.solve_decomposed(p, fine)
    assert np.abs(to_np(Vb3).astype(np.float64) - Vr).max() < TOL_V


def test_local_iterations_same_fixed_point(hjb, orc):
    """Several applications of T per staged tile (the halo held) reach the
    fixed point of plain value iteration in fewer sweeps: each GPU result is
    within 1e-4 of the oracle's fixed point, for the full-domain, decomposed
    and batched solves."""
    n, A = 321, 32
    X, Y = S.mesh2(n, n)
    g = S.rng("misc", 32)
    lab = S.disk_labels(X, Y, S.disk_centers(g, 4, 0.1), 0.1)
    d = dict(shape=(n, n), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
             controls=S.f32(S.circle_controls(A)), labels=lab, ntargets=4,
             speed=S.f32(S.speed_field(g, X, Y)), current=S.f32(S.current_field(g, X, Y)),
             h=2.0 / (n - 1), lam=1.0, v_out=1.0)
    p = gpu_problem(hjb, d)
    p2 = gpu_problem(hjb, d)
    po = oracle_problem(orc, d)
    _, lab_o, _ = orc.ra(po, (16, 16), 0.2, tol=1e-11, nthreads=8)
    fine = orc.project(po, (16, 16), lab_o)
    Vb_o, _, _, _ = orc.isa(po, fine, tol=1e-11, nthreads=8)
    Vo, _, _ = orc.solve(po, tol=1e-11, nthreads=8)
    sweeps = {}
    for L in (1, 2, 4, 16):
        V, st = hjb.solve(p, local_iters=L)
        assert st["converged"] == 1
        sweeps[L] = st["iterations"]
        assert np.abs(to_np(V) - Vo).max() < TOL_V
        Vb, per, tot = hjb.solve_decomposed(p, fine, local_iters=L)
        assert tot["converged"] == 1
        assert np.abs(to_np(Vb) - Vb_o).max() < TOL_V
        Vs, sts = hjb.solve_batch([p, p2], local_iters=L)
        assert np.abs(to_np(Vs[0]) - to_np(V)).max() < 1e-6
    assert sweeps[4] < sweeps[2] < sweeps[1]


def test_dubins_local_iterations(hjb, orc):
    """The 3D kernel's repeated applications per staged tile reach the same
    fixed point (periodic heading, halo layers held)."""
    d = S.c3(nxy=41, nth=16, ntargets=3, stride=(5, 5, 4))
    _, Vo = _ref(orc, d, tol=1e-11)
    p = gpu_problem(hjb, d)
    sweeps = {}
    for L in (1, 4, 16):
        V, st = hjb.solve(p, local_iters=L)
        assert st["converged"] == 1
        sweeps[L] = st["iterations"]
        assert np.abs(to_np(V) - Vo).max() < TOL_V
    assert sweeps[4] < sweeps[1]


def test_vdp_full_and_decomposed(hjb, orc):
    """Van der Pol (Sec. 5, Example ex3): drift as a node field, running cost
    |x| (V form), target disk in 4 cake slices; full solve, RA labels and the
    decomposed solve against the oracle."""
    d = S.vdp(n=129, slices=4)
    po = oracle_problem(orc, d)
    Vo, _, _ = orc.solve(po, tol=1e-11, nthreads=8)
    p = gpu_problem(hjb, d)
    V, st = hjb.solve(p)
    assert st["converged"] == 1
    assert np.abs(to_np(V) - Vo).max() < TOL_V
    stride, delta = d["stride"], 0.1
    Vaux_o, lab_o, _ = orc.ra(po, stride, delta, tol=1e-11, nthreads=8)
    fine_o = orc.project(po, stride, lab_o)
    fine, coarse, aux, _ = hjb.subdomains(p, stride, delta=delta, want_aux=True)
    assert np.abs(to_np(aux).reshape(Vaux_o.shape) - Vaux_o).max() < TOL_V
    diff = to_np(coarse).astype(np.uint32) ^ lab_o
    vmin = Vaux_o.min(0)
    for k in range(d["ntargets"]):
        bad = ((diff >> k) & 1) == 1
        assert np.all(np.abs(np.abs(Vaux_o[k][bad] - vmin[bad]) - delta) <= TOL_V)
    Vb_o, unc, _, _ = orc.isa(po, fine_o, tol=1e-11, nthreads=8)
    Vb, per, tot = hjb.solve_decomposed(p, fine_o)
    assert tot["converged"] == 1
    assert np.abs(to_np(Vb) - Vb_o).max() < TOL_V


def test_game_silent_second_player(hjb, orc):
    """A second player whose only control is b = 0 leaves the control
    problem unchanged (the game kernel path against the plain one)."""
    d = S.c2(n=97, A=16, ntargets=3, stride=8)
    p = gpu_problem(hjb, d)
    V, _ = hjb.solve(p, local_iters=1)
    g = dict(d)
    g["controls_b"] = np.zeros((1, 2), np.float32)
    Vg, st = hjb.solve(gpu_problem(hjb, g), local_iters=1)
    assert st["converged"] == 1
    assert np.abs(to_np(Vg) - to_np(V)).max() < 1e-6


def test_pursuit_evasion_game(hjb, orc):
    """The pursuit-evasion game (Sec. 5, Example ex4): per-axis scale field,
    the max over the evader's b of the min over the pursuer's a, running cost
    field; full solve, RA labels and the decomposed solve against the
    oracle."""
    d = S.pursuit_evasion(n=129, slices=4)
    po = oracle_problem(orc, d)
    Vo, _, _ = orc.solve(po, tol=1e-11, nthreads=8)
    p = gpu_problem(hjb, d)
    V, st = hjb.solve(p)
    assert st["converged"] == 1
    assert np.abs(to_np(V) - Vo).max() < TOL_V
    stride, delta = d["stride"], 0.1
    Vaux_o, lab_o, _ = orc.ra(po, stride, delta, tol=1e-11, nthreads=8)
    fine_o = orc.project(po, stride, lab_o)
    fine, coarse, aux, _ = hjb.subdomains(p, stride, delta=delta, want_aux=True)
    assert np.abs(to_np(aux).reshape(Vaux_o.shape) - Vaux_o).max() < TOL_V
    diff = to_np(coarse).astype(np.uint32) ^ lab_o
    vmin = Vaux_o.min(0)
    for k in range(d["ntargets"]):
        bad = ((diff >> k) & 1) == 1
        assert np.all(np.abs(np.abs(Vaux_o[k][bad] - vmin[bad]) - delta) <= TOL_V)
    Vb_o, _, _, _ = orc.isa(po, fine_o, tol=1e-11, nthreads=8)
    Vb, per, tot = hjb.solve_decomposed(p, fine_o)
    assert tot["converged"] == 1
    assert np.abs(to_np(Vb) - Vb_o).max() < TOL_V


@pytest.mark.parametrize("which", ["c1", "vdp"])
def test_implicit_step_weights(hjb, orc, which):
    """The 1/(1 + lambda h) weights of the printed scheme (Sec. 3), W form
    (constant cost) and V form (cost field), full and decomposed solves."""
    d = S.c1(n=81) if which == "c1" else S.vdp(n=97, slices=4)
    d = dict(d, weights=1)
    po = oracle_problem(orc, d)
    Vo, _, _ = orc.solve(po, tol=1e-11, nthreads=8)
    p = gpu_problem(hjb, d)
    V, st = hjb.solve(p)
    assert st["converged"] == 1
    assert np.abs(to_np(V) - Vo).max() < TOL_V
    q = gpu_problem(hjb, dict(d, weights=0))
    assert np.abs(to_np(hjb.solve(q)[0]) - Vo).max() > 10 * TOL_V
    stride = (4, 4) if which == "c1" else d["stride"]
    _, lab_o, _ = orc.ra(po, stride, 0.15, tol=1e-11)
    fine = orc.project(po, stride, lab_o)
    Vb_o, _, _, _ = orc.isa(po, fine, tol=1e-11, nthreads=8)
    Vb, _, tot = hjb.solve_decomposed(p, fine)
    assert np.abs(to_np(Vb) - Vb_o).max() < TOL_V


@pytest.mark.parametrize("which", ["c1", "c2"])
def test_p1_interpolation(hjb, orc, which):
    """P1 interpolation on the Kuhn triangles (Sec. 3): W form (c1) and a
    speed/current problem (c2, 61 controls: the generic-count kernel), full
    and decomposed solves against the oracle; P1 and Q1 results differ."""
    d = S.c1(n=81) if which == "c1" else S.c2(n=129, A=61, ntargets=5, stride=8)
    d = dict(d, interp=1)
    po = oracle_problem(orc, d)
    Vo, _, _ = orc.solve(po, tol=1e-11, nthreads=8)
    p = gpu_problem(hjb, d)
    V, st = hjb.solve(p)
    assert st["converged"] == 1
    assert np.abs(to_np(V) - Vo).max() < TOL_V
    q = gpu_problem(hjb, dict(d, interp=0))
    assert np.abs(to_np(hjb.solve(q)[0]) - Vo).max() > 10 * TOL_V
    stride = (4, 4) if which == "c1" else d["stride"]
    _, lab_o, _ = orc.ra(po, stride, 0.15, tol=1e-11)
    fine = orc.project(po, stride, lab_o)
    Vb_o, _, _, _ = orc.isa(po, fine, tol=1e-11, nthreads=8)
    Vb, _, tot = hjb.solve_decomposed(p, fine)
    assert tot["converged"] == 1
    assert np.abs(to_np(Vb) - Vb_o).max() < TOL_V


def test_decomposed_with_32_targets(hjb, orc):
    """The largest label set (32 target components, bit 31 of the masks):
    RA labels, the decomposed solve against the oracle's ISA, and equal
    sub-domains (two components given the same node set) solved once."""
    n = 129
    X, Y = S.mesh2(n, n)
    lab = np.zeros((n, n), np.uint8)
    k = 0
    for cy in np.linspace(-0.8, 0.8, 6):
        for cx in np.linspace(-0.8, 0.8, 6):
            if k == 32:
                break
            lab[np.hypot(X - cx, Y - cy) <= 0.07] = k + 1
            k += 1
    g = S.rng("misc", 33)
    d = dict(shape=(n, n), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
             controls=S.f32(S.circle_controls(16)), labels=lab, ntargets=32,
             speed=S.f32(S.speed_field(g, X, Y)), current=None, h=2.0 / (n - 1), lam=1.0,
             v_out=1.0)
    po = oracle_problem(orc, d)
    stride, delta = (4, 4), 0.05
    Vaux_o, lab_o, _ = orc.ra(po, stride, delta, tol=1e-11)
    p = gpu_problem(hjb, d)
    fine, coarse, aux, _ = hjb.subdomains(p, stride, delta=delta, want_aux=True)
    assert np.abs(to_np(aux).reshape(Vaux_o.shape) - Vaux_o).max() < TOL_V
    diff = to_np(coarse).astype(np.uint32) ^ lab_o
    vmin = Vaux_o.min(0)
    for b in range(32):
        bad = ((diff >> b) & 1) == 1
        assert np.all(np.abs(np.abs(Vaux_o[b][bad] - vmin[bad]) - delta) <= TOL_V)
    fine_o = orc.project(po, stride, lab_o).astype(np.uint32)
    # components 30 and 31 get the node set of component 0
    b0 = fine_o & np.uint32(1)
    fine_o = (fine_o & ~np.uint32(0xC0000000)) | (b0 << np.uint32(30)) | (b0 << np.uint32(31))
    Vb_o, _, _, _ = orc.isa(po, fine_o, tol=1e-11, nthreads=8)
    Vb, per, tot = hjb.solve_decomposed(p, fine_o)
    assert tot["converged"] == 1
    assert np.abs(to_np(Vb) - Vb_o).max() < TOL_V
    assert per[30]["node_updates"] == 0 and per[31]["node_updates"] == 0
    assert per[0]["node_updates"] > 0


def _box_split_case():
    n = 41
    lab = np.zeros((n, n), dtype=np.uint8)
    lab[0, :] = 1
    lab[:, n - 1] = 2
    lab[n - 1, :] = 3
    lab[:, 0] = 4
    two = np.where(lab <= 2, np.where(lab > 0, 1, 0), 2).astype(np.uint8)
    d = dict(shape=(n, n), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
             controls=S.f32(S.circle_controls(32)), labels=two, ntargets=2, speed=None,
             current=None, h=2.0 / (n - 1), lam=1.0, v_out=1.0)
    return d, (4, 4)


@pytest.mark.parametrize("which", ["box", "vdp"])
def test_resplitting_against_oracle(hjb, orc, which):
    """Recursive re-splitting of the target components (Conclusions; reading
    R22) on the GPU against the oracle's: the same final division (labels
    bit for bit), the coarse labels of that division (tie-tolerant) and the
    decomposed solve of its sub-domains against the oracle's ISA.  The box
    boundary given as two components reaches the four sides; Van der Pol
    keeps its four slices (splitting a slice does not shrink its
    sub-domain)."""
    import torch
    if which == "box":
        d, stride = _box_split_case()
        splits = 2
    else:
        d = S.vdp(n=97, slices=4, stride=8)
        stride, splits = (8, 8), 4
    po = oracle_problem(orc, d)
    Vaux0, _, _ = orc.ra(po, stride, 0.0, tol=1e-12)
    delta, _ = orc.delta(po, stride, Vaux0)
    comp_o, fine_o, m_o, largest_o = orc.ra_split(po, stride, delta, max_splits=splits,
                                                  tol=1e-12, nthreads=8)
    p = gpu_problem(hjb, d)
    split = torch.zeros(p.N, dtype=torch.uint8, device="cuda")
    fine, coarse, _, st = hjb.subdomains(p, stride, delta=delta, max_splits=splits,
                                         split_labels=split)
    assert st["subdomains"] == m_o
    assert np.array_equal(to_np(split).astype(np.int32), comp_o)
    # the coarse labels of the final division against the oracle's RA on it
    pk = oracle_problem(orc, dict(d, labels=comp_o.reshape(d["labels"].shape), ntargets=m_o))
    Vaux_o, lab_o, _ = orc.ra(pk, stride, delta, tol=1e-12)
    diff = to_np(coarse).astype(np.uint32) ^ lab_o
    vmin = Vaux_o.min(0)
    for k in range(m_o):
        bad = ((diff >> k) & 1) == 1
        assert np.all(np.abs(np.abs(Vaux_o[k][bad] - vmin[bad]) - delta) <= TOL_V)
    reads = projection_reads(orc.coarse_shape(po, stride), stride[0], diff != 0, d["shape"])
    assert np.array_equal(to_np(fine).astype(np.uint32)[~reads], fine_o[~reads])
    # ISA steps 3-4 on the oracle's final division (targets: every target
    # node inside a sub-domain, the same set whatever the division)
    Vb_o, unc, _, _ = orc.isa(pk, fine_o, tol=1e-12, nthreads=8)
    fm = torch.as_tensor(fine_o.astype(np.int32)).cuda()
    Vb, per, tot = hjb.solve_decomposed(p, fm, n_subdomains=m_o)
    assert tot["converged"] == 1
    assert np.abs(to_np(Vb) - Vb_o).max() < TOL_V


def test_coarse_to_fine_warm_start(hjb, orc):
    """The decomposed solve started from the reconstruction's coarse
    auxiliary solutions interpolated onto the fine grid (a warm start
    between ISA steps 2 and 3) reaches the same fixed point: the oracle's
    ISA on the same decomposition within 1e-4."""
    import torch
    d = S.c2(n=129, ntargets=6, stride=8)
    po = oracle_problem(orc, d)
    _, lab_o, _ = orc.ra(po, (8, 8), 0.15, tol=1e-12)
    fine_o = orc.project(po, (8, 8), lab_o)
    Vb_o, _, _, _ = orc.isa(po, fine_o, tol=1e-12, nthreads=8)
    p = gpu_problem(hjb, d)
    hjb.subdomains(p, (8, 8), delta=0.15)  # the coarse auxiliary solutions of the start
    fine = torch.as_tensor(fine_o.astype(np.int32)).cuda()
    Vw, _, totw = hjb.solve_decomposed(p, fine, warm_start=1)
    assert totw["converged"] in (1, 2)
    assert np.abs(to_np(Vw) - Vb_o).max() < TOL_V
    Vc, _, totc = hjb.solve_decomposed(p, fine)
    assert np.abs(to_np(Vc) - Vb_o).max() < TOL_V
