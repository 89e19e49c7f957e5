"""Pins of the FP64 oracle to things other than itself.

Each test checks the oracle against what the paper or the mathematics fixes:
exactness of Q1 interpolation on multilinear functions, brute-force policy
enumeration with exact linear solves, policy iteration (Howard) with sparse
exact solves on 41^2 and Dubins grids, graph shortest paths where every foot
lands on a node, closed-form solutions (distance to disks, constant drift,
the strip of Example 3.1, the box-boundary distance of Sec. 4.1), the
invariants of the iteration and of the reconstruction (Sec. 3), the defining
property of independent sub-domains (a restricted solve reproduces the full
values on policy-closed sets), the concave-hull projection against a direct
enumeration of labelled simplices, Table 1 of the paper, and for the adjoint
gradient central finite differences and the dot product with the
tangent-linear model.
"""
import itertools
import json
import math
import os
from collections import deque

import numpy as np
import pytest

import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Q1 interpolation (Sec. 3, the interpolation at the feet)

def test_q1_exact_on_bilinear(orc):
    g = np.random.default_rng(1)
    nx, ny = 7, 5
    lo, hi = (-1.0, 0.5), (2.0, 3.0)
    x = np.linspace(lo[0], hi[0], nx)
    y = np.linspace(lo[1], hi[1], ny)
    X, Y = np.meshgrid(x, y, indexing="xy")
    a, b, c, d = g.normal(size=4)
    F = a + b * X + c * Y + d * X * Y
    p = orc.Problem((nx, ny), lo, hi, [[1.0, 0.0]], np.zeros((ny, nx)), h=0.1)
    for _ in range(200):
        q = g.uniform(lo, hi)
        exact = a + b * q[0] + c * q[1] + d * q[0] * q[1]
        assert abs(orc.interp(p, F, q) - exact) < 1e-12


def test_q1_exact_on_trilinear_and_periodic_wrap(orc):
    g = np.random.default_rng(2)
    n = (4, 6, 5)
    lo, hi = (0.0, -1.0, 2.0), (1.5, 1.0, 3.0)
    ax = [np.linspace(lo[d], hi[d], n[d]) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    cf = g.normal(size=8)

    def f(x, y, z):
        return (cf[0] + cf[1] * x + cf[2] * y + cf[3] * z + cf[4] * x * y + cf[5] * y * z
                + cf[6] * x * z + cf[7] * x * y * z)

    F = f(X, Y, Z)
    p = orc.Problem(n, lo, hi, [[0.0]], np.zeros(F.shape), h=0.1, dyn=1)
    for _ in range(200):
        q = g.uniform(lo, hi)
        assert abs(orc.interp(p, F, q) - f(*q)) < 1e-12
    # periodic third dimension: n nodes on a period; the last cell wraps to node 0
    pp = orc.Problem(n, lo, hi, [[0.0]], np.zeros(F.shape), h=0.1, dyn=1, periodic=(0, 0, 1))
    V = g.normal(size=F.shape)
    dz = (hi[2] - lo[2]) / n[2]
    xq, yq = ax[0][1], ax[1][2]
    for t in (0.0, 0.25, 0.5, 0.9):
        zq = lo[2] + (n[2] - 1 + t) * dz
        want = (1 - t) * V[n[2] - 1, 2, 1] + t * V[0, 2, 1]
        assert abs(orc.interp(pp, V, (xq, yq, zq)) - want) < 1e-12
        assert abs(orc.interp(pp, V, (xq, yq, zq + (hi[2] - lo[2]))) - want) < 1e-12


# --------------------------------------------------------------------------
# Brute force: the optimal value of a discounted problem with finitely many
# states is the componentwise minimum over deterministic stationary policies
# of the policy values, each the solution of a linear system.

def _grid_index(shape, idx):
    out, mul = 0, 1
    for d in range(len(shape)):
        out += idx[d] * mul
        mul *= shape[d]
    return out


def _stencil(shape, spacing, periodic, idx, off, p1=False):
    """Independent restatement of the foot rule: returns None when the foot
    is outside the closed box (beyond 1e-6 cells), else [(flat, weight)].
    p1 (2D): the barycentric weights of the triangle of the cell's split
    along its (0,0)-(1,1) diagonal that holds the foot."""
    nd = len(shape)
    cells = []
    for d in range(nd):
        o = off[d] / spacing[d]
        gd = idx[d] + o
        n = shape[d]
        if periodic[d]:
            gd = gd % n
            c = min(int(math.floor(gd)), n - 1)
            cells.append((c, (c + 1) % n, gd - c))
        else:
            if o < -idx[d] - 1e-6 or o > (n - 1 - idx[d]) + 1e-6:
                return None
            gd = min(max(gd, 0.0), n - 1.0)
            c = min(max(int(math.floor(gd)), 0), n - 2)
            cells.append((c, c + 1, gd - c))
    if p1:
        (x0, x1, tx), (y0, y1, ty) = cells
        if tx >= ty:
            corners = [((x0, y0), 1 - tx), ((x1, y0), tx - ty), ((x1, y1), ty)]
        else:
            corners = [((x0, y0), 1 - ty), ((x0, y1), ty - tx), ((x1, y1), tx)]
        return [(_grid_index(shape, list(c)), w) for c, w in corners]
    out = []
    for bits in itertools.product((0, 1), repeat=nd):
        w, ii = 1.0, []
        for d, bt in enumerate(bits):
            c0, c1, t = cells[d]
            ii.append(c1 if bt else c0)
            w *= t if bt else 1.0 - t
        out.append((_grid_index(shape, ii), w))
    return out


def _brute_force(shape, spacing, periodic, target, feet, cost, lam, h, v_out, implicit=False,
                 p1=False):
    """feet[i][j] = physical offset h f(x_i, a_j).  Returns the optimal V.
    Step weights: e^{-lam h} and (1 - e^{-lam h}) / lam, or with implicit the
    1 / (1 + lam h) and h / (1 + lam h) of the printed scheme."""
    N = int(np.prod(shape))
    if implicit:
        beta, gam = 1.0 / (1.0 + lam * h), h / (1.0 + lam * h)
    else:
        beta = math.exp(-lam * h)
        gam = (1 - beta) / lam
    free = [i for i in range(N) if target[i] == 0]
    pos = {i: k for k, i in enumerate(free)}
    F, A = len(free), len(feet[free[0]])
    R = np.zeros((F, A, F))
    b = np.zeros((F, A))
    for k, i in enumerate(free):
        idx = []
        r = i
        for d in range(len(shape)):
            idx.append(r % shape[d])
            r //= shape[d]
        for j in range(A):
            st = _stencil(shape, spacing, periodic, idx, feet[i][j], p1=p1)
            b[k, j] = gam * cost[i]
            if st is None:
                b[k, j] += beta * v_out
                continue
            for flat, w in st:
                if target[flat] == 0:
                    R[k, j, pos[flat]] += w
    pols = np.array(list(itertools.product(range(A), repeat=F)), dtype=np.int64)
    ar = np.arange(F)
    M = np.eye(F)[None] - beta * R[ar[None, :], pols]
    rhs = b[ar[None, :], pols]
    vals = np.linalg.solve(M, rhs[..., None])[..., 0]
    vstar = vals.min(axis=0)
    # a single policy attains the minimum in every component
    assert np.abs(vals - vstar[None]).max(axis=1).min() < 1e-12
    V = np.zeros(N)
    V[free] = vstar
    return V


def test_brute_force_speed_current_cost(orc):
    g = np.random.default_rng(3)
    shape = (4, 3)
    lo, hi = (0.0, 0.0), (3.0, 1.0)  # dx = 1, dy = 0.5: anisotropic cells
    spacing = (1.0, 0.5)
    N = 12
    target = np.zeros(N, dtype=np.int32)
    target[[0, 7, 9, 10]] = [1, 2, 1, 3]
    ang = 0.3 + np.pi / 2 * np.arange(4)
    ctr = np.stack([np.cos(ang), np.sin(ang)], 1)
    s = g.uniform(0.5, 1.5, N)
    cur = g.uniform(-0.2, 0.2, (N, 2))
    cost = g.uniform(0.5, 2.0, N)
    lam, h, v_out = 0.7, 0.8, 3.0
    feet = [[h * (s[i] * ctr[j] + cur[i]) for j in range(4)] for i in range(N)]
    Vb = _brute_force(shape, spacing, (0, 0), target, feet, cost, lam, h, v_out)
    p = orc.Problem(shape, lo, hi, ctr, target, h=h, lam=lam, speed=s, current=cur, cost=cost,
                    v_out=v_out)
    V, it, r = orc.solve(p, tol=1e-15, max_iters=100000)
    assert np.abs(V - Vb).max() < 1e-12


def test_brute_force_implicit_weights(orc):
    """The weights printed in the scheme of Sec. 3, 1/(1 + lambda h) and
    h/(1 + lambda h), against the brute-force solve with the same weights."""
    g = np.random.default_rng(5)
    shape = (4, 3)
    lo, hi = (0.0, 0.0), (3.0, 1.0)
    N = 12
    target = np.zeros(N, dtype=np.int32)
    target[[0, 7, 10]] = [1, 2, 1]
    ang = 0.4 + np.pi / 2 * np.arange(4)
    ctr = np.stack([np.cos(ang), np.sin(ang)], 1)
    s = g.uniform(0.5, 1.5, N)
    cost = g.uniform(0.5, 2.0, N)
    lam, h, v_out = 1.3, 0.6, 2.0
    feet = [[h * s[i] * ctr[j] for j in range(4)] for i in range(N)]
    Vb = _brute_force(shape, (1.0, 0.5), (0, 0), target, feet, cost, lam, h, v_out, implicit=True)
    p = orc.Problem(shape, lo, hi, ctr, target, h=h, lam=lam, speed=s, cost=cost, v_out=v_out,
                    weights=1)
    V, _, _ = orc.solve(p, tol=1e-15, max_iters=100000)
    assert np.abs(V - Vb).max() < 1e-12
    q = orc.Problem(shape, lo, hi, ctr, target, h=h, lam=lam, speed=s, cost=cost, v_out=v_out)
    assert np.abs(orc.solve(q, tol=1e-15, max_iters=100000)[0] - Vb).max() > 1e-3


def test_p1_interpolation_closed_forms(orc):
    """P1 on the Kuhn triangles (Sec. 3: linear interpolation in n
    dimensions): exact on affine data; on the corner data (0, 0, 0, 1) of
    one cell (the function xy) it is min(t_x, t_y), where Q1 gives t_x t_y."""
    g = np.random.default_rng(21)
    lab = np.zeros((3, 4), np.uint8)
    lab[0, 0] = 1
    ctr = np.array([[1.0, 0.0]])
    p = orc.Problem((4, 3), (0.0, 0.0), (3.0, 2.0), ctr, lab, 0.5, interp=1)
    q = orc.Problem((4, 3), (0.0, 0.0), (3.0, 2.0), ctr, lab, 0.5)
    X, Y = np.meshgrid(np.arange(4.0), np.arange(3.0))
    a, b, c = g.normal(size=3)
    V = (a + b * X + c * Y).reshape(-1)
    for y in g.uniform([0, 0], [3, 2], size=(50, 2)):
        assert abs(orc.interp(p, V, y) - (a + b * y[0] + c * y[1])) < 1e-12
    e = np.zeros(12)
    e[1 * 4 + 2] = 1.0  # node (2, 1): the (1,1) corner of cell (1, 0)
    for t in g.uniform(0, 1, size=(50, 2)):
        y = np.array([1.0 + t[0], 0.0 + t[1]])
        assert abs(orc.interp(p, e, y) - min(t[0], t[1])) < 1e-12
        assert abs(orc.interp(q, e, y) - t[0] * t[1]) < 1e-12


def test_brute_force_p1(orc):
    g = np.random.default_rng(9)
    shape = (4, 3)
    lo, hi = (0.0, 0.0), (3.0, 1.0)
    N = 12
    target = np.zeros(N, dtype=np.int32)
    target[[0, 7, 9]] = [1, 2, 1]
    ang = 0.3 + np.pi / 2 * np.arange(4)
    ctr = np.stack([np.cos(ang), np.sin(ang)], 1)
    s = g.uniform(0.5, 1.5, N)
    cur = g.uniform(-0.2, 0.2, (N, 2))
    cost = g.uniform(0.5, 2.0, N)
    lam, h, v_out = 0.7, 0.8, 3.0
    feet = [[h * (s[i] * ctr[j] + cur[i]) for j in range(4)] for i in range(N)]
    Vb = _brute_force(shape, (1.0, 0.5), (0, 0), target, feet, cost, lam, h, v_out, p1=True)
    p = orc.Problem(shape, lo, hi, ctr, target, h=h, lam=lam, speed=s, current=cur, cost=cost,
                    v_out=v_out, interp=1)
    V, _, _ = orc.solve(p, tol=1e-15, max_iters=100000)
    assert np.abs(V - Vb).max() < 1e-12
    Vq = _brute_force(shape, (1.0, 0.5), (0, 0), target, feet, cost, lam, h, v_out)
    assert np.abs(Vq - Vb).max() > 1e-4


def test_brute_force_long_feet_constant_drift(orc):
    shape = (3, 3)
    lo, hi = (-1.0, -1.0), (1.0, 1.0)
    target = np.zeros(9, dtype=np.int32)
    target[4] = 1
    ang = 0.1 + np.pi / 2 * np.arange(4)
    ctr = np.stack([np.cos(ang), np.sin(ang)], 1)
    cur = np.tile([0.2, -0.1], (9, 1))
    h = 1.3
    feet = [[h * (ctr[j] + cur[i]) for j in range(4)] for i in range(9)]
    Vb = _brute_force(shape, (1.0, 1.0), (0, 0), target, feet, np.ones(9), 1.0, h, 1.0)
    p = orc.Problem(shape, lo, hi, ctr, target, h=h, current=cur)
    V, _, _ = orc.solve(p, tol=1e-15)
    assert np.abs(V - Vb).max() < 1e-12


def test_brute_force_dubins_periodic(orc):
    shape = (2, 2, 3)
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 2 * np.pi)
    N = 12
    target = np.zeros(N, dtype=np.int32)
    for t in range(3):
        target[_grid_index(shape, (0, 0, t))] = 1
    ctr = np.array([[-1.0], [0.0], [1.0]])
    h = 0.7
    dth = 2 * np.pi / 3
    feet = []
    for i in range(N):
        th = (i // 4) * dth
        feet.append([np.array([h * np.cos(th), h * np.sin(th), h * u]) for u in (-1.0, 0.0, 1.0)])
    Vb = _brute_force(shape, (1.0, 1.0, dth), (0, 0, 1), target, feet, np.ones(N), 1.0, h, 1.0)
    p = orc.Problem(shape, lo, hi, ctr, target, h=h, dyn=1, periodic=(0, 0, 1))
    V, _, _ = orc.solve(p, tol=1e-15)
    assert np.abs(V - Vb).max() < 1e-12


# --------------------------------------------------------------------------
# Policy iteration (Howard): an exact solver of the same discrete problem by
# alternating exact policy evaluation (a sparse linear solve) and greedy
# improvement.  It stops when no node's control can improve, which for a
# discounted problem happens after finitely many steps at the optimal value,
# so it pins the value iteration at sizes brute force cannot reach.

def _transitions(shape, spacing, periodic, target, feet, cost, lam, h, v_out, implicit=False,
                 p1=False, ghost=None):
    """(R, b, free, beta): R sparse [F * A, F], row k * A + j the interpolation
    weights of the foot of free node k under control j on the free nodes
    (target nodes hold 0); b [F, A] the running cost plus beta v_out for a
    foot outside the box, and beta w v_out for each stencil weight w on a
    ghost node (ghost: bool [N], nodes outside a restricted problem)."""
    import scipy.sparse as sp
    N = int(np.prod(shape))
    if implicit:
        beta, gam = 1.0 / (1.0 + lam * h), h / (1.0 + lam * h)
    else:
        beta = math.exp(-lam * h)
        gam = (1 - beta) / lam
    gh = np.zeros(N, dtype=bool) if ghost is None else np.asarray(ghost, dtype=bool)
    free = np.nonzero((np.asarray(target) == 0) & ~gh)[0]
    pos = np.full(N, -1)
    pos[free] = np.arange(len(free))
    A = len(feet[free[0]])
    rows, cols, vals = [], [], []
    b = np.zeros((len(free), A))
    for k, i in enumerate(free):
        idx, r = [], int(i)
        for d in range(len(shape)):
            idx.append(r % shape[d])
            r //= shape[d]
        for j in range(A):
            st = _stencil(shape, spacing, periodic, idx, feet[i][j], p1=p1)
            b[k, j] = gam * cost[i]
            if st is None:
                b[k, j] += beta * v_out
                continue
            for flat, w in st:
                if gh[flat]:
                    b[k, j] += beta * w * v_out
                elif pos[flat] >= 0 and w != 0.0:
                    rows.append(k * A + j)
                    cols.append(pos[flat])
                    vals.append(w)
    R = sp.csr_matrix((vals, (rows, cols)), shape=(len(free) * A, len(free)))
    return R, b, free, beta


def _howard(R, b, beta, max_steps=2000):
    """Policy iteration from the all-zero policy; a control is replaced only
    by a strictly better one (1e-13), so the iteration cannot cycle."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    F, A = b.shape
    ar = np.arange(F)
    pol = np.zeros(F, dtype=np.int64)
    eye = sp.identity(F, format="csr")
    for step in range(max_steps):
        V = spl.spsolve((eye - beta * R[ar * A + pol]).tocsc(), b[ar, pol])
        Q = b + beta * (R @ V).reshape(F, A)
        best = Q.argmin(axis=1)
        better = Q[ar, best] < Q[ar, pol] - 1e-13
        if not better.any():
            return V, step
        pol = np.where(better, best, pol)
    raise AssertionError("policy iteration did not terminate")


def _zermelo_fields(n, A, seed):
    X, Y = S.mesh2(n, n)
    g = np.random.default_rng(seed)
    s = S.speed_field(g, X, Y).reshape(-1)
    cur = S.current_field(g, X, Y).reshape(-1, 2)
    cost = g.uniform(0.5, 2.0, n * n)
    cen = S.disk_centers(g, 3, radius=0.15)
    lab = S.disk_labels(X, Y, cen, 0.15).reshape(-1)
    return s, cur, cost, lab


@pytest.mark.parametrize("variant", ["q1", "implicit", "p1"])
def test_policy_iteration_zermelo(orc, variant):
    """41^2 grid, 16 controls, speed, divergence-free current, cost field,
    lambda = 0.8, three target disks: the value iteration's fixed point equals
    Howard's exact solution, with the exponential or the printed implicit step
    weights, with Q1 or P1 interpolation."""
    n, A = 41, 16
    s, cur, cost, lab = _zermelo_fields(n, A, 21)
    ctr = S.circle_controls(A)
    h, lam, v_out = 2.0 / (n - 1), 0.8, 2.5
    dx = 2.0 / (n - 1)
    feet = [[h * (s[i] * ctr[j] + cur[i]) for j in range(A)] for i in range(n * n)]
    implicit, p1 = variant == "implicit", variant == "p1"
    R, b, free, beta = _transitions((n, n), (dx, dx), (0, 0), lab, feet, cost, lam, h, v_out,
                                    implicit=implicit, p1=p1)
    Vh, steps = _howard(R, b, beta)
    assert steps >= 2
    p = orc.Problem((n, n), (-1, -1), (1, 1), ctr, lab, h, lam=lam, speed=s, current=cur,
                    cost=cost, v_out=v_out, weights=int(implicit), interp=int(p1))
    V, _, _ = orc.solve(p, tol=1e-14, max_iters=1_000_000)
    assert np.abs(V[free] - Vh).max() < 1e-11
    assert np.abs(V[lab != 0]).max() == 0.0


@pytest.mark.parametrize("own", [False, True])
def test_policy_iteration_restricted_subproblems(orc, own):
    """ISA step 3 (Sec. 4) on the oracle's own decomposition of a 33^2 problem
    with three targets (threshold 0.5, so that sub-domains reach into other
    components): each restricted solve equals Howard's exact solution
    of the problem on that sub-domain (nodes outside it are ghosts carrying
    value_out), with every target node inside the sub-domain as a target
    (the operator of Sec. 4 as written), or only target component k (the
    target choice of RA step 1, Sec. 3)."""
    n, A = 33, 16
    s, cur, cost, lab = _zermelo_fields(n, A, 22)
    ctr = S.circle_controls(A)
    h = dx = 2.0 / (n - 1)
    p = orc.Problem((n, n), (-1, -1), (1, 1), ctr, lab, h, lam=0.8, speed=s, current=cur,
                    cost=cost, v_out=2.5)
    _, lab_c, _ = orc.ra(p, (4, 4), 0.5, tol=1e-13)
    fine = orc.project(p, (4, 4), lab_c)
    Vbar, unc, _, Vk = orc.isa(p, fine, tol=1e-14, keep_vk=True, own_targets=own)
    feet = [[h * (s[i] * ctr[j] + cur[i]) for j in range(A)] for i in range(n * n)]
    m = int(lab.max())
    assert m == 3
    for k in range(m):
        inside = ((fine >> k) & 1) == 1
        assert 0 < inside.sum() < n * n
        tk = np.where(inside & ((lab == k + 1) if own else (lab != 0)), lab, 0)
        R, b, free, beta = _transitions((n, n), (dx, dx), (0, 0), tk, feet, cost, 0.8, h, 2.5,
                                        ghost=~inside)
        Vh, _ = _howard(R, b, beta)
        assert np.abs(Vk[k][free] - Vh).max() < 1e-11
    # the assembly: the minimum over the sub-domains holding a node
    ref = np.where(fine != 0, np.min(np.where(((fine[None, :] >> np.arange(m)[:, None]) & 1) == 1,
                                              Vk, np.inf), axis=0), 2.5)
    assert np.array_equal(Vbar, ref)
    # at this threshold sub-domains 1 and 3 hold nodes of other components,
    # so the two choices of targets are different problems
    other = [int(np.sum(((fine >> k) & 1)[(lab != 0) & (lab != k + 1)])) for k in range(m)]
    assert max(other) > 0
    if own:
        _, _, _, Vk3 = orc.isa(p, fine, tol=1e-14, keep_vk=True)
        assert np.abs(Vk - Vk3).max() > 0.1


def test_policy_iteration_dubins(orc):
    """Dubins car on 16 x 16 x 12 with periodic heading, three turn rates,
    two target disks: value iteration equals Howard's exact solution."""
    nx, nth = 16, 12
    shape = (nx, nx, nth)
    dx, dth = 2.0 / (nx - 1), 2 * np.pi / nth
    h = dx
    x = np.linspace(-1, 1, nx)
    lab = np.zeros(shape[::-1], dtype=np.int32)
    for k, (cx, cy) in enumerate([(-0.4, 0.3), (0.5, -0.5)]):
        inside = (x[None, :] - cx) ** 2 + (x[:, None] - cy) ** 2 <= 0.3 ** 2
        lab[:, inside] = k + 1
    lab = lab.reshape(-1)
    N = lab.size
    feet = []
    for i in range(N):
        th = (i // (nx * nx)) * dth
        feet.append([np.array([h * np.cos(th), h * np.sin(th), h * u]) for u in (-1.0, 0.0, 1.0)])
    R, b, free, beta = _transitions(shape, (dx, dx, dth), (0, 0, 1), lab, feet, np.ones(N), 1.0,
                                    h, 1.0)
    Vh, steps = _howard(R, b, beta)
    assert steps >= 2
    p = orc.Problem(shape, (-1, -1, 0), (1, 1, 2 * np.pi), [[-1.0], [0.0], [1.0]], lab, h,
                    dyn=1, periodic=(0, 0, 1))
    V, _, _ = orc.solve(p, tol=1e-14, max_iters=1_000_000)
    assert np.abs(V[free] - Vh).max() < 1e-11


# --------------------------------------------------------------------------
# Graph special case: every foot lands on a node, so V = 1 - beta^k with k
# the graph distance to the target set (lambda = 1, l = 1).

def _bfs(n_nodes, sources, neighbours):
    dist = np.full(n_nodes, -1)
    q = deque()
    for s in sources:
        dist[s] = 0
        q.append(s)
    while q:
        u = q.popleft()
        for v in neighbours(u):
            if dist[v] < 0:
                dist[v] = dist[u] + 1
                q.append(v)
    return dist


@pytest.mark.parametrize("moves", ["axis", "king"])
def test_graph_distance_2d(orc, moves):
    nx, ny = 13, 9
    g = np.random.default_rng(4)
    target = np.zeros(nx * ny, dtype=np.int32)
    target[g.choice(nx * ny, 3, replace=False)] = [1, 2, 3]
    ctr = S.axis_controls() if moves == "axis" else S.king_controls()
    h = 1.0
    p = orc.Problem((nx, ny), (0.0, 0.0), (nx - 1.0, ny - 1.0), ctr, target, h=h)
    V, _, _ = orc.solve(p, tol=1e-15)
    steps = [tuple(int(v) for v in c) for c in ctr]

    def nb(u):  # reversed edges: v -> u whenever u = v + step
        x, y = u % nx, u // nx
        out = []
        for dx, dy in steps:
            vx, vy = x - dx, y - dy
            if 0 <= vx < nx and 0 <= vy < ny and target[vy * nx + vx] == 0:
                out.append(vy * nx + vx)
        return out

    k = _bfs(nx * ny, np.nonzero(target)[0], nb)
    assert (k >= 0).all()
    want = 1.0 - np.exp(-h) ** k
    assert np.abs(V - want).max() < 1e-12


def test_graph_distance_dubins(orc):
    # heading grid of 4 angles; h = dx = dtheta = pi/2: a step moves one node
    # along the heading and turns by u * 90 degrees.
    nx, ny, nt = 7, 6, 4
    d = np.pi / 2
    shape = (nx, ny, nt)
    N = nx * ny * nt
    g = np.random.default_rng(5)
    cells = g.choice(nx * ny, 2, replace=False)
    target = np.zeros(N, dtype=np.int32)
    for t in range(nt):
        target[cells + t * nx * ny] = [1, 2]
    p = orc.Problem(shape, (0.0, 0.0, 0.0), ((nx - 1) * d, (ny - 1) * d, 2 * np.pi),
                    [[-1.0], [0.0], [1.0]], target, h=d, dyn=1, periodic=(0, 0, 1))
    V, _, _ = orc.solve(p, tol=1e-15)
    head = [(1, 0), (0, 1), (-1, 0), (0, -1)]
    fwd = {}
    for v in range(N):
        x, y, t = v % nx, (v // nx) % ny, v // (nx * ny)
        for u in (-1, 0, 1):
            X, Y, Tn = x + head[t][0], y + head[t][1], (t + u) % nt
            if 0 <= X < nx and 0 <= Y < ny:
                fwd.setdefault(X + Y * nx + Tn * nx * ny, []).append(v)

    def nb(u):
        return [v for v in fwd.get(u, []) if target[v] == 0]

    k = _bfs(N, np.nonzero(target)[0], nb)
    want = np.where(k >= 0, 1.0 - np.exp(-d) ** np.maximum(k, 0), 1.0)
    assert np.abs(V - want).max() < 1e-12


# --------------------------------------------------------------------------
# Closed forms

def test_disk_distance_convergence(orc):
    """f = a, |a| = 1: v = 1 - exp(-dist) (Kruzhkov transform, Sec. 4.1)."""
    errs = []
    for n in (51, 101, 201):
        d = S.c1(n=n)
        p = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"])
        V, _, _ = orc.solve(p, tol=1e-12, nthreads=4)
        X, Y = S.mesh2(n, n)
        dist = np.min([np.maximum(np.hypot(X - c[0], Y - c[1]) - 0.1, 0) for c in d["centers"]], 0)
        errs.append(np.abs(V.reshape(n, n) - (1 - np.exp(-dist))).max())
    assert errs[1] < 0.025
    assert errs[0] / errs[1] > 1.6 and errs[1] / errs[2] > 1.6


def _drift_time(X, Y, q, rho, c):
    dxx, dyy = q[0] - X, q[1] - Y
    dc = dxx * c[0] + dyy * c[1]
    c2 = c[0] ** 2 + c[1] ** 2
    dd = dxx ** 2 + dyy ** 2
    T = (-(dc + rho) + np.sqrt((dc + rho) ** 2 + (1 - c2) * (dd - rho ** 2))) / (1 - c2)
    return np.where(dd <= rho ** 2, 0.0, T)


def test_constant_drift_closed_form(orc):
    """f = a + c with constant c: the reachable set at time T is the disk of
    radius T around x + cT, so the arrival time at a disk solves a quadratic.
    Pins the sign of the foot (x + h f) and the x/y order of the current."""
    c = (0.3, -0.15)
    cen = [(-0.5, 0.4), (0.45, -0.3)]
    rho = 0.15
    errs = []
    for n in (51, 101, 201):
        X, Y = S.mesh2(n, n)
        lab = S.disk_labels(X, Y, np.array(cen), rho)
        cur = np.tile(c, (n * n, 1))
        p = orc.Problem((n, n), (-1, -1), (1, 1), S.circle_controls(64), lab, 2 / (n - 1),
                        current=cur)
        V, _, _ = orc.solve(p, tol=1e-12, nthreads=4)
        T = np.minimum(*[_drift_time(X, Y, q, rho, c) for q in cen])
        errs.append(np.abs(V.reshape(n, n) - (1 - np.exp(-T))).max())
    assert errs[1] < 0.03
    assert errs[0] > errs[1] > errs[2]
    # the mirrored current must give a clearly different answer
    n = 101
    X, Y = S.mesh2(n, n)
    T_wrong = np.minimum(*[_drift_time(X, Y, q, rho, (c[1], c[0])) for q in cen])
    assert np.abs(V.reshape(201, 201)[::2, ::2] - (1 - np.exp(-T_wrong))).max() > 0.05


@pytest.mark.parametrize("delta", [1.0, 0.5])
def test_strip_example_exact(orc, delta):
    """Example 3.1 (Sec. 3): strip, f = a_1, lambda = delta, l = 1, exits at
    x1 = +-1 with g = 0.  Corrected closed form (the printed one is garbled):
    v = (1 - exp(-delta (1 - |x1|)))/delta.  With axis controls and h = dx the
    scheme is exact at the nodes."""
    nx, ny = 41, 8
    target = np.zeros((ny, nx), dtype=np.int32)
    target[:, 0] = 2
    target[:, -1] = 1
    h = 2.0 / (nx - 1)
    p = orc.Problem((nx, ny), (-1.0, 0.0), (1.0, 1.0), S.axis_controls(), target, h=h,
                    lam=delta, periodic=(0, 1), v_out=1.0 / delta)
    V, _, _ = orc.solve(p, tol=1e-15)
    x = np.linspace(-1, 1, nx)
    want = (1 - np.exp(-delta * (1 - np.abs(x)))) / delta
    assert np.abs(V.reshape(ny, nx) - want[None, :]).max() < 1e-12
    # off-node feet (32 controls, h = dx/2) converge to the same closed form
    errs = []
    for m in (41, 81):
        tg = np.zeros((ny, m), dtype=np.int32)
        tg[:, 0] = 2
        tg[:, -1] = 1
        p2 = orc.Problem((m, ny), (-1.0, 0.0), (1.0, 1.0), S.circle_controls(32), tg,
                         h=1.0 / (m - 1), lam=delta, periodic=(0, 1), v_out=1.0 / delta)
        V2, _, _ = orc.solve(p2, tol=1e-13)
        xm = np.linspace(-1, 1, m)
        wm = (1 - np.exp(-delta * (1 - np.abs(xm)))) / delta
        errs.append(np.abs(V2.reshape(ny, m) - wm[None, :]).max())
    assert errs[0] < 6e-3 and errs[0] / errs[1] > 1.8


def _box_labels(n):
    lab = np.zeros((n, n), dtype=np.int32)
    lab[0, :] = 1      # y = -1
    lab[:, n - 1] = 2  # x = +1
    lab[n - 1, :] = 3  # y = +1
    lab[:, 0] = 4      # x = -1
    return lab


def test_box_boundary_distance_exact(orc):
    """Sec. 4.1: distance to the boundary of (-1,1)^2, lambda = 1:
    v = 1 - exp(-(1 - max(|x1|, |x2|))) (the printed 'min' is a misprint)."""
    n = 81
    p = orc.Problem((n, n), (-1, -1), (1, 1), S.circle_controls(32), _box_labels(n), 2 / (n - 1))
    V, _, _ = orc.solve(p, tol=1e-14)
    X, Y = S.mesh2(n, n)
    want = 1 - np.exp(-(1 - np.maximum(np.abs(X), np.abs(Y))))
    assert np.abs(V.reshape(n, n) - want).max() < 1e-12


# --------------------------------------------------------------------------
# Invariants (Sec. 3)

def _sym_problem(orc, shape, lo, hi, ctr, lab, **kw):
    p = orc.Problem(shape, lo, hi, ctr, lab, 0.08, lam=0.8, v_out=2.0, **kw)
    return orc.solve(p, tol=1e-14)[0].reshape(shape[1], shape[0])


@pytest.mark.parametrize("fields", ["speed", "scale", "p1"])
def test_symmetries_of_the_scheme(orc, fields):
    """The discrete problem (Sec. 3) on a non-square grid with an asymmetric
    control set, speed or per-axis factors, a current and a cost field:
    mirroring x (controls, current x-component, every field and the targets)
    mirrors V, and exchanging x and y (grid, box, fields, vector components)
    transposes V, to rounding.  This catches what a single case cannot:
    lower and upper faces handled differently, the two spacings or strides
    mixed up.  The P1 split along the (0,0)-(1,1) diagonal is invariant under
    the exchange of x and y but not under the mirror, which maps it to the
    other diagonal (a different scheme), so P1 is checked under the exchange
    only."""
    g = np.random.default_rng(5)
    nx, ny = 23, 17
    lo, hi = (-1.0, -0.7), (1.0, 0.9)
    X, Y = S.mesh2(nx, ny, lo=lo, hi=hi)
    lab = S.disk_labels(X, Y, np.array([[-0.4, 0.2], [0.5, -0.3]]), 0.2)
    cur = g.uniform(-0.3, 0.3, X.shape + (2,))
    cost = g.uniform(0.5, 2.0, X.shape)
    F = g.uniform(0.4, 1.4, X.shape + (2,)) if fields == "scale" else g.uniform(0.5, 1.5, X.shape)
    ctr = S.circle_controls(12) @ np.array([[1.0, 0.2], [0.1, 0.9]])
    key = "scale" if fields == "scale" else "speed"
    extra = dict(interp=1) if fields == "p1" else {}
    c = np.ascontiguousarray
    V = _sym_problem(orc, (nx, ny), lo, hi, ctr, lab, current=cur, cost=cost, **{key: F}, **extra)
    if fields != "p1":
        Vm = _sym_problem(orc, (nx, ny), lo, hi, ctr * [-1, 1], c(lab[:, ::-1]),
                          current=c(cur[:, ::-1] * [-1, 1]), cost=c(cost[:, ::-1]),
                          **{key: c(F[:, ::-1])}, **extra)
        assert np.abs(Vm[:, ::-1] - V).max() < 1e-12
    Ft = c(F.transpose(1, 0, 2)[..., ::-1]) if fields == "scale" else c(F.T)
    Vt = _sym_problem(orc, (ny, nx), lo[::-1], hi[::-1], c(ctr[:, ::-1]), c(lab.T),
                      current=c(cur.transpose(1, 0, 2)[..., ::-1]), cost=c(cost.T),
                      **{key: Ft}, **extra)
    assert np.abs(Vt.T - V).max() < 1e-12


def test_symmetry_of_the_dubins_scheme(orc):
    """Dubins car (Sec. 5 setting, heading periodic on [-pi, pi)): mirroring
    y together with the heading (theta -> -theta, node k -> n - k) and the
    turn rate (u -> -u) mirrors V, to rounding."""
    n, nth = 21, 16
    x = np.linspace(-1, 1, n)
    lab = np.zeros((nth, n, n), dtype=np.int32)
    lab[:, (x[None, :] - 0.3) ** 2 + (x[:, None] - 0.35) ** 2 <= 0.25 ** 2] = 1
    h = 2.0 / (n - 1)
    box = ((-1, -1, -np.pi), (1, 1, np.pi))

    def solve(u, labels):
        p = orc.Problem((n, n, nth), *box, u, labels, h, dyn=1, periodic=(0, 0, 1))
        return orc.solve(p, tol=1e-14)[0].reshape(nth, n, n)

    V = solve([[-1.0], [0.0], [1.0]], lab)
    Vm = solve([[1.0], [0.0], [-1.0]], np.ascontiguousarray(lab[:, ::-1, :]))
    assert np.abs(Vm[(-np.arange(nth)) % nth][:, ::-1, :] - V).max() < 1e-12


def test_iteration_invariants(orc):
    d = S.c2(n=65)
    p = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"],
                    speed=d["speed"], current=d["current"])
    V = orc.initial(p)
    for _ in range(60):
        Vn, r = orc.apply(p, V)
        assert (Vn <= V + 1e-15).all()  # monotone from the supersolution start
        assert (Vn >= 0).all() and (Vn <= 1).all()
        V = Vn
    Vs, it, r = orc.solve(p, tol=1e-13)
    assert r <= 1e-13
    assert (Vs <= V + 1e-15).all()
    # contraction bound of the stopping remark: ||V^n - V*|| <= beta/(1-beta) r_n
    V = orc.initial(p)
    for _ in range(40):
        Vn, r = orc.apply(p, V)
        V = Vn
    Vn, r = orc.apply(p, V)
    beta = p.beta
    assert np.abs(Vn - Vs).max() <= beta / (1 - beta) * r + 1e-12
    # Gauss-Seidel reaches the same fixed point
    Vg, _, _ = orc.solve(p, tol=1e-13, gs=True)
    assert np.abs(Vg - Vs).max() < 1e-11


def test_ra_invariants_and_exact_quarters(orc):
    """RA (Sec. 3): every node carries a label, X_k is in Sigma_k, V <= V_k,
    and for the 4-split of the box boundary the sets tend to the exact
    quarters (25 %, Table 1)."""
    fr = []
    for n in (41, 81):
        p = orc.Problem((n, n), (-1, -1), (1, 1), S.circle_controls(32), _box_labels(n),
                        2 / (n - 1))
        Vaux, lab, ties = orc.ra(p, (1, 1), 1e-9)
        Vfull, _, _ = orc.solve(p, tol=1e-14)
        assert (lab != 0).all()
        tl = _box_labels(n).reshape(-1)
        for k in range(4):
            assert ((lab >> k) & 1)[tl == k + 1].all()
            assert (Vfull <= Vaux[k] + 1e-12).all()
        fr.append(max(((lab >> k) & 1).mean() for k in range(4)))
    assert 0.25 <= fr[1] < fr[0] <= 0.25 + 1.5 / 41


def test_resplitting_reaches_the_four_sides(orc):
    """Recursive re-splitting of the target components (Conclusions; reading
    R22).  The box boundary divided into two components (bottom + right,
    top + left): the first split separates bottom from right, the second top
    from left -- the same coarse labels and projected sub-domains, up to the
    numbering of the components, as RA run directly on the four sides.
    Further splits (of single sides) keep shrinking the largest sub-domain,
    never growing it."""
    n, st = 41, 4
    four = _box_labels(n)
    two = np.where(four <= 2, np.where(four > 0, 1, 0), 2)
    p2 = orc.Problem((n, n), (-1, -1), (1, 1), S.circle_controls(32), two, 2 / (n - 1))
    p4 = orc.Problem((n, n), (-1, -1), (1, 1), S.circle_controls(32), four, 2 / (n - 1))
    Vaux, _, _ = orc.ra(p2, (st, st), 0.0, tol=1e-13)
    delta, _ = orc.delta(p2, (st, st), Vaux)  # 2 M dx_K, the same for every division
    comp, fine, m, largest = orc.ra_split(p2, (st, st), delta, max_splits=2, tol=1e-13)
    assert m == 4
    # the split components are the four sides (in the order of the splits)
    f4 = four.reshape(-1)
    ren = {}
    for c in range(1, 5):
        sides = np.unique(f4[comp == c])
        assert len(sides) == 1 and sides[0] != 0
        ren[c] = int(sides[0])
    assert sorted(ren.values()) == [1, 2, 3, 4]
    assert np.array_equal((comp != 0), (f4 != 0))
    _, lab4, _ = orc.ra(p4, (st, st), delta, tol=1e-13)
    fine4 = orc.project(p4, (st, st), lab4)
    perm = np.zeros_like(fine)
    for k_split, k_direct in ren.items():
        perm |= ((fine >> (k_split - 1)) & 1) << (k_direct - 1)
    assert np.array_equal(perm, fine4)
    assert largest == max(int(((fine4 >> k) & 1).sum()) for k in range(4))
    # without splits the two halves are much larger (the threshold is wide here)
    _, _, m2, largest2 = orc.ra_split(p2, (st, st), delta, max_splits=0, tol=1e-13)
    assert m2 == 2 and largest2 > 1.4 * largest
    prev = largest2
    for ms in (1, 2, 4, 6):
        _, f, mm, lg = orc.ra_split(p2, (st, st), delta, max_splits=ms, tol=1e-13)
        assert mm == 2 + ms and lg <= prev
        assert (f != 0).all()  # every node stays in some sub-domain
        prev = lg


def test_resplitting_keeps_an_unbalanced_division(orc):
    """Van der Pol (Sec. 5, Example ex3): every slice of the small target
    disk costs nearly the same from far away, so splitting the largest
    slice does not shrink its sub-domain and the refinement keeps the given
    division (the direct RA's sub-domains)."""
    d = S.vdp(n=41, slices=4, stride=4)
    p = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"],
                    current=d["current"], cost=d["cost"], v_out=d["v_out"], ntargets=4)
    comp, fine, m, largest = orc.ra_split(p, (4, 4), 0.1, max_splits=4, tol=1e-12)
    assert m == 4
    assert np.array_equal(comp, p.target)
    _, lab, _ = orc.ra(p, (4, 4), 0.1, tol=1e-12)
    assert np.array_equal(fine, orc.project(p, (4, 4), lab))


def test_table1_shape(orc):
    """Table 1 of Sec. 4.1: the largest reconstructed sub-domain shrinks as
    the coarse grid is refined (eq. incap) towards the exact 25 %.  With the
    threshold delta = dx_K the finer rows agree with the paper within 0.05."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_table1_distance.json")))
    prev = 2.0
    for n, _, paper in gold["rows"]:
        dx = 2.0 / (n - 1)
        p = orc.Problem((n, n), (-1, -1), (1, 1), S.circle_controls(32), _box_labels(n), dx)
        _, lab, _ = orc.ra(p, (1, 1), dx)
        f = max(((lab >> k) & 1).mean() for k in range(4))
        assert f < prev and f >= gold["exact_max_fraction"]
        prev = f
        if n >= 15:
            assert abs(f - paper) < 0.05, (n, f, paper)


@pytest.mark.parametrize("case", ["scale_current_cost", "dubins"])
def test_ra_auxiliary_solves_are_the_coarse_problems(orc, case):
    """RA step 1 (Sec. 3): auxiliary problem k lives on the grid of every
    stride-th node, with every node field sampled there, time step
    h_K = stride h, and only target component k as its target.  Each
    auxiliary solution equals a direct solve of that coarse problem, built
    here by slicing the fields: per-axis factors that differ on the two axes,
    a current and a cost field, lambda != 1; and the Dubins car with a
    periodic heading (every second heading kept)."""
    g = np.random.default_rng(12)
    if case == "dubins":
        d = S.c3(nxy=33, nth=16, ntargets=3, stride=(4, 4, 2))
        stride = (4, 4, 2)
        p = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"], dyn=1,
                        periodic=d["periodic"], ntargets=3)
        lab = np.asarray(d["labels"])
        labc = lab[::2, ::4, ::4]
        q = orc.Problem(labc.shape[::-1], d["lo"], d["hi"], d["controls"], labc, d["h"] * 4,
                        dyn=1, periodic=d["periodic"], ntargets=3)
    else:
        n, m = 49, 3
        X, Y = S.mesh2(n, n)
        lab = S.disk_labels(X, Y, S.disk_centers(g, m, 0.15), 0.15)
        D = np.stack([g.uniform(0.5, 1.5, X.shape), g.uniform(0.2, 0.8, X.shape)], -1)
        cur = S.current_field(g, X, Y, cmax=0.3)
        cost = g.uniform(0.5, 2.0, X.shape)
        h = 2.0 / (n - 1)
        stride = (4, 4)
        ctr = S.circle_controls(16)
        p = orc.Problem((n, n), (-1, -1), (1, 1), ctr, lab, h, lam=0.7, scale=D, current=cur,
                        cost=cost, v_out=2.0, ntargets=m)
        sl = (slice(None, None, 4), slice(None, None, 4))
        labc = lab[sl]
        q = orc.Problem(labc.shape[::-1], (-1, -1), (1, 1), ctr, labc, h * 4, lam=0.7,
                        scale=D[sl], current=cur[sl], cost=cost[sl], v_out=2.0, ntargets=m)
    Vaux, _, _ = orc.ra(p, stride, 0.1, tol=1e-13)
    for k in range(Vaux.shape[0]):
        Vk, _, _ = orc.solve(q, tol=1e-13, only_target=k + 1)
        assert np.abs(Vaux[k] - Vk).max() < 1e-11
    # a swap of the two factors changes the coarse problem
    if case != "dubins":
        qs = orc.Problem(labc.shape[::-1], (-1, -1), (1, 1), ctr, labc, h * 4, lam=0.7,
                         scale=D[sl][..., ::-1], current=cur[sl], cost=cost[sl], v_out=2.0,
                         ntargets=m)
        assert np.abs(Vaux[0] - orc.solve(qs, tol=1e-13, only_target=1)[0]).max() > 1e-3


def test_nesting_in_threshold(orc):
    d = S.c1(n=41)
    p = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"])
    Vaux, lab_small, _ = orc.ra(p, (1, 1), 0.02)
    _, lab_big, _ = orc.ra(p, (1, 1), 0.08)
    assert ((lab_small & ~lab_big) == 0).all()
    vmin, lab2, _ = orc.label(Vaux, d["labels"], 0.02)
    assert (lab2 == lab_small).all()
    assert np.allclose(vmin, Vaux.min(0))


def test_exact_sets_inside_reconstructed_sets(orc):
    """Sec. 3 (the reconstruction contains the set it approximates): the set
    Sigma_k where target k alone gives the value (V_k = V within 1e-9, from
    full solves on the fine grid) lies inside the projected RA set of the
    coarse grid four times coarser, once the threshold is 2 dx_K (the rule
    2 M dx_K with the distance's gradient bound M = 1).  The reconstructed
    sets are not trivial (1.18 N in total), and half that threshold already
    misses a few nodes, so the check has teeth."""
    n, stride = 161, 4
    d = S.c1(n=n, A=16)
    p = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"])
    nt = orc.max_threads()
    V, _, _ = orc.solve(p, tol=1e-11, nthreads=nt)
    m = d["ntargets"]
    sig = np.array([np.abs(orc.solve(p, tol=1e-11, only_target=k + 1, nthreads=nt)[0] - V) <= 1e-9
                    for k in range(m)])
    assert sig.any(axis=0).mean() > 0.99
    dxk = stride * 2.0 / (n - 1)
    missed = {}
    for delta in (dxk, 2 * dxk):
        _, lab, _ = orc.ra(p, (stride, stride), delta, tol=1e-11, nthreads=nt)
        fine = orc.project(p, (stride, stride), lab)
        sbar = np.array([((fine >> k) & 1) == 1 for k in range(m)])
        missed[delta] = int((sig & ~sbar).sum())
        total = sbar.sum() / V.size
    assert missed[2 * dxk] == 0
    assert missed[dxk] > 0
    assert total < 1.2


# --------------------------------------------------------------------------
# Defining property of independent sub-domains (Def. and Prop. 2.1; Prop. 4.1)

def _policy_closed(p, pol, member, shape):
    """Largest subset of `member` closed under the policy stencils."""
    nx, ny = shape
    dxs = [p.spacing(0), p.spacing(1)]
    keep = member.copy()
    st = {}
    sp = p.speed if p.speed is not None else np.ones(p.N)
    cu = p.current if p.current is not None else np.zeros((p.N, 2))
    for i in np.nonzero(member)[0]:
        if p.target[i] != 0 or pol[i] < 0:
            continue
        a = p.controls[pol[i]]
        off = p.h * (sp[i] * a + cu[i])
        s = _stencil(shape, dxs, (0, 0), (i % nx, i // nx), off)
        st[i] = [] if s is None else [f for f, w in s if w > 0]
    changed = True
    while changed:
        changed = False
        for i, nbrs in st.items():
            if keep[i] and any(not keep[j] for j in nbrs):
                keep[i] = False
                changed = True
    return keep


def test_threshold_estimate_exact_cases(orc):
    """The threshold of eq. (rep), delta = 2 (C dx_K^q + M dx_K), with M
    estimated by the largest discrete gradient norm of min_k V_k on the
    coarse grid (reading R5).  Fixed by mathematics, not by a retyped
    formula: differences of an affine field are its gradient exactly
    (anisotropic spacings, so transposed axes or spacings fail); the
    estimate takes the minimum over the auxiliary solutions (a min switching
    between two affine fields has the larger slope); on V = x^2 on [-1, 1]
    centred differences give 2|x| and the one-sided edge difference 2 - dx,
    the maximum; a periodic dimension wraps (sin over a full period); and
    the C dx^q term adds 2 C dx^q."""
    nx, ny = 9, 5  # fine grid; stride 2 gives a 5 x 3 coarse grid on [-1,1] x [-1,1]
    lab = np.zeros((ny, nx), dtype=np.int32)
    lab[0, 0] = 1
    lab[-1, -1] = 2
    p = orc.Problem((nx, ny), (-1, -1), (1, 1), S.circle_controls(4), lab, 0.25)
    nk = orc.coarse_shape(p, (2, 2))
    assert nk == (5, 3)
    Xk, Yk = S.mesh2(5, 3)
    dxk = 0.5
    a, b = 0.3, -0.7
    aff = (a * Xk + b * Yk + 0.2).reshape(1, -1)
    two = np.concatenate([aff, aff + 5.0])  # the min is the first
    dl, M = orc.delta(p, (2, 2), two)
    assert abs(M - math.hypot(a, b)) < 1e-14
    assert abs(dl - 2 * M * dxk) < 1e-14
    sw = np.concatenate([(0.5 * Xk).reshape(1, -1), (-2.0 * Xk).reshape(1, -1)])
    assert abs(orc.delta(p, (2, 2), sw)[1] - 2.0) < 1e-14
    quad = np.concatenate([(Xk ** 2).reshape(1, -1)] * 2)
    assert abs(orc.delta(p, (2, 2), quad)[1] - (2 - dxk)) < 1e-14
    dl_c, _ = orc.delta(p, (2, 2), two, C_=0.7, q=0.5)
    assert abs(dl_c - (dl + 2 * 0.7 * math.sqrt(dxk))) < 1e-14
    assert abs(orc.delta(p, (2, 2), two, M=3.0)[0] - 2 * 3.0 * dxk) < 1e-14
    # periodic third dimension: 8 layers on [0, 2 pi), stride 2 keeps 4; the
    # wrapped centred difference of sin at the layer theta = 0 is
    # (sin(pi/2) - sin(-pi/2)) / pi = 2 / pi, the largest over the layers
    lab3 = np.zeros((8, ny, nx), dtype=np.int32)
    lab3[:, 0, 0] = 1
    p3 = orc.Problem((nx, ny, 8), (-1, -1, 0), (1, 1, 2 * np.pi), [[-1.0], [1.0]], lab3, 0.25,
                     periodic=(0, 0, 1), dyn=1)
    th = np.arange(4) * (np.pi / 2)
    V3 = np.broadcast_to(np.sin(th)[:, None, None], (4, 3, 5)).reshape(1, -1).copy()
    assert abs(orc.delta(p3, (2, 2, 2), V3)[1] - 2 / np.pi) < 1e-14


def test_threshold_estimate_on_the_box_distance(orc):
    """On the distance to the boundary of (-1,1)^2 (Sec. 4.1; RA with the box
    sides as the four target components) the discrete value is the closed
    form 1 - exp(-(1 - max|x|)) and its gradient norm exp(-d) <= 1 peaks at
    the boundary; the estimate is the one-sided edge difference there,
    (1 - exp(-dx_K)) / dx_K."""
    n, st = 81, 8
    p = orc.Problem((n, n), (-1, -1), (1, 1), S.circle_controls(32), _box_labels(n), 2 / (n - 1))
    Vaux, _, _ = orc.ra(p, (st, st), 0.1, tol=1e-14)
    dl, M = orc.delta(p, (st, st), Vaux)
    dxk = 2.0 / ((n - 1) // st)
    assert abs(M - (1 - math.exp(-dxk)) / dxk) < 1e-10
    assert abs(dl - 2 * M * dxk) < 1e-14


@pytest.mark.parametrize("which", ["c1", "c2"])
def test_restricted_solve_reproduces_full(orc, which):
    """Prop. 2.1 / Prop. 4.1: a solve restricted to a reconstructed
    sub-domain reproduces the full-domain values on every subset closed under
    the optimal policy; elsewhere (next to switching curves, where the
    discrete union-of-targets value mixes both basins) the assembled ISA value
    can only be larger, by at most the discretisation error."""
    if which == "c1":
        d = S.c1(n=81)
        stride = (4, 4)
    else:
        d = S.c2(n=97, ntargets=6)
        stride = (4, 4)
    n = d["shape"][0]
    p = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"],
                    speed=d["speed"], current=d["current"])
    V, _, _ = orc.solve(p, tol=1e-13)
    pol, _ = orc.policy(p, V)
    # threshold of eq. (rep) with the Lipschitz constant M estimated by the
    # largest discrete gradient of the coarse V = min_k V_k (C dx^q dropped)
    Vaux, _, _ = orc.ra(p, stride, 0.0, tol=1e-13)
    delta, _ = orc.delta(p, stride, Vaux)
    vmin, lab, _ = orc.label(Vaux, p.target.reshape(n, n)[::stride[1], ::stride[0]], delta)
    fine = orc.project(p, stride, lab)
    Vbar, unc, its, Vk = orc.isa(p, fine, tol=1e-13, keep_vk=True)
    assert unc == 0
    covered = np.zeros(p.N, dtype=bool)
    for k in range(p.ntargets):
        member = ((fine >> k) & 1).astype(bool)
        Dk = _policy_closed(p, pol, member, d["shape"])
        assert (Vk[k][member] >= V[member] - 1e-12).all()  # restriction cannot help
        assert np.abs(Vk[k][Dk] - V[Dk]).max(initial=0) < 1e-10
        covered |= Dk
    assert covered.mean() > 0.8
    assert np.abs(Vbar - V)[covered].max() < 1e-10
    assert (Vbar >= V - 1e-12).all()
    assert (Vbar - V).max() < 2 * d["h"]
    # a restriction to the whole grid is the full problem
    Vall, _, _ = orc.solve(p, tol=1e-13, mask=np.ones(p.N, dtype=np.uint32), bit=0)
    assert np.abs(Vall - V).max() < 1e-12


def test_isa_error_bound_distance(orc):
    """Prop. 4.1 and Table 3 (Sec. 4.1): the ISA value converges to the exact
    solution at the rate of the full solve, and is no farther from it."""
    errs_full, errs_isa = [], []
    for n, st in ((41, 4), (81, 4)):
        d = S.c1(n=n)
        p = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"])
        V, _, _ = orc.solve(p, tol=1e-13)
        Vaux, lab, _ = orc.ra(p, (st, st), 0.25, tol=1e-13)
        fine = orc.project(p, (st, st), lab)
        Vbar, unc, _, _ = orc.isa(p, fine, tol=1e-13)
        assert unc == 0
        X, Y = S.mesh2(n, n)
        dist = np.min([np.maximum(np.hypot(X - c[0], Y - c[1]) - 0.1, 0) for c in d["centers"]], 0)
        ex = (1 - np.exp(-dist)).reshape(-1)
        errs_full.append(np.abs(V - ex).max())
        errs_isa.append(np.abs(Vbar - ex).max())
    assert errs_isa[1] <= errs_full[1] + 1e-12
    assert errs_isa[0] / errs_isa[1] > 1.5


# --------------------------------------------------------------------------
# Projection through the concave hull Con (Sec. 4): direct enumeration of
# every face of the Kuhn triangulation whose vertices are all labelled.

def _con_2d(nK, r, coarse):
    n = (nK - 1) * r + 1
    fine = np.zeros((n, n), dtype=np.uint32)
    cl = coarse.reshape(nK, nK)
    for cy in range(nK - 1):
        for cx in range(nK - 1):
            tris = [[(0, 0), (1, 0), (1, 1)], [(0, 0), (0, 1), (1, 1)]]
            for tri in tris:
                for k in range(1, len(tri) + 1):
                    for face in itertools.combinations(tri, k):
                        bits = np.uint32(0xFFFFFFFF)
                        for vx, vy in face:
                            bits &= cl[cy + vy, cx + vx]
                        if bits == 0:
                            continue
                        # fine nodes in the closed face: convex hull test via
                        # barycentric coordinates on the lattice
                        P = np.array(face, dtype=float) * r
                        for py in range(r + 1):
                            for px in range(r + 1):
                                if _in_hull((px, py), P):
                                    fine[cy * r + py, cx * r + px] |= bits
    return fine.reshape(-1)


def _in_hull(q, P):
    q = np.array(q, dtype=float)
    if len(P) == 1:
        return np.allclose(q, P[0])
    if len(P) == 2:
        a, b = P
        ab, aq = b - a, q - a
        cross = ab[0] * aq[1] - ab[1] * aq[0]
        t = aq @ ab / (ab @ ab)
        return abs(cross) < 1e-9 and -1e-9 <= t <= 1 + 1e-9
    a, b, c = P
    M = np.array([b - a, c - a]).T
    l1, l2 = np.linalg.solve(M, q - a)
    return l1 >= -1e-9 and l2 >= -1e-9 and l1 + l2 <= 1 + 1e-9


def test_projection_matches_concave_hull(orc):
    g = np.random.default_rng(6)
    nK, r = 6, 4
    coarse = g.integers(0, 8, size=nK * nK).astype(np.uint32)
    n = (nK - 1) * r + 1
    p = orc.Problem((n, n), (-1, -1), (1, 1), [[1.0, 0.0]], np.zeros(n * n), 0.1)
    got = orc.project(p, (r, r), coarse)
    assert (got == _con_2d(nK, r, coarse)).all()
    # coarse nodes map exactly
    assert (got.reshape(n, n)[::r, ::r].reshape(-1) == coarse).all()


def test_projection_3d_periodic(orc):
    """Kuhn tetrahedra: a fine node inside a coarse cell whose 8 corners all
    carry bit k carries bit k; a node on a coarse edge needs only the edge's
    two end points; theta wraps."""
    nKx, r = 4, 2
    nKt, rt = 3, 2
    n = ((nKx - 1) * r + 1, (nKx - 1) * r + 1, nKt * rt)
    coarse = np.zeros((nKt, nKx, nKx), dtype=np.uint32)
    coarse[...] = 1
    coarse[0, 0, 0] = 0
    p = orc.Problem(n, (0, 0, 0), (1, 1, 2 * np.pi), [[0.0]], np.zeros(int(np.prod(n))), 0.1,
                    dyn=1, periodic=(0, 0, 1))
    fine = orc.project(p, (r, r, rt), coarse.reshape(-1)).reshape(n[2], n[1], n[0])
    assert fine[0, 0, 0] == 0                 # the unlabelled coarse node
    assert fine[0, 0, 1] == 0                 # on the edge to it
    assert fine[0, 2, 2] == 1                 # a labelled coarse node
    assert fine[1, 1, 1] == 0                 # interior of a cell touching it
    assert fine[3, 3, 3] == 1                 # interior of a fully labelled cell
    assert fine[5, 3, 3] == 1                 # the wrapped last layer (theta -> 0)
    assert fine[5, 0, 0] == 0                 # wrapped edge ending at the unlabelled node
    assert fine[5, 0, 1] == 1                 # wrapped diagonal edge that avoids it


# --------------------------------------------------------------------------
# Adjoint: central finite differences with the policy frozen

def _c5_small(n=21, A=16):
    X, Y = S.mesh2(n, n)
    g = np.random.default_rng(7)
    th = 0.3 * np.sin(2.1 * X + 0.7) * np.cos(1.3 * Y - 0.2) + 0.1 * g.normal(size=X.shape)
    cen = np.array([[-0.5, -0.4], [0.5, 0.45]])
    lab = S.disk_labels(X, Y, cen, 0.2)
    pts = g.uniform(-0.9, 0.9, size=(64, 2))
    return X, Y, th, lab, pts


def test_adjoint_matches_finite_differences(orc):
    n, A = 21, 16
    X, Y, th, lab, pts = _c5_small(n, A)
    ctr = S.circle_controls(A)
    h = 2.0 / (n - 1)

    def prob(theta, cost=None):
        return orc.Problem((n, n), (-1, -1), (1, 1), ctr, lab, h, speed=np.exp(theta),
                           cost=cost)

    def loss(theta, cost=None):
        p = prob(theta, cost)
        V, _, _ = orc.solve(p, tol=1e-15, max_iters=200000)
        vals, _ = orc.points(p, V, pts, with_grad=False)
        pol, _ = orc.policy(p, V)
        return vals.mean(), pol

    p = prob(th)
    V, _, _ = orc.solve(p, tol=1e-15, max_iters=200000)
    pol, _ = orc.policy(p, V)
    _, gV = orc.points(p, V, pts)
    lam, it, r = orc.adjoint(p, pol, gV, tol=1e-15)
    gt, gc = orc.grad(p, V, pol, lam)
    g = np.random.default_rng(8)
    free = np.nonzero(lab.reshape(-1) == 0)[0]
    idx = g.choice(free, 16, replace=False)
    eps = 1e-6
    checked = 0
    for i in idx:
        tp = th.reshape(-1).copy()
        tm = tp.copy()
        tp[i] += eps
        tm[i] -= eps
        Lp, pp = loss(tp.reshape(n, n))
        Lm, pm = loss(tm.reshape(n, n))
        if (pp != pol).any() or (pm != pol).any():
            continue  # kink: the policy changes inside the stencil
        fd = (Lp - Lm) / (2 * eps)
        assert abs(fd - gt[i]) <= 1e-6 * max(1e-3, abs(gt[i])) + 1e-9, (i, fd, gt[i])
        checked += 1
    assert checked >= 12
    # cost field: L is affine in l with the policy frozen
    cost = np.ones(n * n)
    for i in idx[:6]:
        cp = cost.copy()
        cp[i] += 1e-3
        Lp, pp = loss(th, cp)
        L0, _ = loss(th, cost)
        if (pp != pol).any():
            continue
        assert abs((Lp - L0) / 1e-3 - gc[i]) < 1e-8 + 1e-6 * abs(gc[i])


def _q1_gradient(shape, spacing, idx, off):
    """d/dy of the bilinear interpolant at the foot x_idx + off, as
    [(flat, d weight / dy_x, d weight / dy_y)], in the cell the foot rule
    picks (the last cell on the upper face)."""
    cells = []
    for d in range(2):
        gd = min(max(idx[d] + off[d] / spacing[d], 0.0), shape[d] - 1.0)
        c = min(max(int(math.floor(gd)), 0), shape[d] - 2)
        cells.append((c, gd - c))
    (cx, tx), (cy, ty) = cells
    out = []
    for bx, by in itertools.product((0, 1), repeat=2):
        wx = tx if bx else 1.0 - tx
        wy = ty if by else 1.0 - ty
        sx = 1.0 if bx else -1.0
        sy = 1.0 if by else -1.0
        out.append((_grid_index(shape, (cx + bx, cy + by)), sx * wy / spacing[0],
                    sy * wx / spacing[1]))
    return out


@pytest.mark.parametrize("variant", ["speed", "current_cost", "implicit"])
def test_adjoint_tangent_linear_dot_product(orc, variant):
    """The adjoint against the tangent-linear model (exact linear solves, no
    oracle code): with the optimal policy frozen, a perturbation d of
    theta = log s moves V by dV solving (I - beta P) dV = beta c d, where c_i
    is the derivative of I[V] at the foot along h s_i a_pi(i).  The loss
    derivative g . dV must equal (dL/dtheta) . d to rounding, for several
    random directions; and dV agrees with central differences of full oracle
    solves along a smooth direction.  Variants: speed only; with a current,
    a cost field and lambda = 0.7 (the foot moves with the current, the
    derivative does not); with the implicit step weights 1/(1 + lambda h)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    n, A = 21, 16
    X, Y, th, lab, pts = _c5_small(n, A)
    lab = lab.reshape(-1)
    ctr = S.circle_controls(A)
    h = dx = 2.0 / (n - 1)
    s = np.exp(th.reshape(-1))
    g0 = np.random.default_rng(23)
    cur = S.current_field(g0, X, Y, cmax=0.3).reshape(-1, 2) if variant == "current_cost" \
        else np.zeros((n * n, 2))
    cost = g0.uniform(0.5, 2.0, n * n) if variant == "current_cost" else np.ones(n * n)
    lam_ = 0.7 if variant == "current_cost" else 1.0
    implicit = variant == "implicit"
    kw = dict(lam=lam_, weights=int(implicit))
    if variant == "current_cost":
        kw.update(current=cur, cost=cost)

    def prob(theta):
        return orc.Problem((n, n), (-1, -1), (1, 1), ctr, lab, h, speed=np.exp(theta), **kw)

    p = prob(th.reshape(-1))
    V, _, _ = orc.solve(p, tol=1e-15, max_iters=200000)
    pol, _ = orc.policy(p, V)
    _, gV = orc.points(p, V, pts)
    lam, _, _ = orc.adjoint(p, pol, gV, tol=1e-15)
    gt, _ = orc.grad(p, V, pol, lam)
    feet = [[h * (s[i] * ctr[j] + cur[i]) for j in range(A)] for i in range(n * n)]
    R, b, free, beta = _transitions((n, n), (dx, dx), (0, 0), lab, feet, cost, lam_, h,
                                    1.0, implicit=implicit)
    F = len(free)
    ar = np.arange(F)
    # the oracle's policy is optimal for the independently built problem
    Q = b + beta * (R @ V[free]).reshape(F, A)
    assert np.abs(Q[ar, pol[free]] - Q.min(axis=1)).max() < 1e-12
    assert np.abs(Q[ar, pol[free]] - V[free]).max() < 1e-12
    c = np.zeros(F)
    inside = np.zeros(F, dtype=bool)
    for k, i in enumerate(free):
        idx = (i % n, i // n)
        off = feet[i][pol[i]]
        if _stencil((n, n), (dx, dx), (0, 0), idx, off) is None:
            continue
        inside[k] = True
        direc = h * s[i] * ctr[pol[i]]
        for flat, gx, gy in _q1_gradient((n, n), (dx, dx), idx, off):
            c[k] += V[flat] * (gx * direc[0] + gy * direc[1])
    assert inside.sum() > 0.9 * F
    M = (sp.identity(F, format="csr") - beta * R[ar * A + pol[free]]).tocsc()
    lu = spl.splu(M)
    g = np.random.default_rng(17)
    for _ in range(4):
        d = np.zeros(n * n)
        d[free] = g.normal(size=F)
        dV = lu.solve(beta * c * d[free])
        lhs = gV[free] @ dV
        rhs = gt @ d
        assert abs(lhs - rhs) <= 1e-10 * (np.abs(gt) @ np.abs(d)), (lhs, rhs)
    # tangent-linear model against central differences along a smooth field
    d = np.where(lab == 0, (np.sin(1.7 * X + 0.4) * np.cos(0.9 * Y)).reshape(-1), 0.0)
    dV = lu.solve(beta * c * d[free])
    eps = 1e-6
    Vp, _, _ = orc.solve(prob(th.reshape(-1) + eps * d), tol=1e-15, max_iters=200000)
    Vm, _, _ = orc.solve(prob(th.reshape(-1) - eps * d), tol=1e-15, max_iters=200000)
    fd = (Vp[free] - Vm[free]) / (2 * eps)
    assert np.abs(fd - dV).max() <= 1e-5 * np.abs(dV).max()


def test_points_loss_gradient_is_interpolation_weights(orc):
    n = 9
    p = orc.Problem((n, n), (-1, -1), (1, 1), [[1.0, 0.0]], np.zeros(n * n), 0.1)
    g = np.random.default_rng(9)
    V = g.normal(size=n * n)
    pts = g.uniform(-1, 1, size=(5, 2))
    vals, gr = orc.points(p, V, pts)
    # L is linear in V: L(V) = gr . V
    assert abs(vals.mean() - gr @ V) < 1e-12
    assert abs(gr.sum() - 1.0) < 1e-12


def test_tie_influence_is_the_closure_of_the_seeds(orc):
    """The non-unique set used by the full-size gradient comparison: it holds
    every near-tied node, is closed under "corners of the chosen foot", and
    holds nothing else (each member is a seed or a corner of a member)."""
    n, A = 25, 16
    X, Y, th, lab, pts = _c5_small(n, A)
    h = 2.0 / (n - 1)
    p = orc.Problem((n, n), (-1, -1), (1, 1), S.circle_controls(A), lab, h, speed=np.exp(th))
    V, _, _ = orc.solve(p, tol=1e-14)
    pol, _ = orc.policy(p, V)
    eps = 2e-3
    out = orc.tie_influence(p, V, pol, eps=eps, face_eps=-1.0)
    N = n * n
    xs = np.linspace(-1, 1, n)
    ctr = S.circle_controls(A)
    s = np.exp(th).reshape(-1)

    def corners(i, j):
        iy, ix = divmod(i, n)
        y = np.array([xs[ix], xs[iy]]) + h * s[i] * ctr[j]
        if np.any(y < -1 - 1e-9) or np.any(y > 1 + 1e-9):
            return None, None
        g = np.clip((y + 1) / h, 0, n - 1)
        c = np.minimum(np.floor(g).astype(int), n - 2)
        t = g - c
        ids, ws = [], []
        for dy in (0, 1):
            for dx in (0, 1):
                ids.append((c[1] + dy) * n + c[0] + dx)
                ws.append((t[0] if dx else 1 - t[0]) * (t[1] if dy else 1 - t[1]))
        return ids, ws

    seeds = np.zeros(N, bool)
    for i in range(N):
        if pol[i] < 0 or lab.reshape(-1)[i] != 0:
            continue
        q = []
        for j in range(A):
            ids, ws = corners(i, j)
            q.append(1.0 if ids is None else sum(w * V[k] for k, w in zip(ids, ws)))
        q = np.sort(q)
        seeds[i] = q[1] - q[0] <= eps
    assert seeds.any() and not out.all()
    assert np.array_equal(orc.tie_influence(p, V, pol, eps=eps, face_eps=-1.0, closure=False),
                          seeds)
    assert np.all(out[seeds])
    reached = seeds.copy()
    for i in np.nonzero(out)[0]:
        if pol[i] < 0 or lab.reshape(-1)[i] != 0:
            continue
        ids, ws = corners(i, pol[i])
        if ids is None:
            continue
        for k, w in zip(ids, ws):
            if w > 0:
                assert out[k]
                reached[k] = True
    assert np.array_equal(reached, out)


def test_vdp_decomposition_keeps_the_error(orc):
    """Table 5 (Sec. 5, Van der Pol): the ISA error against a finer reference
    equals the original problem's error for 2, 4 and 8 cake slices, and both
    fall as the grid is refined.  The reference is the oracle on a 201^2
    grid (the paper uses 400^2); the grids are nested, so errors are taken
    at common nodes.  The paper's absolute numbers depend on its unstated
    control sampling and time step, so the magnitude is only checked loosely."""
    import json
    gold = json.load(open(os.path.join(GOLDEN, "paper_table5_vdp.json")))
    assert all(gold["rows"][k] == gold["rows"]["original"]
               for k in ("2-subsets", "4-subsets", "8-subsets"))
    ref = S.vdp(n=201, slices=1)
    Vr, _, _ = orc.solve(_vdp_problem(orc, ref), tol=1e-10, nthreads=orc.max_threads())
    Vr = Vr.reshape(201, 201)
    errs = {}
    for n in (51, 101):
        sub = Vr[:: 200 // (n - 1), :: 200 // (n - 1)].reshape(-1)
        V0, _, _ = orc.solve(_vdp_problem(orc, S.vdp(n=n, slices=1)), tol=1e-10,
                             nthreads=orc.max_threads())
        e0 = np.abs(V0 - sub)
        errs[n] = (e0.max(), e0.mean())
        if n != 101:
            continue
        for slices in (2, 4, 8):
            d = S.vdp(n=n, slices=slices)
            po = _vdp_problem(orc, d)
            _, lab, _ = orc.ra(po, (5, 5), 0.1, tol=1e-10, nthreads=orc.max_threads())
            fm = orc.project(po, (5, 5), lab)
            Vb, unc, _, _ = orc.isa(po, fm, tol=1e-10, nthreads=orc.max_threads())
            assert unc == 0
            e = np.abs(Vb - sub)
            assert abs(e.max() - e0.max()) <= 1e-3 * e0.max()
            assert abs(e.mean() - e0.mean()) <= 2e-2 * e0.mean()
            # the sub-domains are proper subsets
            assert all(((fm >> k) & 1).mean() < 1.0 for k in range(slices))
    assert errs[101][0] < errs[51][0] and errs[101][1] < errs[51][1]
    # the same order of magnitude as the paper's 100^2 row
    assert 0.2 * gold["rows"]["original"][1][1] < errs[101][1] < 5 * gold["rows"]["original"][1][1]


def _vdp_problem(orc, d):
    return orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"],
                       current=d["current"], cost=d["cost"], lam=d["lam"], v_out=d["v_out"],
                       ntargets=d["ntargets"])


# --------------------------------------------------------------------------
# Games (Sec. 2, max over b of min over a; Example ex4): the second player's control b
# enters as f = D(x)(a - b) + c(x).

def test_game_with_a_silent_second_player_is_the_control_problem(orc):
    d = S.c2(n=41, A=16, ntargets=3, stride=8)
    base = dict(h=d["h"], speed=d["speed"], current=d["current"], ntargets=3)
    p = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], **base)
    g = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"],
                    controls_b=np.zeros((1, 2)), **base)
    V, _, _ = orc.solve(p, tol=1e-13)
    W, _, _ = orc.solve(g, tol=1e-13)
    assert np.array_equal(V, W)


def test_brute_force_game(orc):
    """The game's fixed point is the best over the second player's
    stationary strategies sigma of the first player's optimal value against
    sigma: V = max_sigma V_sigma, node by node (T_sigma <= T with equality
    at the maximising sigma, and both are monotone contractions).  V_sigma is
    the minimum over every first-player policy of the dense linear solve."""
    g = np.random.default_rng(11)
    shape = (3, 2)
    lo, hi = (0.0, 0.0), (2.0, 1.0)
    N = 6
    target = np.zeros(N, dtype=np.int32)
    target[0] = 1
    angA = 0.2 + 2 * np.pi / 3 * np.arange(3)
    A = np.stack([np.cos(angA), np.sin(angA)], 1)
    angB = 1.0 + np.pi * np.arange(2)
    B = 0.5 * np.stack([np.cos(angB), np.sin(angB)], 1)
    D = g.uniform(0.5, 1.5, (N, 2))
    cur = g.uniform(-0.2, 0.2, (N, 2))
    cost = g.uniform(0.5, 2.0, N)
    lam, h, v_out = 0.8, 0.7, 3.0
    free = [i for i in range(N) if target[i] == 0]
    best = None
    for sigma in itertools.product(range(len(B)), repeat=len(free)):
        sg = dict(zip(free, sigma))
        feet = [[h * (D[i] * (A[j] - B[sg.get(i, 0)]) + cur[i]) for j in range(len(A))]
                for i in range(N)]
        Vs = _brute_force(shape, (1.0, 1.0), (0, 0), target, feet, cost, lam, h, v_out)
        best = Vs if best is None else np.maximum(best, Vs)
    p = orc.Problem(shape, lo, hi, A, target, h=h, lam=lam, current=cur, cost=cost, v_out=v_out,
                    scale=D, controls_b=B)
    V, _, _ = orc.solve(p, tol=1e-15, max_iters=100000)
    assert np.abs(V - best).max() < 1e-12


def test_pursuit_evasion_strip_exact(orc):
    """f = D (a - b), D = diag(d, 1), a in {+-e1, +-e2}, b in 1/2 {+-e1, +-e2},
    target the strip |x1| <= 0.2, y periodic (V does not depend on y).  Away
    from the strip the evader's best answer is b = -e1/2 (moving away), the
    pursuer's a = -e1, so the foot lies o = d h / (2 dx) cells closer and the
    scheme reduces to the recursion V_i = (beta o V_{i-1} + gamma) /
    (1 - beta (1 - o)) from V = 0 on the strip (lambda = 1, l = 1): every
    other pair of answers gives a smaller value."""
    n, ny, d = 41, 4, 1.3
    x = np.linspace(-1, 1, n)
    h = 2.0 / (n - 1)
    E = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [0.0, -1.0]])
    lab = np.tile((np.abs(x) <= 0.2 + 1e-12).astype(np.uint8), (ny, 1))
    D = np.tile([d, 1.0], (n * ny, 1))
    p = orc.Problem((n, ny), (-1.0, 0.0), (1.0, 1.0), E, lab, h, periodic=(0, 1), scale=D,
                    controls_b=0.5 * E)
    V, _, _ = orc.solve(p, tol=1e-15, max_iters=100000)
    V = V.reshape(ny, n)
    beta = math.exp(-h)
    gam = 1 - beta
    o = 0.5 * d
    ref = np.zeros(n)
    c = n // 2
    for i in range(c, n):
        if abs(x[i]) > 0.2 + 1e-12:
            ref[i] = (beta * o * ref[i - 1] + gam) / (1 - beta * (1 - o))
    ref[:c] = ref[c + 1:][::-1]
    assert np.abs(V - ref[None, :]).max() < 1e-12


def test_scale_field_with_equal_axes_is_the_speed_field(orc):
    """f = diag(D) a with D = (s, s) is f = s a: the full solve and the
    coarse auxiliary solves of RA (which sample every node field at the
    coarse stride) agree exactly."""
    d = S.c2(n=49, A=16, ntargets=3, stride=8)
    kw = dict(h=d["h"], current=d["current"], ntargets=3)
    p = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], speed=d["speed"], **kw)
    D = np.repeat(np.asarray(d["speed"]).reshape(-1, 1), 2, axis=1)
    q = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], scale=D, **kw)
    assert np.array_equal(orc.solve(p, tol=1e-12)[0], orc.solve(q, tol=1e-12)[0])
    Va, la, _ = orc.ra(p, (8, 8), 0.1, tol=1e-12)
    Vb, lb, _ = orc.ra(q, (8, 8), 0.1, tol=1e-12)
    assert np.array_equal(Va, Vb) and np.array_equal(la, lb)


def test_c5_finite_difference_golden_pins_the_oracle_adjoint():
    """The stored FP64 central differences of the 1025^2 adjoint workload
    (tests/golden/c5_fd_1025.json, written by make_c5_fd_golden.py from the
    oracle's forward solves alone) pin the oracle's adjoint gradient, stored
    beside them, at full size: the gradient is the transposed fixed point
    with the policy frozen, the differences are of the loss itself.  Every
    entry whose quotient is at least 1e-3 of the largest agrees within 1e-3
    relative (measured <= 4.5e-4, the smallest such quotients being at the
    differences' resolution of ~1e-12); the rest within 1e-5 of the largest
    in absolute terms.  Entries at a kink would be excluded (none occur)."""
    with open(os.path.join(GOLDEN, "c5_fd_1025.json")) as f:
        gold = json.load(f)
    assert gold["n"] == 1025 and len(gold["entries"]) == 64 and "eps=1e-05" in gold["method"]
    scale = max(abs(e["fd"]) for e in gold["entries"])
    resolved = 0
    for e in gold["entries"]:
        assert 0 <= e["index"] < 1025 * 1025
        if e["kink"]:
            continue
        err = abs(e["adjoint"] - e["fd"])
        if abs(e["fd"]) >= 1e-3 * scale:
            assert err <= 1e-3 * abs(e["fd"]), e
            resolved += 1
        else:
            assert err <= 1e-5 * scale, e
    assert resolved >= 48
    assert sum(e["kink"] for e in gold["entries"]) == gold["kinks"]
