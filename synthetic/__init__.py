"""Seeded synthetic inputs shaped like the paper's workloads.

This module builds problem DATA only: grids, control sets, target disks,
speed/current fields, log-speed fields and loss points.  It holds none of the
method's arithmetic (no operator, interpolation, iteration or labelling), so
that the oracle and the CUDA path can both consume it without sharing code.

Every stream is drawn from numpy's default_rng seeded with
SeedSequence(20140513, spawn_key=(purpose, index)).  Values are generated in
FP64; the CUDA path receives them cast to FP32 and the oracle receives the
same FP32-rounded values widened back to FP64, so both solve the identical
discrete problem.

The workloads (box [-1,1]^2, Kruzhkov lambda = 1, h = dx, disk targets) follow
the distance-function example of Sec. 4.1 of the paper and the five problem
families this library is benchmarked on:
  c1  2D minimum time, f = a, 32 unit controls, 101^2, 4 disks of radius 0.1
  c2  2D Zermelo navigation f = s a + c, 64 controls, 1025^2, 16 disks
  c3  3D Dubins car (x, y, theta), 256 x 256 x 128, u in {-1, 0, 1}, 8 disks
  c4  batch of 512 square problems, sides ~ U{64..512}, 1-8 disks, 32 controls
  c5  2D f = exp(theta) a on 1025^2, theta a Gaussian random field, 4 disks,
      4096 loss points
  vdp the Van der Pol oscillator of Sec. 5 (Example ex3) as a target problem:
      running cost |x|, target B(0, 0.2) split into angular "cake slices"
"""
from __future__ import annotations

import math

import numpy as np

SEED = 20140513
PURPOSE = {"targets": 1, "speed": 2, "current": 3, "theta": 4, "points": 5,
           "batch": 6, "fd": 7, "misc": 8}


def rng(purpose: str, index: int = 0) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(SEED, spawn_key=(PURPOSE[purpose], index)))


def f32(a):
    """Round to FP32 and widen back: the exact values both solvers see."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def axis(n: int, lo: float, hi: float, periodic: bool = False) -> np.ndarray:
    if periodic:
        return lo + (hi - lo) * np.arange(n) / n
    return lo + (hi - lo) * np.arange(n) / (n - 1)


def mesh2(nx: int, ny: int, lo=(-1.0, -1.0), hi=(1.0, 1.0)):
    """Node coordinates (X, Y), arrays shaped (ny, nx) with x fastest."""
    x = axis(nx, lo[0], hi[0])
    y = axis(ny, lo[1], hi[1])
    return np.meshgrid(x, y, indexing="xy")


def circle_controls(A: int) -> np.ndarray:
    """A unit vectors at angles 2 pi j / A (the discrete control set of Sec. 3).
    For even A the second half is the exact negation of the first (a_{j + A/2}
    = -a_j, as on the circle; cos and sin of the shifted angles would differ
    from it by rounding in components near zero)."""
    t = 2.0 * np.pi * np.arange(A) / A
    a = np.stack([np.cos(t), np.sin(t)], axis=1)
    if A % 2 == 0:
        a[A // 2:] = -a[: A // 2]
    return a


def king_controls() -> np.ndarray:
    """The 8 'king move' controls (+-1,0), (0,+-1), (+-1,+-1)."""
    return np.array([[1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]],
                    dtype=np.float64)


def axis_controls() -> np.ndarray:
    return np.array([[1, 0], [0, 1], [-1, 0], [0, -1]], dtype=np.float64)


def disk_centers(g: np.random.Generator, count: int, radius: float = 0.1, min_sep: float = 0.3,
                 lo: float = -0.85, hi: float = 0.85) -> np.ndarray:
    """Centres uniform in [lo, hi]^2, rejected until pairwise distance >= min_sep."""
    out = []
    tries = 0
    while len(out) < count:
        c = g.uniform(lo, hi, size=2)
        tries += 1
        if all(np.hypot(*(c - o)) >= min_sep for o in out):
            out.append(c)
        if tries > 100000:
            raise RuntimeError("cannot place disks")
    return np.array(out).reshape(count, 2)


def disk_labels(X: np.ndarray, Y: np.ndarray, centers: np.ndarray, radius: float) -> np.ndarray:
    """Label k (1-based) on nodes inside closed disk k, 0 elsewhere (uint8)."""
    lab = np.zeros(X.shape, dtype=np.uint8)
    for k, (cx, cy) in enumerate(centers):
        inside = (X - cx) ** 2 + (Y - cy) ** 2 <= radius * radius
        lab[inside & (lab == 0)] = k + 1
    return lab


def _modes(g: np.random.Generator, m: int = 8, kmax: float = 4 * np.pi):
    ang = g.uniform(0, 2 * np.pi, size=m)
    mag = g.uniform(0.5, kmax, size=m)
    k = np.stack([mag * np.cos(ang), mag * np.sin(ang)], axis=1)
    amp = g.normal(size=m)
    ph = g.uniform(0, 2 * np.pi, size=m)
    return k, amp, ph


def speed_field(g: np.random.Generator, X: np.ndarray, Y: np.ndarray, smin=0.5, smax=1.5):
    """s = smin + (smax-smin) (z - min z)/(max z - min z), z a sum of 8 random sines."""
    k, amp, ph = _modes(g)
    z = np.zeros_like(X)
    for m in range(len(amp)):
        z += amp[m] * np.sin(k[m, 0] * X + k[m, 1] * Y + ph[m])
    return smin + (smax - smin) * (z - z.min()) / (z.max() - z.min())


def current_field(g: np.random.Generator, X: np.ndarray, Y: np.ndarray, cmax=0.4):
    """c = rot(psi) = (d psi/dy, -d psi/dx), psi a sum of 8 random sines
    (differentiated analytically, so exactly divergence-free), scaled so that
    max over nodes of |c| = cmax.  Returns (ny, nx, 2)."""
    k, amp, ph = _modes(g)
    cx = np.zeros_like(X)
    cy = np.zeros_like(X)
    for m in range(len(amp)):
        arg = k[m, 0] * X + k[m, 1] * Y + ph[m]
        cx += amp[m] * k[m, 1] * np.cos(arg)
        cy -= amp[m] * k[m, 0] * np.cos(arg)
    mag = np.sqrt(cx * cx + cy * cy).max()
    return np.stack([cx, cy], axis=-1) * (cmax / mag)


def grf_logspeed(g: np.random.Generator, n: int, corr: float = 0.1, lo=math.log(0.5),
                 hi=math.log(1.5)):
    """theta: white noise filtered by a Gaussian kernel of correlation length
    `corr` (domain units on [-1,1]^2) via FFT, mapped affinely to [lo, hi]."""
    w = g.normal(size=(n, n))
    dx = 2.0 / (n - 1)
    kf = np.fft.fftfreq(n, d=dx) * 2 * np.pi
    KX, KY = np.meshgrid(kf, kf, indexing="xy")
    filt = np.exp(-0.5 * (KX ** 2 + KY ** 2) * corr ** 2)
    z = np.real(np.fft.ifft2(np.fft.fft2(w) * filt))
    return lo + (hi - lo) * (z - z.min()) / (z.max() - z.min())


def uniform_points(g: np.random.Generator, P: int, lo=-1.0, hi=1.0) -> np.ndarray:
    return g.uniform(lo, hi, size=(P, 2))


# ---------------------------------------------------------------------------
# Workload builders.  Each returns a dict with:
#   shape (nx, ny[, nz]), lo, hi, periodic, dyn (0 speed/current, 1 Dubins),
#   controls [A, cdim], labels (uint8, (ny, nx) or (nz, ny, nx)), ntargets,
#   speed (or None), current (or None), log_speed (or None), h, lam, v_out,
#   stride (coarse stride of the reconstruction), and for c5 the loss points.
# All float arrays are already FP32-rounded (see f32).

def _base2(n, A, ntargets, index, with_speed, with_current, radius=0.1, stride=16,
           nx=None):
    nx = n if nx is None else nx
    X, Y = mesh2(nx, n)
    cen = disk_centers(rng("targets", index), ntargets, radius)
    lab = disk_labels(X, Y, cen, radius)
    dx = 2.0 / (nx - 1)
    return dict(
        shape=(nx, n), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
        controls=f32(circle_controls(A)), labels=lab, ntargets=ntargets, centers=cen,
        radius=radius,
        speed=f32(speed_field(rng("speed", index), X, Y)) if with_speed else None,
        current=f32(current_field(rng("current", index), X, Y)) if with_current else None,
        log_speed=None, h=dx, lam=1.0, v_out=1.0, stride=(stride, stride))


def c1(n=101, A=32, ntargets=4):
    """2D minimum time, f = a, h = dx = 0.02 at n = 101."""
    return _base2(n, A, ntargets, 1, False, False, stride=10 if (n - 1) % 10 == 0 else 1)


def c2(n=1025, A=64, ntargets=16, stride=16):
    """2D Zermelo navigation f = s a + c, s in [0.5, 1.5], |c| <= 0.4."""
    if (n - 1) % stride:
        stride = 1
    return _base2(n, A, ntargets, 2, True, True, stride=stride)


def c3(nxy=256, nth=128, ntargets=8, stride=(5, 5, 8)):
    """3D Dubins car (x, y, theta): f = (cos th, sin th, u), u in {-1, 0, 1}.
    (x, y) in [-1, 1]^2, theta periodic on [-pi, pi), h = dx."""
    X, Y = mesh2(nxy, nxy)
    cen = disk_centers(rng("targets", 3), ntargets, 0.1)
    lab2 = disk_labels(X, Y, cen, 0.1)
    lab = np.broadcast_to(lab2, (nth, nxy, nxy)).copy()
    dx = 2.0 / (nxy - 1)
    return dict(
        shape=(nxy, nxy, nth), lo=(-1.0, -1.0, -np.pi), hi=(1.0, 1.0, np.pi),
        periodic=(0, 0, 1), dyn=1, controls=np.array([[-1.0], [0.0], [1.0]]), labels=lab,
        ntargets=ntargets, centers=cen, radius=0.1, speed=None, current=None, log_speed=None,
        dubins_v=1.0, h=dx, lam=1.0, v_out=1.0, stride=stride)


def c4_sides(count=512, lo=64, hi=512):
    return rng("batch", 0).integers(lo, hi + 1, size=count)


def c4_problem(i: int, n: int, A: int = 32):
    """Problem i of the batch: n x n on [-1,1]^2, own speed field, c = 0,
    1..8 disk targets."""
    g = rng("batch", 1 + i)
    nt = int(g.integers(1, 9))
    X, Y = mesh2(n, n)
    cen = disk_centers(g, nt, 0.1)
    lab = disk_labels(X, Y, cen, 0.1)
    return dict(
        shape=(n, n), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
        controls=f32(circle_controls(A)), labels=lab, ntargets=nt, centers=cen, radius=0.1,
        speed=f32(speed_field(g, X, Y)), current=None, log_speed=None, h=2.0 / (n - 1),
        lam=1.0, v_out=1.0, stride=(1, 1))


def c5(n=1025, A=32, ntargets=4, P=4096):
    """2D f = exp(theta) a, theta a smooth Gaussian random field in
    [ln 0.5, ln 1.5]; loss = mean of v at P uniform points."""
    d = _base2(n, A, ntargets, 5, False, False, stride=16 if (n - 1) % 16 == 0 else 1)
    th = f32(grf_logspeed(rng("theta", 5), n))
    d["log_speed"] = th
    d["speed"] = None
    d["points"] = f32(uniform_points(rng("points", 5), P))
    return d


def vdp(n=101, A=21, slices=4, rho=0.2, stride=None):
    """Van der Pol oscillator as a target problem (Sec. 5, Example ex3):
    f(x, a) = (x2, (1 - x1^2) x2 - x1 + a) on (-1, 1)^2 with a in [-1, 1]
    sampled at A equispaced points, running cost l(x) = |x|, lambda = 1,
    g = 0, target the closed disk B(0, rho) split into `slices` equal angular
    sectors (label k + 1 for angles in [2 pi k / slices, 2 pi (k + 1) / slices)),
    h = dx.  The state-dependent part of f is the node field `current`, the
    control part the control vectors (0, a_j).  Trajectories that must leave
    the box take value_out = sup l / lambda = sqrt(2), the discounted cost of
    never arriving bounded from above."""
    X, Y = mesh2(n, n)
    r = np.hypot(X, Y)
    ang = np.mod(np.arctan2(Y, X), 2 * np.pi)
    k = np.minimum((ang / (2 * np.pi / slices)).astype(np.int64), slices - 1) + 1
    lab = np.where(r <= rho + 1e-12, k, 0).astype(np.uint8)
    drift = np.stack([Y, (1.0 - X * X) * Y - X], axis=-1)
    a = np.linspace(-1.0, 1.0, A)
    controls = np.stack([np.zeros_like(a), a], axis=-1)
    if stride is None:
        stride = next((s for s in (16, 10, 8, 5, 4, 2) if (n - 1) % s == 0), 1)
    return dict(
        shape=(n, n), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
        controls=f32(controls), labels=lab, ntargets=slices, speed=None,
        current=f32(drift), cost=f32(r), log_speed=None, h=2.0 / (n - 1), lam=1.0,
        v_out=float(np.float32(math.sqrt(2.0))), stride=(stride, stride))


def pursuit_evasion(n=129, A=16, B=8, slices=4, rho=0.2, stride=None):
    """The pursuit-evasion game of Sec. 5 (Example ex4): f(x, a, b) =
    D(x) (a - b) with D(x) = diag(x2 + 1, 1), the pursuer's a on the unit
    circle (A directions), the evader's b on the circle of radius 1/2 (B
    directions), running cost l(x) = x1^2 + 0.1 (the printed "x1 + 0.1" is
    negative on part of the box, against hypothesis H0; the Hamiltonian the
    example states carries x1^2 + 0.1), lambda = 1, capture on the closed
    disk B(0, rho) split into `slices` angular sectors, h = dx, value_out =
    sup l / lambda = 1.1."""
    X, Y = mesh2(n, n)
    r = np.hypot(X, Y)
    ang = np.mod(np.arctan2(Y, X), 2 * np.pi)
    k = np.minimum((ang / (2 * np.pi / slices)).astype(np.int64), slices - 1) + 1
    lab = np.where(r <= rho + 1e-12, k, 0).astype(np.uint8)
    scale = np.stack([Y + 1.0, np.ones_like(Y)], axis=-1)
    ta = 2 * np.pi * np.arange(A) / A
    tb = 2 * np.pi * (np.arange(B) + 0.5) / B
    if stride is None:
        stride = next((s for s in (16, 10, 8, 5, 4, 2) if (n - 1) % s == 0), 1)
    return dict(
        shape=(n, n), lo=(-1.0, -1.0), hi=(1.0, 1.0), periodic=(0, 0), dyn=0,
        controls=f32(np.stack([np.cos(ta), np.sin(ta)], -1)),
        controls_b=f32(0.5 * np.stack([np.cos(tb), np.sin(tb)], -1)),
        labels=lab, ntargets=slices, speed=None, current=None, scale=f32(scale),
        cost=f32(X * X + 0.1), log_speed=None, h=2.0 / (n - 1), lam=1.0,
        v_out=float(np.float32(1.1)), stride=(stride, stride))
