"""Writes c5_fd_1025.json: FP64 central finite differences of the loss of the
1025 x 1025 adjoint workload (f = exp(theta) a, 32 controls, 4 disk targets,
theta a Gaussian random field; L = mean of V at 4096 seeded points) with
respect to 64 seeded non-target entries of theta, from the oracle alone.

Per entry i: theta +- eps e_i, each solved by Gauss-Seidel warm-started from
the converged V and stopped when one sweep changes V by at most 1e-15 (then
checked by one Jacobi application), and fd_i = (L(theta + eps e_i) -
L(theta - eps e_i)) / (2 eps) with eps = 1e-5.  An entry is a kink, and is
excluded from comparisons, when the optimal policy differs between the two
perturbed solutions at any node that carries adjoint mass (lambda_j > 0),
where the value is not differentiable in theta_i.  The oracle's adjoint
gradient (the transposed fixed point with the policy frozen) is stored
beside each entry.

Usage: python tests/golden/make_c5_fd_golden.py [--n 1025] [--entries 64]
[--procs 8]  (about 20 minutes on 8 cores at the full size).
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
import synthetic as S  # noqa: E402

EPS = 1e-5
TOL = 1e-15


def _problem(d, theta):
    return orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"],
                       speed=np.exp(theta), ntargets=d["ntargets"])


def _state(n):
    d = S.c5(n=n)
    th = np.asarray(d["log_speed"], dtype=np.float32).astype(np.float64).reshape(-1)
    return d, th


_G = {}


def _init(n, V):
    d, th = _state(n)
    _G.update(d=d, th=th, V=V)


def _one(i):
    d, th, V = _G["d"], _G["th"], _G["V"]
    out = []
    for sgn in (1.0, -1.0):
        t = th.copy()
        t[i] += sgn * EPS
        p = _problem(d, t)
        Vs, sweeps, r = orc.solve(p, tol=TOL, max_iters=100000, V0=V, gs=True)
        vals, _ = orc.points(p, Vs, d["points"], with_grad=False)
        pol, _ = orc.policy(p, Vs)
        out.append((float(vals.mean()), pol, sweeps, r))
    return i, out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1025)
    ap.add_argument("--entries", type=int, default=64)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    t0 = time.time()
    d, th = _state(args.n)
    p = _problem(d, th)
    nt = orc.max_threads()
    V, _, _ = orc.solve(p, tol=1e-12, nthreads=nt)
    V, _, r0 = orc.solve(p, tol=TOL, max_iters=100000, V0=V, gs=True)
    pol, _ = orc.policy(p, V, nthreads=nt)
    _, gV = orc.points(p, V, d["points"])
    lam, _, _ = orc.adjoint(p, pol, gV, tol=1e-15)
    gt, _ = orc.grad(p, V, pol, lam)
    free = np.nonzero(d["labels"].reshape(-1) == 0)[0]
    g = S.rng("fd", 5)
    idx = np.sort(g.choice(free, args.entries, replace=False))
    carrying = lam > 0
    ctx = mp.get_context("spawn")
    res = {}
    with ctx.Pool(args.procs, initializer=_init, initargs=(args.n, V)) as pool:
        for i, out in pool.imap_unordered(_one, [int(i) for i in idx]):
            res[i] = out
    entries = []
    for i in idx:
        (Lp, pp, sp, rp), (Lm, pm, sm, rm) = res[int(i)]
        kink = bool(((pp != pm) & carrying).any())
        entries.append({"index": int(i), "xy": [int(i) % args.n, int(i) // args.n],
                        "fd": (Lp - Lm) / (2 * EPS), "adjoint": float(gt[i]),
                        "lambda": float(lam[i]), "kink": kink,
                        "gs_sweeps": [int(sp), int(sm)], "residuals": [rp, rm]})
    out = {
        "source": "oracle/ (FP64) on synthetic.c5(n=%d); written by "
                  "tests/golden/make_c5_fd_golden.py" % args.n,
        "method": "central differences, eps=%g, Gauss-Seidel warm start to %g; kink = policy "
                  "change between +-eps at a node with lambda > 0" % (EPS, TOL),
        "n": args.n, "controls": int(d["controls"].shape[0]), "targets": int(d["ntargets"]),
        "points": int(len(d["points"])), "base_residual": r0,
        "kinks": int(sum(e["kink"] for e in entries)),
        "entries": entries, "seconds": time.time() - t0,
    }
    name = "c5_fd_%d.json" % args.n
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")
    ok = [e for e in entries if not e["kink"]]
    rel = max(abs(e["fd"] - e["adjoint"]) / max(abs(e["fd"]), 1e-300) for e in ok) if ok else 0.0
    print(name, "%d entries, %d kinks, max relative |fd - adjoint| %.2e, %.0f s"
          % (len(entries), out["kinks"], rel, out["seconds"]))


if __name__ == "__main__":
    main()
