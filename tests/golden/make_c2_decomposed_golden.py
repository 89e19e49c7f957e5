"""Writes c2_decomposed_1025.json: the FP64 oracle's reconstruction and
decomposed solve of the 1025 x 1025 Zermelo workload (64 controls, 16 disk
targets, coarse stride 16) with the threshold the benchmark applies, and its
full-domain solve.  Every value comes from oracle/ on the seeded inputs of
synthetic/; nothing here reads the CUDA library.

- RA (Sec. 3): the 16 auxiliary solves on the 65 x 65 coarse grid, V = min_k
  V_k, the threshold delta = 2 M dx_K of eq. (rep) with M the largest
  discrete gradient norm of V on the coarse grid (reading R5, C = 0), and the
  coarse labels.
- ISA steps 2-4 (Sec. 4): the projection through Con, the 16 restricted
  fine solves and the min-assembly Vbar.
- The full-domain solve V of eq. (SL).

Stored: delta and M; per-sub-domain label and mask sizes; the count of label
decisions within 1e-4 of the threshold; a digest of the fine mask (so that a
test can confirm it rebuilt the same decomposition); max |Vbar - V| and where
it occurs; and Vbar and V at 2048 seeded nodes plus the 256 nodes where they
differ most.  The solves stop at ||V^{n+1} - V^n||_inf <= 1e-10.

Usage: python tests/golden/make_c2_decomposed_golden.py [--n 1025] [--stride 16]
(about 15 minutes on 8 cores at the full size).
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
import synthetic as S  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1025)
    ap.add_argument("--stride", type=int, default=16)
    ap.add_argument("--tol", type=float, default=1e-10)
    args = ap.parse_args()
    d = S.c2(n=args.n, stride=args.stride)
    n = args.n
    stride = d["stride"]
    p = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"],
                    speed=d["speed"], current=d["current"], ntargets=d["ntargets"])
    nt = orc.max_threads()
    t0 = time.time()
    Vaux, _, _ = orc.ra(p, stride, 0.0, tol=1e-11, nthreads=nt)
    delta, M = orc.delta(p, stride, Vaux)
    nk = orc.coarse_shape(p, stride)
    tgt = p.target.reshape(n, n)[::stride[1], ::stride[0]].reshape(-1)
    vmin, lab, ties = orc.label(Vaux, tgt, delta)
    near = int(sum(((np.abs(np.abs(Vaux[k] - vmin) - delta) <= 1e-4)).sum()
                   for k in range(d["ntargets"])))
    fine = orc.project(p, stride, lab)
    Vf, it_full, _ = orc.solve(p, tol=args.tol, nthreads=nt)
    Vb, unc, its, _ = orc.isa(p, fine, tol=args.tol, nthreads=nt)
    diff = np.abs(Vb - Vf)
    g = np.random.default_rng(np.random.SeedSequence(S.SEED, spawn_key=(S.PURPOSE["misc"], 1025)))
    idx = np.unique(np.concatenate([g.integers(0, p.N, 2048), np.argsort(-diff)[:256]]))
    am = int(diff.argmax())
    out = {
        "source": "oracle/ (FP64) on synthetic.c2(n=%d, stride=%d); written by "
                  "tests/golden/make_c2_decomposed_golden.py" % (n, args.stride),
        "paper": "RA steps 1-3 (Sec. 3), eq. (rep) of Prop. 3.1 with M estimated (reading R5), "
                 "ISA steps 2-4 (Sec. 4), eq. (SL)",
        "n": n, "stride": list(stride), "controls": int(d["controls"].shape[0]),
        "targets": int(d["ntargets"]), "tol": args.tol, "coarse": list(nk),
        "delta": delta, "lipschitz": M, "label_ties_1e-6": ties, "label_near_1e-4": near,
        "coarse_label_counts": [int(((lab >> k) & 1).sum()) for k in range(d["ntargets"])],
        "fine_mask_counts": [int(((fine >> k) & 1).sum()) for k in range(d["ntargets"])],
        "fine_mask_sha256": hashlib.sha256(fine.astype("<u4").tobytes()).hexdigest(),
        "uncovered": unc, "full_iterations": it_full, "isa_iterations": [int(x) for x in its],
        "max_abs_isa_minus_full": float(diff.max()), "argmax_xy": [am % n, am // n],
        "nodes_above_1e-4": int((diff > 1e-4).sum()),
        "sample_index": idx.tolist(),
        "sample_isa": [float(x) for x in Vb[idx]],
        "sample_full": [float(x) for x in Vf[idx]],
        "seconds": time.time() - t0, "threads": nt,
    }
    name = "c2_decomposed_%d.json" % n
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")
    print(name, "delta %.6f M %.5f max|Vbar - V| %.3e at %s, %d nodes above 1e-4, %.0f s"
          % (delta, M, diff.max(), out["argmax_xy"], out["nodes_above_1e-4"], out["seconds"]))


if __name__ == "__main__":
    main()
