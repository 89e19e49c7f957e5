#!/usr/bin/env python
"""Benchmark: node-updates/s to convergence of the decomposed solve of a
1025 x 1025 Zermelo navigation problem (64 controls, 16 disk targets,
speed in [0.5, 1.5], divergence-free current |c| <= 0.4), against the
full-domain solve on the same GPU, both at the 1e-4 L-infinity accuracy of
the stopping rule.

One step = the whole hot path: reconstruction of the independent
sub-domains on the stride-16 coarse grid (RA, Sec. 3 of Festa,
arXiv:1405.3521: 16 auxiliary solves, labels, projection) followed by the
decomposed fine solve with all 16 sub-domains in one persistent,
graph-captured launch and the min-assembly (ISA, Sec. 4).

value = full-domain-equivalent node-updates/s = (free nodes x sweeps the
full-domain solve needs) / step time, summed over ranks (weak scaling: every
rank solves its own copy).  The raw rate (node-updates actually performed /
step time) and the full-domain solve are reported beside it.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node-updates/s to convergence, decomposed+batched vs full-domain GPU at 1e-4 L∞"
UNIT = "node-updates/s"
WORKLOAD = "zermelo-1025x1025-A64-16targets"
# Algorithmic FP32 work of one control evaluation of the 2D sweep: foot (2 FMA),
# cell and fraction (2 floor + 2 sub), three lerps (6), one compare = 13.
OPS_PER_CONTROL = 13


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1025, help="grid side (default: the 1025^2 workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="zermelo", choices=["zermelo", "dubins", "batch", "adjoint", "vdp", "game"],
                    help="zermelo: the 1025^2 Zermelo problem (default, the headline line); "
                         "dubins, batch, adjoint, vdp, game: the other rows, each printing its own line")
    ap.add_argument("--small", action="store_true",
                    help="dubins / adjoint: a reduced size (126x126x64 / 257^2) for detailed "
                         "profiler captures; not a benchmark configuration")
    ap.add_argument("--profile", choices=["full", "decomposed", "ra"], default=None,
                    help="run one solve of that path (zermelo: the full solve, the reconstruction, "
                         "or the reconstruction and the decomposed solve; dubins: one step; "
                         "adjoint: the forward solve and one backward) for a profiler; prints "
                         "per-solve statistics instead of the JSON line")
    return ap.parse_args()


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def aggregate(step_ms, units_per_rank, dist=None, device="cuda"):
    """Max step time over ranks and the whole-job rate (units of all ranks
    divided by that time)."""
    if dist is None:
        return step_ms, units_per_rank / (step_ms / 1e3)
    import torch
    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units_per_rank], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return ms, float(u.item()) / (ms / 1e3)


TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "sweep2d_zermelo1025_dram_traffic.md")
KERNEL_SOURCES = ("paper_1405_3521_gb300/csrc/sweep.cu", "paper_1405_3521_gb300/csrc/hjb_internal.cuh")


ADJOINT_SOURCES = ("paper_1405_3521_gb300/csrc/adjoint.cu", "paper_1405_3521_gb300/csrc/hjb_internal.cuh")
ADJOINT_PROFILE = os.path.join(ROOT, "profiles", "adjoint1025_launch_list_traffic.md")


def kernel_sources_sha256(sources=KERNEL_SOURCES):
    """Digest of the sources a kernel is built from (default: the sweeps)."""
    import hashlib
    h = hashlib.sha256()
    for rel in sources:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def sweep_traffic(path=TRAFFIC_PROFILE, rows=None, local_iters=None):
    """DRAM bytes per sweep launch from a committed ncu summary, for the tile
    shape (`rows`) and applications per tile (`local_iters`) the timed run
    used, or None when the summary has no line for them or the kernel
    sources changed after the counters were taken.  Lines are
    `- traffic_bytes_per_launch_rows<R>_li<L>: <bytes>` and
    `- node_updates_per_launch_rows<R>_li<L>: <count>` (3D: rows 8)."""
    try:
        with open(path) as f:
            kv = dict(line.strip("- \n").split(": ", 1) for line in f
                      if line.startswith("- ") and ": " in line)
        if kv.get("sources_sha256") != kernel_sources_sha256():
            return None
        sfx = "_rows%d_li%d" % (rows or 8, local_iters or 6)
        if "traffic_bytes_per_launch" + sfx not in kv:
            return None
        out = {"bytes_per_launch": float(kv["traffic_bytes_per_launch" + sfx])}
        if "node_updates_per_launch" + sfx in kv:
            out["node_updates_per_launch"] = float(kv["node_updates_per_launch" + sfx])
        return out
    except (OSError, KeyError, ValueError):
        return None


def adjoint_traffic(path=ADJOINT_PROFILE):
    """DRAM bytes per launch of the adjoint's iteration kernels from a committed
    ncu summary (`- traffic_bytes_per_launch_<kernel>: <bytes>`), or None when
    the sources changed after the counters were taken."""
    try:
        with open(path) as f:
            kv = dict(line.strip("- \n").split(": ", 1) for line in f
                      if line.startswith("- ") and ": " in line)
        if kv.get("sources_sha256") != kernel_sources_sha256(ADJOINT_SOURCES):
            return None
        return {k[len("traffic_bytes_per_launch_"):]: float(v) for k, v in kv.items()
                if k.startswith("traffic_bytes_per_launch_")}
    except (OSError, ValueError):
        return None


def oracle_gap(n, stride):
    """The oracle's max |Vbar - V| at the benchmark's threshold, from the
    committed golden file, when it was written for this grid and stride."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "c2_decomposed_%d.json" % n)) as f:
            g = json.load(f)
        if list(g["stride"]) != list(stride):
            return None
        return {"max_abs_isa_minus_full": g["max_abs_isa_minus_full"], "delta": g["delta"]}
    except (OSError, ValueError, KeyError):
        return None


def breakdown(ms_ra, ms_fine, tot, rst, fst, full_ms, nfree):
    """Where the decomposed step's time goes against the full-domain solve:
    the reconstruction, then the fine solve as sweeps x time per sweep, with
    the node-updates it performs relative to the full solve's."""
    return {
        "ra_ms": ms_ra,
        "fine_ms": ms_fine,
        "fine_sweeps": tot["iterations"],
        "fine_us_per_sweep": 1e3 * ms_fine / max(1, tot["iterations"]),
        "full_sweeps": fst["iterations"],
        "full_us_per_sweep": 1e3 * full_ms / max(1, fst["iterations"]),
        "fine_node_updates": tot["node_updates"],
        "full_node_updates": fst["node_updates"],
        "node_update_ratio": tot["node_updates"] / max(1, fst["node_updates"]),
        "labelled_over_free": rst["labelled"] / max(1, nfree),
    }


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for row in csv.reader(f):
                if len(row) < 9:
                    continue
                try:
                    sm.append(float(row[1]))
                    smax.append(float(row[2]))
                except ValueError:
                    continue
                for name, val in zip(names, row[5:9]):
                    if val.strip().lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cpu():
    """The host processor as /proc/cpuinfo names it (model name on x86, the
    implementer/part codes on Arm), with the machine type."""
    import platform
    name = None
    try:
        with open("/proc/cpuinfo") as f:
            info = {}
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    info.setdefault(k.strip().lower(), v.strip())
        name = info.get("model name") or (
            "implementer %s part %s" % (info.get("cpu implementer"), info.get("cpu part"))
            if "cpu part" in info else None)
    except OSError:
        pass
    return "%s (%s)" % (name or "unknown", platform.machine())


def cpu_baseline(seconds, n):
    """The FP64 oracle as it stands (OpenMP Jacobi applications of T) on the
    host cores, on a bounded sample of the workload: whole sweeps over the
    same grid until about `seconds` have elapsed."""
    import numpy as np

    import oracle as orc
    import synthetic as S
    d = S.c2(n=n)
    p = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"],
                    speed=d["speed"], current=d["current"], ntargets=d["ntargets"])
    cores = os.cpu_count() or 1
    V = orc.initial(p)
    nfree = int((d["labels"] == 0).sum())
    # the first sweeps of the iteration (a front near the targets) cost the
    # same per node as any other sweep: every free node evaluates every control
    t0 = time.perf_counter()
    sweeps = 0
    while True:
        V, _ = orc.apply(p, V, nthreads=cores)
        sweeps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return {"value": nfree * sweeps / el, "unit": UNIT, "cores": orc.max_threads() if cores < 1
            else cores, "kind": "oracle", "cpu": host_cpu(),
            "sample": "%d Jacobi sweeps of the FP64 oracle over the %dx%d grid (%d free nodes, "
                      "64 controls) in %.1f s" % (sweeps, n, n, nfree, el)}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle as orc
    import synthetic as S
    orc.build()
    d = S.c2(n=args.n)
    p = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"],
                    speed=d["speed"], current=d["current"], ntargets=d["ntargets"])
    cores = os.cpu_count() or 1
    nfree = int((d["labels"] == 0).sum())
    V = orc.initial(p)
    per_step = 2  # Jacobi sweeps per step: a bounded sample of the solve
    for _ in range(args.warmup):
        for _ in range(per_step):
            V, _ = orc.apply(p, V, nthreads=cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for _ in range(per_step):
            V, _ = orc.apply(p, V, nthreads=cores)
        times.append(time.perf_counter() - t0)
    el = sum(times)
    value = nfree * per_step * args.steps / el
    sample = ("%d Jacobi sweeps per step of the FP64 oracle over the %dx%d grid (%d free nodes, "
              "64 controls), %d threads" % (per_step, args.n, args.n, nfree, cores))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "grid": [args.n, args.n],
                                        "controls": 64, "targets": 16},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": host_cpu(),
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _timed_steps(step, steps, warmup, flush, local):
    """Run `warmup` untimed steps, then `steps` steps each between CUDA events
    on the current stream (L2 flushed before each, outside the events), with
    the clocks sampled meanwhile.  Returns (mean ms, last result, clocks)."""
    import torch
    for _ in range(warmup):
        step()
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    sampler.start()
    res = None
    for k in range(steps):
        flush.zero_()
        evs[k][0].record(stream)
        res = step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    return sum(a.elapsed_time(b) for a, b in evs) / steps, res, clocks


def _line(args, metric, value, unit, ms, config, **extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config}
    line.update(extra)
    print(json.dumps(line))


def run_dubins(args, hjb, S, dev, flush, local):
    """3D Dubins car, 256 x 256 x 128, reconstruction (stride 5, 5, 8) and the
    decomposed solve against the full-domain solve."""
    import numpy as np
    d = S.c3(nxy=126, nth=64, stride=(5, 5, 8)) if args.small else S.c3()
    nfree = int((d["labels"] == 0).sum())
    p = hjb.Problem(d["shape"], d["lo"], d["hi"], d["controls"], dev(d["labels"], np.uint8), d["h"],
                    dyn=hjb.HJB_DYN_DUBINS, periodic=(0, 0, 1), n_targets=d["ntargets"])
    if args.profile:
        # one step (reconstruction + decomposed solve) for a profiler
        fine, _, _, rst = hjb.subdomains(p, d["stride"], delta=-1.0, C_=0.0, M=-1.0)
        _, _, tot = hjb.solve_decomposed(p, fine)
        import torch
        torch.cuda.synchronize()
        print(json.dumps({"ra": rst, "total": tot}))
        return
    # work unit: the sweeps of plain (Jacobi) value iteration on the full grid
    _, fst_j = hjb.solve(p, local_iters=1)
    iters_full = fst_j["iterations"]
    ms_full, (Vf, fst), _ = _timed_steps(lambda: hjb.solve(p), args.steps, 1, flush, local)

    def step():
        fine, _, _, rst = hjb.subdomains(p, d["stride"], delta=-1.0, C_=0.0, M=-1.0)
        Vb, per, tot = hjb.solve_decomposed(p, fine)
        return Vb, rst, tot, per

    ms, (Vb, rst, tot, per), clocks = _timed_steps(step, args.steps, args.warmup, flush, local)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6660.0)
    # algorithmic work of the 3D sweep: 53 FP32 operations per node-update
    # (the foot's cell and fractions 10, bilinear values at three heading
    # layers 18, per control the heading interpolation and extremum 8 x 3,
    # the discount 1); 9 bytes per node of a staged tile (V read and write,
    # labels), once per tile visit however many applications it runs
    layers = tot.get("tile_layers") or 4
    nodes_per_tile = 32 * 8 * layers
    peak_ops = torch_sms(local) * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6
    ach_ops = tot["node_updates"] * 53 / (tot["ms"] / 1e3)
    alg_bytes = tot["tile_visits"] * nodes_per_tile * 9
    ach_bw = alg_bytes / (tot["ms"] / 1e3) / 1e9
    traffic = sweep_traffic(os.path.join(ROOT, "profiles", "sweep3d_dubins256_dram_traffic.md"),
                            rows=8, local_iters=tot.get("local_iters"))
    cpu = None
    if not args.no_cpu_baseline:
        import oracle as orc
        po = orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"], d["h"], dyn=1,
                         periodic=(0, 0, 1), ntargets=d["ntargets"])
        cores = os.cpu_count() or 1
        V = orc.initial(po)
        t0, sw = time.perf_counter(), 0
        while time.perf_counter() - t0 < args.cpu_seconds:
            V, _ = orc.apply(po, V, nthreads=cores)
            sw += 1
        el = time.perf_counter() - t0
        cpu = {"value": nfree * sw / el, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": host_cpu(),
               "sample": "%d Jacobi sweeps of the FP64 oracle over the 256x256x128 grid in %.1f s"
                         % (sw, el)}
    _line(args, "node-updates/s to convergence, decomposed vs full-domain GPU (3D Dubins)",
          nfree * iters_full / (ms / 1e3), UNIT, ms,
          {"workload": "dubins-%dx%dx%d-u3-8targets" % tuple(d["shape"]), "coarse_stride": list(d["stride"])},
          full_domain={"sweeps": fst["iterations"], "jacobi_sweeps": iters_full, "ms": ms_full,
                       "node_updates_per_s": nfree * iters_full / (ms_full / 1e3)},
          decomposed={"ms_ra": rst["ms"], "ms_fine": tot["ms"], "max_subdomain_iters": tot["iterations"],
                      "labelled_fraction": rst["labelled"] / d["labels"].size,
                      "max_abs_diff_vs_full": float((Vb - Vf).abs().max().item()),
                      "solved_subdomains": sum(1 for s in per if s["node_updates"] > 0)},
          raw_node_updates_per_s=(rst["node_updates"] + tot["node_updates"]) / (ms / 1e3),
          roofline={"bound": "alu", "achieved": ach_ops / 1e12, "peak": peak_ops / 1e12,
                    "unit": "Top/s", "frac": ach_ops / peak_ops,
                    "traffic": traffic["bytes_per_launch"] if traffic else None,
                    "traffic_unit": "DRAM bytes per sweep launch (ncu, warm L2, three launches "
                                    "of the fine solve's middle sweeps)",
                    "algorithmic_bytes_per_launch": alg_bytes / max(1, tot["iterations"]),
                    "hbm": {"achieved_gbs": ach_bw, "peak_gbs": hbm, "frac": ach_bw / hbm,
                            "bytes_per_tile_node": 9},
                    "ops_per_node_update": 53, "tile_layers": layers,
                    "kernel": "sweep3d_kernel (decomposed fine solve)"},
          cpu_baseline=cpu, gpu_launches=rst["launches"] + tot["launches"], clocks=clocks)


def run_vdp(args, hjb, S, dev, flush, local):
    """Van der Pol oscillator (Sec. 5, Example ex3) on 1025^2, 21 controls,
    running cost |x|, target disk in 4 cake slices: reconstruction at stride
    16 with delta = 0.1 and the decomposed solve against the full solve."""
    import numpy as np
    d = S.vdp(n=args.n, slices=4)
    nfree = int((d["labels"] == 0).sum())
    p = hjb.Problem(d["shape"], d["lo"], d["hi"], d["controls"], dev(d["labels"], np.uint8), d["h"],
                    current=dev(d["current"]), cost=dev(d["cost"]), n_targets=d["ntargets"],
                    value_out=d["v_out"])
    _, fst_j = hjb.solve(p, local_iters=1)
    iters_full = fst_j["iterations"]
    ms_full, (Vf, fst), _ = _timed_steps(lambda: hjb.solve(p), args.steps, 1, flush, local)
    delta = 0.1

    def step():
        fine, _, _, rst = hjb.subdomains(p, d["stride"], delta=delta)
        Vb, per, tot = hjb.solve_decomposed(p, fine)
        return Vb, rst, tot, per

    ms, (Vb, rst, tot, per), clocks = _timed_steps(step, args.steps, args.warmup, flush, local)
    peak = torch_sms(local) * 128 * measured_peaks().get("sm_max_mhz", 2070.0) * 1e6
    ach = tot["node_updates"] * d["controls"].shape[0] * OPS_PER_CONTROL / (tot["ms"] / 1e3)
    # recursive re-splitting of the slices (Conclusions remark on Example ex3)
    fine_s, _, _, sst = hjb.subdomains(p, d["stride"], delta=delta, max_splits=4)
    Vs, _, tot_s = hjb.solve_decomposed(p, fine_s, n_subdomains=sst["subdomains"])
    resplit = {"max_splits": 4, "subdomains": sst["subdomains"],
               "labelled_fraction": sst["labelled"] / d["labels"].size,
               "largest_fraction": sst["largest"] / d["labels"].size,
               "unsplit_largest_fraction": rst["largest"] / d["labels"].size,
               "ms_ra_with_splits": sst["ms"], "ms_fine": tot_s["ms"],
               "max_abs_diff_vs_unsplit": float((Vs - Vb).abs().max().item())}
    _line(args, "node-updates/s to convergence, decomposed vs full-domain GPU (Van der Pol)",
          nfree * iters_full / (ms / 1e3), UNIT, ms,
          {"workload": "vdp-%dx%d-A21-4slices" % (args.n, args.n), "coarse_stride": list(d["stride"]),
           "delta": delta},
          full_domain={"sweeps": fst["iterations"], "jacobi_sweeps": iters_full, "ms": ms_full,
                       "node_updates_per_s": nfree * iters_full / (ms_full / 1e3)},
          decomposed={"ms_ra": rst["ms"], "ms_fine": tot["ms"], "max_subdomain_iters": tot["iterations"],
                      "labelled_fraction": rst["labelled"] / d["labels"].size,
                      "max_abs_diff_vs_full": float((Vb - Vf).abs().max().item()),
                      "solved_subdomains": sum(1 for s in per if s["node_updates"] > 0)},
          raw_node_updates_per_s=(rst["node_updates"] + tot["node_updates"]) / (ms / 1e3),
          roofline={"bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "Top/s",
                    "frac": ach / peak, "traffic": None, "kernel": "sweep2d_kernel<0,V,4>"},
          resplit=resplit,
          cpu_baseline=None, gpu_launches=rst["launches"] + tot["launches"], clocks=clocks)


def run_game(args, hjb, S, dev, flush, local):
    """The pursuit-evasion game (Sec. 5, Example ex4) on 1025^2: 16 pursuer
    by 8 evader directions (128 pairs per node), per-axis scale field,
    running cost x1^2 + 0.1, capture disk in 4 slices; reconstruction at
    stride 16 (delta = 0.1) and the decomposed solve against the full solve."""
    import numpy as np
    d = S.pursuit_evasion(n=args.n, slices=4)
    nfree = int((d["labels"] == 0).sum())
    p = hjb.Problem(d["shape"], d["lo"], d["hi"], d["controls"], dev(d["labels"], np.uint8), d["h"],
                    scale=dev(d["scale"]), cost=dev(d["cost"]), n_targets=d["ntargets"],
                    value_out=d["v_out"], controls_b=d["controls_b"])
    _, fst_j = hjb.solve(p, local_iters=1)
    iters_full = fst_j["iterations"]
    ms_full, (Vf, fst), _ = _timed_steps(lambda: hjb.solve(p), args.steps, 1, flush, local)
    delta = 0.1

    def step():
        fine, _, _, rst = hjb.subdomains(p, d["stride"], delta=delta)
        Vb, per, tot = hjb.solve_decomposed(p, fine)
        return Vb, rst, tot, per

    ms, (Vb, rst, tot, per), clocks = _timed_steps(step, args.steps, args.warmup, flush, local)
    pairs = d["controls"].shape[0] * d["controls_b"].shape[0]
    peak = torch_sms(local) * 128 * measured_peaks().get("sm_max_mhz", 2070.0) * 1e6
    ach = tot["node_updates"] * pairs * OPS_PER_CONTROL / (tot["ms"] / 1e3)
    _line(args, "node-updates/s to convergence, decomposed vs full-domain GPU (pursuit-evasion game)",
          nfree * iters_full / (ms / 1e3), UNIT, ms,
          {"workload": "game-%dx%d-A16xB8-4slices" % (args.n, args.n),
           "coarse_stride": list(d["stride"]), "delta": delta},
          full_domain={"sweeps": fst["iterations"], "jacobi_sweeps": iters_full, "ms": ms_full,
                       "node_updates_per_s": nfree * iters_full / (ms_full / 1e3)},
          decomposed={"ms_ra": rst["ms"], "ms_fine": tot["ms"], "max_subdomain_iters": tot["iterations"],
                      "labelled_fraction": rst["labelled"] / d["labels"].size,
                      "max_abs_diff_vs_full": float((Vb - Vf).abs().max().item()),
                      "solved_subdomains": sum(1 for s in per if s["node_updates"] > 0)},
          raw_node_updates_per_s=(rst["node_updates"] + tot["node_updates"]) / (ms / 1e3),
          roofline={"bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "Top/s",
                    "frac": ach / peak, "traffic": None, "kernel": "sweep2d_kernel<0,V,2> (game)",
                    "evaluations_per_node_update": pairs},
          cpu_baseline=None, gpu_launches=rst["launches"] + tot["launches"], clocks=clocks)


def run_batch(args, hjb, S, dev, flush, local):
    """512 independent square problems, sides ~ U{64..512}, one launch."""
    import numpy as np
    sides = S.c4_sides()
    ds = [S.c4_problem(i, int(n)) for i, n in enumerate(sides)]
    ps = [hjb.Problem(d["shape"], d["lo"], d["hi"], d["controls"], dev(d["labels"], np.uint8),
                      d["h"], speed=dev(d["speed"]), n_targets=d["ntargets"]) for d in ds]
    nfree = [int((d["labels"] == 0).sum()) for d in ds]
    # work unit: the sweeps plain (Jacobi) value iteration needs per problem
    _, sts_j = hjb.solve_batch(ps, local_iters=1)
    ms, (Vs, sts), clocks = _timed_steps(lambda: hjb.solve_batch(ps), args.steps, args.warmup,
                                         flush, local)
    equiv = sum(nf * st["iterations"] for nf, st in zip(nfree, sts_j))
    upd = sum(st["node_updates"] for st in sts)
    peak = torch_sms(local) * 128 * measured_peaks().get("sm_max_mhz", 2070.0) * 1e6
    ach = upd * 32 * OPS_PER_CONTROL / (sts[0]["ms"] / 1e3)
    cpu = None
    if not args.no_cpu_baseline:
        import oracle as orc
        cores = os.cpu_count() or 1
        idx = np.argsort(sides)[:: len(sides) // 16]  # a stratified sample over the sizes
        pos = []
        for i in idx:
            d = ds[i]
            pos.append((i, orc.Problem(d["shape"], d["lo"], d["hi"], d["controls"], d["labels"],
                                       d["h"], speed=d["speed"], ntargets=d["ntargets"])))
        t0, done, rounds = time.perf_counter(), 0, 0
        while time.perf_counter() - t0 < args.cpu_seconds:
            for i, po in pos:
                V = orc.initial(po)
                for _ in range(3):
                    V, _ = orc.apply(po, V, nthreads=cores)
                done += 3 * nfree[i]
            rounds += 1
        el = time.perf_counter() - t0
        cpu = {"value": done / el, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": host_cpu(),
               "sample": "%d rounds of 3 Jacobi sweeps of the FP64 oracle on a size-stratified "
                         "sample of 16 batch problems (%d node-updates in %.1f s)"
                         % (rounds, done, el)}
    _line(args, "node-updates/s to convergence, batch of 512 uneven problems in one launch",
          equiv / (ms / 1e3), UNIT, ms,
          {"workload": "batch-512-sides64to512-A32", "problems": len(ps),
           "nodes": int(sum(int(n) ** 2 for n in sides))},
          raw_node_updates_per_s=upd / (ms / 1e3),
          max_iterations=max(st["iterations"] for st in sts),
          max_iterations_jacobi=max(st["iterations"] for st in sts_j),
          roofline={"bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "Top/s",
                    "frac": ach / peak, "traffic": None, "kernel": "sweep2d_kernel<32,W,2>"},
          cpu_baseline=cpu, gpu_launches=sts[0]["launches"], clocks=clocks)


def run_adjoint(args, hjb, S, dev, flush, local):
    """Gradient of the mean of V at 4096 points w.r.t. a 1025^2 log-speed field."""
    import numpy as np
    import torch
    d = S.c5(n=257) if args.small else S.c5()
    theta = dev(d["log_speed"])
    p = hjb.Problem(d["shape"], d["lo"], d["hi"], d["controls"], dev(d["labels"], np.uint8), d["h"],
                    log_speed=theta, n_targets=d["ntargets"])
    V, fst = hjb.solve(p)
    pts = dev(d["points"])
    _, gV = hjb.point_values(p, V, pts)
    if args.profile:
        _, st = hjb.backward(p, V, gV, wrt=0)
        torch.cuda.synchronize()
        print(json.dumps({"forward": fst, "backward": st}))
        return
    ms, (g, st), clocks = _timed_steps(lambda: hjb.backward(p, V, gV, wrt=0), args.steps,
                                       args.warmup, flush, local)
    N = d["labels"].size
    # node-updates of the transposed iteration and of the refinement of the
    # values the policy is decided on (a policy-frozen forward iteration):
    # both run block Gauss-Seidel sweeps; node_updates counts the transposed
    # sweep's applications, the refinement runs as many per tile and sweep
    ref = st["local_iters"]
    apps = st["node_updates"] // max(1, N * st["iterations"])
    upd = N * apps * (st["iterations"] + ref)
    hbm = measured_peaks().get("hbm_gbs", 6660.0)
    # per node and sweep of either: the policy foot's cell 4 B and fractions
    # 8 B, g (or r) 4 B, lambda (or the correction) read 4 B and written 4 B
    ach = N * 24 * (st["iterations"] + ref) / (st["ms"] / 1e3) / 1e9
    # measured DRAM traffic of one backward: the iteration kernels' per-launch
    # bytes (committed ncu windows) times their launches
    tr = adjoint_traffic()
    traffic = None
    if tr and all(k in tr for k in ("adj_tiles", "refine_tiles")):
        traffic = (st["iterations"] * tr["adj_tiles"] + ref * tr["refine_tiles"]
                   + 2 * tr.get("policy_kernel", 0.0))
    _line(args, "adjoint node-updates/s to convergence (transposed fixed point, policy frozen)",
          upd / (ms / 1e3), UNIT, ms, {"workload": "adjoint-%dx%d-A32-4096points" % tuple(d["shape"])},
          sweeps=st["iterations"], refine_sweeps=ref, forward_iterations=fst["iterations"],
          roofline={"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm, "traffic": traffic,
                    "traffic_unit": "DRAM bytes per backward (ncu, per-launch windows x launches)",
                    "algorithmic_bytes": N * 24 * (st["iterations"] + ref),
                    "kernel": "adj_tiles, refine_tiles",
                    "bytes_per_node_sweep": 24},
          cpu_baseline=None, gpu_launches=st["launches"], clocks=clocks)


def torch_sms(local):
    import torch
    return torch.cuda.get_device_properties(local).multi_processor_count


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "zermelo":
        import numpy as np
        import torch
        rank, world, local = env_rank()
        torch.cuda.set_device(local)
        import paper_1405_3521_gb300 as hjb
        import synthetic as S
        hjb._capi.lib()
        dev = lambda a, dt=np.float32: torch.as_tensor(np.ascontiguousarray(np.asarray(a).astype(dt))).cuda()  # noqa
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        {"dubins": run_dubins, "batch": run_batch, "adjoint": run_adjoint,
         "vdp": run_vdp, "game": run_game}[args.workload](
            args, hjb, S, dev, flush, local)
        return
    import numpy as np
    import torch

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import paper_1405_3521_gb300 as hjb
    import synthetic as S

    hjb._capi.lib()
    n = args.n
    d = S.c2(n=n)
    stride = d["stride"]
    nfree = int((d["labels"] == 0).sum())
    dev = lambda a, dt=torch.float32: torch.as_tensor(np.asarray(a)).to(dt).cuda().contiguous()  # noqa
    p = hjb.Problem(d["shape"], d["lo"], d["hi"], d["controls"], dev(d["labels"], torch.uint8),
                    d["h"], speed=dev(d["speed"]), current=dev(d["current"]),
                    n_targets=d["ntargets"])
    # the end-to-end leg's host buffers are page-locked, like the outputs the
    # package allocates for host problems
    host = lambda a, dt=np.float32: hjb.pinned_copy(a, dt)  # noqa
    ph = hjb.Problem(d["shape"], d["lo"], d["hi"], d["controls"], host(d["labels"], np.uint8),
                     d["h"], speed=host(d["speed"]), current=host(d["current"]),
                     n_targets=d["ntargets"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step(prob):
        fine, coarse, _, rst = hjb.subdomains(prob, stride, delta=-1.0, C_=0.0, M=-1.0)
        Vbar, per, tot = hjb.solve_decomposed(prob, fine)
        return Vbar, fine, rst, tot

    if args.profile:
        # one solve of the chosen path for a profiler: set HJB_TUNE=off and
        # pin HJB_TILE_ROWS / HJB_TILE_LANES / HJB_LOCAL_ITERS so that no
        # tuning runs precede it
        if args.profile == "full":
            _, info = hjb.solve(p)
        elif args.profile == "ra":
            _, _, _, info = hjb.subdomains(p, stride, delta=-1.0, C_=0.0, M=-1.0)
        else:
            fine, _, _, rst = hjb.subdomains(p, stride, delta=-1.0, C_=0.0, M=-1.0)
            _, per, tot = hjb.solve_decomposed(p, fine)
            info = {"ra": rst, "total": tot,
                    "per": [(s_["iterations"], s_["node_updates"]) for s_ in per]}
        torch.cuda.synchronize()
        print(json.dumps(info))
        return

    # full-domain reference solves on the same GPU (same stopping rule): plain
    # value iteration (Jacobi sweeps), whose sweep count fixes the work unit
    # N_free x iters_full of every rate below, and the default solve
    def full_times(local_iters):
        for _ in range(max(1, args.warmup)):
            V, st = hjb.solve(p, local_iters=local_iters)
        t = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            V, st = hjb.solve(p, local_iters=local_iters)
            t.append(st["ms"])
        return V, st, statistics.median(t)

    _, fst_j, full_ms_j = full_times(1)
    iters_full = fst_j["iterations"]
    Vfull, fst, full_ms = full_times(0)

    for _ in range(args.warmup):
        step(p)
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches = 0
    upd = 0
    loop_ms = 0.0
    ra_ms = 0.0
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        Vbar, fine, rst, tot = step(p)
        evs[k][1].record(stream)
        launches += rst["launches"] + tot["launches"]
        upd += rst["node_updates"] + tot["node_updates"]
        loop_ms += tot["ms"]
        ra_ms += rst["ms"]
    torch.cuda.synchronize()
    clocks = sampler.stop()
    step_ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    # one step solves one copy of the workload: nfree x iters_full full-domain
    # equivalent node-updates
    step_ms, value = aggregate(step_ms, nfree * iters_full, dist)
    if dist:
        dist.barrier()

    # end to end through the C ABI with host buffers (copies inside the call)
    e2e_times = []
    for k in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fine_h, coarse_h, _, _ = hjb.subdomains(ph, stride, delta=-1.0, C_=0.0, M=-1.0)
        Vbar_h, _, _ = hjb.solve_decomposed(ph, fine_h)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = statistics.median(e2e_times)
    N = n * n
    h2d = 2 * (N * 4 + N * 8 + N) + N * 4  # fields per call (2 calls) + the fine mask
    d2h = N * 4 + len(coarse_h) * 4 + N * 4  # fine mask, coarse labels, V

    # coarse-to-fine warm start of the fine solves (measured once, not the
    # timed step): each sub-domain starts from its coarse auxiliary solution
    # interpolated onto the fine grid
    fine_w, _, _, _ = hjb.subdomains(p, stride, delta=-1.0, C_=0.0, M=-1.0)
    Vcold, _, tot_c = hjb.solve_decomposed(p, fine_w)
    Vwarm, _, tot_w = hjb.solve_decomposed(p, fine_w, warm_start=1)
    warm = {"ms_fine": tot_w["ms"], "sweeps": tot_w["iterations"],
            "node_updates": tot_w["node_updates"], "cold_ms_fine": tot_c["ms"],
            "cold_sweeps": tot_c["iterations"], "cold_node_updates": tot_c["node_updates"],
            "max_abs_diff_vs_cold": float((Vwarm - Vcold).abs().max().item())}

    raw = upd / args.steps / (step_ms / 1e3)
    # roofline of the dominant kernel (the 2D sweep, 64 controls, W form)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peaks = measured_peaks()
    fmax = peaks.get("sm_max_mhz", 2070.0) * 1e6
    peak_ops = sms * 128 * fmax
    achieved = (tot["node_updates"] * 64 * OPS_PER_CONTROL) / (tot["ms"] / 1e3)
    rows = tot.get("tile_rows") or None
    traffic = sweep_traffic(rows=rows, local_iters=tot.get("local_iters"))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle  # noqa: F401
        cpu = cpu_baseline(args.cpu_seconds, n)
    check = float((Vbar - Vfull).abs().max().item())
    gold = oracle_gap(n, stride)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [n, n], "controls": 64, "targets": 16,
                   "coarse_stride": list(stride), "delta": "2 M dx_K (M estimated)",
                   "l2": "flushed between steps (256 MB write outside the event-timed region)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "raw_node_updates_per_s": raw * world,
        "full_domain": {"sweeps": fst["iterations"], "ms": full_ms,
                        "node_updates_per_s": nfree * iters_full / (full_ms / 1e3)},
        "full_domain_jacobi": {"sweeps": iters_full, "ms": full_ms_j,
                               "node_updates_per_s": nfree * iters_full / (full_ms_j / 1e3)},
        "decomposed": {"ms_ra": ra_ms / args.steps, "ms_fine": loop_ms / args.steps,
                       "max_subdomain_iters": tot["iterations"],
                       "labelled_fraction": rst["labelled"] / N, "ra_iters": rst["iterations"],
                       "delta": rst["delta"], "lipschitz": rst["lipschitz"],
                       "max_abs_diff_vs_full": check,
                       # the method's own difference between the assembled ISA value and the
                       # full-domain value at this threshold, from the FP64 oracle
                       # (tests/golden/c2_decomposed_1025.json); the GPU must reproduce it
                       "oracle_max_abs_isa_minus_full": gold["max_abs_isa_minus_full"] if gold else None,
                       "oracle_delta": gold["delta"] if gold else None,
                       "gap_matches_oracle": (abs(check - gold["max_abs_isa_minus_full"]) < 1e-4)
                       if gold else None,
                       "breakdown": breakdown(ra_ms / args.steps, loop_ms / args.steps, tot, rst,
                                              fst, full_ms, nfree)},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "Top/s", "frac": achieved / peak_ops,
                     "traffic": traffic["bytes_per_launch"] if traffic else None,
                     "traffic_unit": "DRAM bytes per sweep launch (ncu, warm L2, three launches "
                                     "of the fine solve's busiest phase)",
                     # 9 B per node-update (V read and write, labels), average sweep
                     "algorithmic_bytes_per_launch": 9 * tot["node_updates"] / max(1, tot["iterations"]),
                     "kernel": "sweep2d_kernel<64 controls, W form> 32x%s tiles, %s (decomposed "
                               "fine solve)" % (rows or "?", "lane split" if tot.get("tile_lanes") == 2
                                                else "control groups"),
                     "peak_source": "SMs x 128 FP32 lanes x max SM clock (derived)"},
        "cpu_baseline": cpu,
        "e2e": {"value": nfree * iters_full / e2e_s * world, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
        "warm_start": warm,
        "tuned": {"fine_tile_rows": tot.get("tile_rows"), "fine_tile_lanes": tot.get("tile_lanes"),
                  "fine_local_iters": tot.get("local_iters"), "ra_local_iters": rst.get("local_iters"),
                  "full_tile_rows": fst.get("tile_rows"), "full_tile_lanes": fst.get("tile_lanes"),
                  "full_local_iters": fst.get("local_iters")},
    }
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
