"""Host-side checks that need no GPU: the C library builds, loads and exports
every entry point declared in include/hjb.h; descriptor validation; the
seeded inputs; the separation of the oracle from the library; the
multi-rank aggregation of the benchmark (gloo, world size 2)."""
import ctypes as C
import os
import re
import shutil
import subprocess
import sys

import numpy as np
import pytest

import synthetic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hjb.h")).read()
    return re.findall(r"^(?:int|const char \*)\s*(hjb_\w+)\(", src, flags=re.M)


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1405_3521_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = set(_declared())
    for n in ["hjb_create", "hjb_destroy", "hjb_solve", "hjb_subdomains", "hjb_solve_decomposed",
              "hjb_solve_batch", "hjb_backward", "hjb_point_values", "hjb_last_error",
              "hjb_version"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = C.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True).stdout
    for name in _declared():
        assert re.search(r" T %s$" % name, out, flags=re.M), name


def test_create_validates_without_touching_the_gpu(libpath):
    import paper_1405_3521_gb300 as hjb
    from paper_1405_3521_gb300 import _capi
    L = _capi.lib()
    g = _capi.hjb_grid()
    g.ndim = 4
    dy, co, di, ct, tg = (_capi.hjb_dynamics(), _capi.hjb_cost(), _capi.hjb_discount(),
                          _capi.hjb_controls(), _capi.hjb_target())
    h = C.c_void_p()
    rc = L.hjb_create(C.byref(g), C.byref(dy), C.byref(co), C.byref(di), C.byref(ct), C.byref(tg),
                      C.byref(h))
    assert rc == _capi.HJB_ERR_INVALID_ARG
    assert b"ndim" in L.hjb_last_error()
    # a valid grid with a bad control set
    lab = np.zeros(16, dtype=np.uint8)
    with pytest.raises(hjb.HJBError):
        hjb.Problem((4, 4), (0, 0), (1, 1), np.full((2, 2), np.nan, np.float32), lab, 0.1,
                    n_targets=1)
    with pytest.raises(hjb.HJBError):
        hjb.Problem((4, 4), (0, 0), (1, 1), S.circle_controls(4), lab, -0.1, n_targets=1)
    with pytest.raises(hjb.HJBError):
        hjb.Problem((4, 4), (0, 0), (1, 1), S.circle_controls(4), lab, 0.1, n_targets=40)
    p = hjb.Problem((4, 4), (0, 0), (1, 1), S.circle_controls(4), lab, 0.1, n_targets=1)
    p.close()
    assert L.hjb_destroy(None) == 0


def test_create_validates_scheme_and_game_options(libpath):
    """The options of the step weights, the interpolation, the per-axis scale
    field and the second player are checked at creation (no GPU needed)."""
    import paper_1405_3521_gb300 as hjb
    lab = np.zeros(16, dtype=np.uint8)
    A = S.circle_controls(4).astype(np.float32)
    ok = dict(n_targets=1)
    for bad in (dict(weights=2), dict(interp=3), dict(interp=-1)):
        with pytest.raises(hjb.HJBError):
            hjb.Problem((4, 4), (0, 0), (1, 1), A, lab, 0.1, **ok, **bad)
    # speed and scale are exclusive
    with pytest.raises(hjb.HJBError):
        hjb.Problem((4, 4), (0, 0), (1, 1), A, lab, 0.1, speed=np.ones(16, np.float32),
                    scale=np.ones((16, 2), np.float32), **ok)
    # second player: count * count_b <= 128, finite components
    with pytest.raises(hjb.HJBError):
        hjb.Problem((4, 4), (0, 0), (1, 1), S.circle_controls(16), lab, 0.1,
                    controls_b=np.zeros((9, 2), np.float32), **ok)
    with pytest.raises(hjb.HJBError):
        hjb.Problem((4, 4), (0, 0), (1, 1), A, lab, 0.1,
                    controls_b=np.full((2, 2), np.inf, np.float32), **ok)
    # P1 and games are 2D speed/current features
    lab3 = np.zeros(4 * 4 * 4, dtype=np.uint8)
    u = np.array([[-1.0], [0.0], [1.0]], np.float32)
    with pytest.raises(hjb.HJBError):
        hjb.Problem((4, 4, 4), (0, 0, 0), (1, 1, 6.28), u, lab3, 0.1, dyn=hjb.HJB_DYN_DUBINS,
                    periodic=(0, 0, 1), interp=1, **ok)
    # valid combinations are accepted
    for good in (dict(weights=1), dict(interp=1), dict(scale=np.ones((16, 2), np.float32)),
                 dict(controls_b=0.5 * A)):
        hjb.Problem((4, 4), (0, 0), (1, 1), A, lab, 0.1, **ok, **good).close()


def test_package_never_reaches_the_oracle():
    """The library path and the oracle share no code and the package never
    imports, loads or runs anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_1405_3521_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b|ohjb_|liboracle", txt), f
    src = open(os.path.join(ROOT, "oracle", "hjb_oracle.c")).read()
    assert "hjb_internal" not in src and "include/hjb.h" not in src


def test_synthetic_inputs_are_seeded_and_shaped():
    d1, d2 = S.c2(n=65), S.c2(n=65)
    assert np.array_equal(d1["speed"], d2["speed"])
    assert d1["speed"].min() >= 0.5 - 1e-6 and d1["speed"].max() <= 1.5 + 1e-6
    c = d1["current"]
    assert np.sqrt((c ** 2).sum(-1)).max() <= 0.4 + 1e-6
    cen = d1["centers"]
    for i in range(len(cen)):
        for j in range(i):
            assert np.hypot(*(cen[i] - cen[j])) >= 0.3
    assert set(np.unique(d1["labels"])) <= set(range(17))
    # the current is divergence-free (analytic curl of a stream function)
    X, Y = S.mesh2(257, 257)
    cf = S.current_field(S.rng("current", 2), X, Y)
    h = 2.0 / 256
    div = np.gradient(cf[..., 0], h, axis=1) + np.gradient(cf[..., 1], h, axis=0)
    assert np.abs(div[2:-2, 2:-2]).max() < 0.05 * np.abs(cf).max() / h * h * 50
    sides = S.c4_sides()
    assert len(sides) == 512 and sides.min() >= 64 and sides.max() <= 512
    th = S.grf_logspeed(S.rng("theta", 1), 65)
    assert abs(th.min() - np.log(0.5)) < 1e-12 and abs(th.max() - np.log(1.5)) < 1e-12


def _agg_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms, total = bench.aggregate(step_ms=10.0 + rank, units_per_rank=1000.0, dist=dist,
                                device="cpu")
    q.put((rank, ms, total))
    dist.destroy_process_group()


def test_bench_aggregation_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_agg_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, total in res:
        assert ms == 11.0  # the slowest rank sets the time
        assert abs(total - 2000.0 / 11.0e-3) < 1e-6 * total  # units of all ranks / that time


def test_bench_traffic_lookup(tmp_path):
    """roofline.traffic comes from a committed ncu summary only for the kernel
    sources, tile shape and applications per tile the summary was taken on."""
    sys.path.insert(0, ROOT)
    import bench
    h = bench.kernel_sources_sha256()
    f = tmp_path / "t.md"
    f.write_text("- traffic_bytes_per_launch_rows8_li6: 100\n- node_updates_per_launch_rows8_li6: 10\n"
                 "- traffic_bytes_per_launch_rows4_li6: 200\n- node_updates_per_launch_rows4_li6: 20\n"
                 "- traffic_bytes_per_launch_rows4_li8: 5\n- sources_sha256: %s\n" % h)
    assert bench.sweep_traffic(str(f), rows=4, local_iters=6) == {
        "bytes_per_launch": 200.0, "node_updates_per_launch": 20.0}
    assert bench.sweep_traffic(str(f), rows=8, local_iters=6)["bytes_per_launch"] == 100.0
    assert bench.sweep_traffic(str(f), rows=4, local_iters=8) == {"bytes_per_launch": 5.0}
    assert bench.sweep_traffic(str(f), rows=2, local_iters=6) is None
    assert bench.sweep_traffic(str(f), rows=4, local_iters=4) is None
    f.write_text(f.read_text().replace(h, "0" * 64))
    assert bench.sweep_traffic(str(f), rows=4, local_iters=6) is None


def test_missing_library_fails_loudly():
    """With no built library the package raises instead of computing
    anything another way (there is no CPU path)."""
    code = ("import paper_1405_3521_gb300 as h\n"
            "try:\n"
            "    h._capi.lib()\n"
            "except ImportError as e:\n"
            "    print('raised:', e)\n"
            "else:\n"
            "    print('loaded')\n")
    env = dict(os.environ, HJB_LIBRARY=os.path.join(ROOT, "_no_such_dir", "libhjb.so"))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.startswith("raised: libhjb.so is not built"), r.stdout


def test_work_queue_limits_are_enforced_on_the_host(libpath):
    """A work-queue entry holds a problem index in 9 bits and a tile index in
    22: a batch of more than 512 problems, or a grid of more than 2^22 tiles
    of 32 x 2 nodes, is refused before anything reaches the GPU."""
    from paper_1405_3521_gb300 import _capi
    L = _capi.lib()
    count = 513
    probs = (C.c_void_p * count)()
    outs = (C.c_void_p * count)()
    rc = L.hjb_solve_batch(probs, count, None, outs, None, None)
    assert rc == _capi.HJB_ERR_INVALID_ARG
    assert b"at most 512 problems" in L.hjb_last_error()
    lab = np.zeros(16, dtype=np.uint8)
    A = np.asarray(S.circle_controls(4), np.float32)

    def create(n0, n1):
        g = _capi.hjb_grid()
        g.ndim = 2
        g.n[0], g.n[1] = n0, n1
        g.lo[0] = g.lo[1] = -1.0
        g.hi[0] = g.hi[1] = 1.0
        dy, co, di, ct, tg = (_capi.hjb_dynamics(), _capi.hjb_cost(), _capi.hjb_discount(),
                              _capi.hjb_controls(), _capi.hjb_target())
        co.l_const = 1.0
        di.h, di.lam = 1e-4, 1.0
        ct.count, ct.dim = 4, 2
        ct.a = A.ctypes.data
        tg.labels = lab.ctypes.data
        tg.n_targets, tg.value_out = 1, 1.0
        h = C.c_void_p()
        rc = L.hjb_create(C.byref(g), C.byref(dy), C.byref(co), C.byref(di), C.byref(ct),
                          C.byref(tg), C.byref(h))
        if rc == 0:
            L.hjb_destroy(h)
        return rc

    # 16384 x 16384 nodes: exactly 2^22 tiles of 32 x 2; one more row of tiles is refused
    assert create(16384, 16384) == 0
    assert create(16384, 16386) == _capi.HJB_ERR_UNSUPPORTED
    assert b"tiles" in L.hjb_last_error()


def test_solve_options_are_validated_on_the_host(libpath):
    """An unknown choice of sub-problem targets is refused before anything
    reaches the GPU."""
    import paper_1405_3521_gb300 as hjb
    from paper_1405_3521_gb300 import _capi
    L = _capi.lib()
    lab = np.zeros(16, dtype=np.uint8)
    lab[0] = 1
    p = hjb.Problem((4, 4), (0, 0), (1, 1), S.circle_controls(4), lab, 0.1, n_targets=1)
    o = hjb._opts(subdomain_targets=2)
    out = np.zeros(16, np.float32)
    rc = L.hjb_solve(p.handle, C.byref(o), out.ctypes.data, None, None)
    assert rc == _capi.HJB_ERR_INVALID_ARG
    assert b"subdomain_targets" in L.hjb_last_error()
    p.close()


def test_bench_reference_arm_line():
    """bench.py --impl reference times the oracle on the host cores and prints
    one JSON line with the contract's keys (no GPU involved)."""
    import json
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--n", "65"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    for key in ("metric", "unit", "n_gpus", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_entry_points_validate_arguments_on_the_host(libpath):
    """Argument errors of the solve, reconstruction, adjoint and point-value
    entry points are refused before any CUDA call (so also without a GPU)."""
    import paper_1405_3521_gb300 as hjb
    from paper_1405_3521_gb300 import _capi
    L = _capi.lib()
    n = 9
    lab = np.zeros(n * n, dtype=np.uint8)
    lab[0] = 1
    p = hjb.Problem((n, n), (0, 0), (1, 1), S.circle_controls(4), lab, 0.1, n_targets=1)
    buf = np.zeros(n * n, np.float32)
    mask = np.zeros(n * n, np.uint32)
    ptr = buf.ctypes.data

    def err(rc, code, text):
        assert rc == code, (rc, L.hjb_last_error())
        assert text in L.hjb_last_error(), L.hjb_last_error()

    ra = _capi.hjb_ra_opts()
    for stride, text in (((0, 2), b"< 1"), ((3, 2), b"does not divide")):
        ra.coarse_stride[0], ra.coarse_stride[1] = stride
        err(L.hjb_subdomains(p.handle, C.byref(ra), mask.ctypes.data, None, None, None, None),
            _capi.HJB_ERR_INVALID_ARG, text)
    err(L.hjb_backward(p.handle, ptr, ptr, 2, None, ptr, None, None),
        _capi.HJB_ERR_INVALID_ARG, b"wrt")
    o = hjb._opts(max_iters=-1)
    err(L.hjb_backward(p.handle, ptr, ptr, 0, C.byref(o), ptr, None, None),
        _capi.HJB_ERR_INVALID_ARG, b"max_iters")
    err(L.hjb_solve_decomposed(p.handle, mask.ctypes.data, C.byref(o), ptr, None, None, None),
        _capi.HJB_ERR_INVALID_ARG, b"max_iters")
    err(L.hjb_point_values(p.handle, ptr, ptr, -1, None, None, None),
        _capi.HJB_ERR_INVALID_ARG, b"bad argument")
    # games have no adjoint
    g = hjb.Problem((n, n), (0, 0), (1, 1), S.circle_controls(4), lab, 0.1, n_targets=1,
                    controls_b=0.5 * np.asarray(S.circle_controls(2), np.float32))
    err(L.hjb_backward(g.handle, ptr, ptr, 0, None, ptr, None, None),
        _capi.HJB_ERR_UNSUPPORTED, b"without games")
    g.close()
    p.close()


C_CLIENT = r"""
#include "hjb.h"
#include <stdio.h>

/* A C client of the library: builds a problem descriptor and checks that a
 * bad grid is refused with a message; never reaches the GPU. */
int main(void) {
    hjb_grid grid = {0};
    hjb_dynamics dyn = {0};
    hjb_cost cost = {0};
    hjb_discount disc = {0};
    hjb_controls controls = {0};
    hjb_target target = {0};
    hjb_solve_opts opts = {0};
    hjb_stats stats = {0};
    hjb_problem *p = NULL;
    grid.ndim = 5;
    opts.subdomain_targets = HJB_SUBDOMAIN_TARGETS_OWN;
    int rc = hjb_create(&grid, &dyn, &cost, &disc, &controls, &target, &p);
    printf("%d %s %d %d\n", rc, hjb_last_error(), (int)sizeof opts, stats.tile_rows);
    return rc == HJB_ERR_INVALID_ARG && p == NULL ? 0 : 1;
}
"""


@pytest.mark.parametrize("lang", ["c99", "c++17"])
def test_header_serves_a_c_client(libpath, tmp_path, lang):
    """include/hjb.h compiles as C99 and as C++ on its own (no CUDA headers),
    and a C program links against libhjb.so and runs its host-side checks."""
    cc = "gcc" if lang == "c99" else "g++"
    if shutil.which(cc) is None:
        pytest.skip(cc + " not available")
    src = tmp_path / ("client.c" if lang == "c99" else "client.cpp")
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(libpath)
    r = subprocess.run([cc, "-std=" + lang, "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", libdir, "-lhjb", "-Wl,-rpath," + libdir, "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ndim" in r.stdout


def test_binding_structs_match_the_header(tmp_path):
    """Every descriptor the Python binding marshals has the size and field
    offsets that include/hjb.h gives it (a C program prints them)."""
    import ctypes as C

    from paper_1405_3521_gb300 import _capi
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not available")
    structs = {"hjb_grid": _capi.hjb_grid, "hjb_dynamics": _capi.hjb_dynamics,
               "hjb_cost": _capi.hjb_cost, "hjb_discount": _capi.hjb_discount,
               "hjb_controls": _capi.hjb_controls, "hjb_target": _capi.hjb_target,
               "hjb_solve_opts": _capi.hjb_solve_opts, "hjb_stats": _capi.hjb_stats,
               "hjb_ra_opts": _capi.hjb_ra_opts, "hjb_tune_choice": _capi.hjb_tune_choice}
    # the binding renames one field (lambda is a Python keyword)
    cname = {("hjb_discount", "lam"): "lambda"}
    lines = []
    for sname, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (sname, sname))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));'
                         % (sname, f, sname, cname.get((sname, f), f)))
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "hjb.h"\nint main(void) {\n'
                   + "\n".join(lines) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True,
                                                       text=True).stdout.splitlines())
    for sname, cls in structs.items():
        assert int(got[sname]) == C.sizeof(cls), sname
        for f, _ in cls._fields_:
            assert int(got[sname + "." + f]) == getattr(cls, f).offset, (sname, f)


TUNE_ROUND_TRIP = r"""
import ctypes as C, json, sys
from paper_1405_3521_gb300 import _capi
L = _capi.lib()
path = sys.argv[1]
assert L.hjb_tune_clear() == 0
keys = [b"NVIDIA GB300/152|decomposed|0|1025|1025|1|64|0|0|0|16|0", b"NVIDIA GB300/152|batch|0|512",
        b"NVIDIA GB300/152|ra|0|65|65|1|64|0|0|0|16|2"]
want = [(4, 2, 6, 13.9, 4), (8, 1, 8, 150.25, 2), (1, 1, 1, 0.5, 4)]
for k, (r, ln, l, ms, ly) in zip(keys, want):
    assert L.hjb_tune_set(k, C.byref(_capi.hjb_tune_choice(r, ln, l, ms, ly))) == 0
bad = _capi.HJB_ERR_INVALID_ARG
assert L.hjb_tune_set(b"x", C.byref(_capi.hjb_tune_choice(3, 1, 6, 0.0, 4))) == bad
assert L.hjb_tune_set(b"x", C.byref(_capi.hjb_tune_choice(8, 2, 6, 0.0, 4))) == bad
assert L.hjb_tune_set(b"x", C.byref(_capi.hjb_tune_choice(8, 1, 6, 0.0, 3))) == bad
assert L.hjb_tune_set(b'a"b', C.byref(_capi.hjb_tune_choice(4, 1, 6, 0.0, 4))) == bad
assert L.hjb_tune_save(path.encode()) == 0
entries = json.load(open(path))
assert sorted(e["key"] for e in entries) == sorted(k.decode() for k in keys)
assert L.hjb_tune_clear() == 0
out = _capi.hjb_tune_choice()
assert L.hjb_tune_get(keys[0], C.byref(out)) == _capi.HJB_ERR_INVALID_ARG
n = C.c_int(0)
assert L.hjb_tune_load(path.encode(), C.byref(n)) == 0 and n.value == 3
for k, (r, ln, l, ms, ly) in zip(keys, want):
    assert L.hjb_tune_get(k, C.byref(out)) == 0
    assert (out.tile_rows, out.lanes, out.local_iters, out.layers) == (r, ln, l, ly)
    assert abs(out.ms - ms) < 1e-3
assert L.hjb_tune_load(b"/nonexistent/tune.json", None) == _capi.HJB_ERR_INVALID_ARG
print("ok")
"""


def test_tuning_table_round_trips_through_a_file(libpath, tmp_path):
    """The autotuner's table survives a save and a load through the C ABI
    (no GPU: the table is host state), and the file is valid JSON."""
    r = subprocess.run([sys.executable, "-c", TUNE_ROUND_TRIP, str(tmp_path / "tune.json")],
                       cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
