"""Benchmark of the FMM-accelerated collocation BEM hot path on one GB300.

Workload (default): Laplace exterior Neumann problem on the cube [-1,1]^3,
45 x 45 graded quads per face split into 24,300 6-node triangles (48,602
nodes), point source at (0.2, -0.1, 0.3), expansion order p = 10, separation
factor 2, leaf size from the autotuner's table for this size class, GMRES(30),
in the mixed form (float32 near field and expansions, float64 Krylov);
--precision f64 times the plain float64 form.

One step = one complete pass of the hot path from a device-resident mesh:
plan build on the device (quadrature geometry, octree, radii, lists,
special-pair correction, diagonal), the right-hand side b = B chi (one fast
product), and the GMRES solve of A phi = b (one fast product per Arnoldi
step).  value = solves per second over all ranks (each rank an independent
replica).  The L2 cache is flushed between steps.

Extra keys: matvecs_per_s (back-to-back A products of a built plan), per-stage
times, the roofline of the dominant kernel against measured peaks, the plain
float64 form on the same workload with the mixed solution's error against it
(f64_form), a served request stream in both forms (serving), batched
instances solved as one group against one at a time (grouped), the CPU oracle
baseline, end-to-end timing through the public API with host buffers.

--impl reference times the CPU oracle (the plain FP64 matrix-free operator
rows) on a bounded sample of the same workload and extrapolates to solves/s.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM-BEM matvecs/s & served solves/s, p50/p99 latency vs plain FP64 at rel.err≤1e-5"
WORKLOAD = "cube45-tri6-laplace"
SOURCE = (0.2, -0.1, 0.3)
FLOPS_PER_PAIR = {"A": 20.0, "B": 11.0}   # near-field kernel, Laplace double / single layer
# DRAM bytes (read + write) per launch of the dominant kernels, from one ncu
# capture of this workload (the command is in profiles/); reported while the
# kernel's source file is unchanged, null otherwise.
NCU_TRAFFIC = {
    # k_near_f32 (unchanged since its capture; the file's other kernels changed)
    "near_l2p": {"bytes": 7472896, "source": "paper_0908_0673_gb300/csrc/fmm.cu",
                 "sha256": "4317124a9ff3d54da8a2ff674b49021ac10198ab50caef2b27b527477827ca7e"},
    # the M2L stage: k_m2l_permute + k_m2l_tc + k_m2l_gather_sym (order-10 products)
    "m2l": {"bytes": 1217024 + (35090432 + 46180096) + 123055872, "source": "paper_0908_0673_gb300/csrc/m2l_tc.cu",
            "sha256": "e7871ff432f963f53dd84460d1103eb7b3af23f26d5a89e5156d1826afe70520"},
}


def tc_issued_macs(p):
    """MACs the tensor-core M2L issues per interaction pair and split term:
    one MMA per K-step of 8 columns a, over the rows b that step reaches (the
    first cum(p - min|a| + 1) rows in degree order, rounded up to 16)."""
    deg = [d for d in range(p + 1) for _ in range((d + 1) * (d + 2) // 2)]
    cum = lambda d: d * (d + 1) * (d + 2) // 6 if d > 0 else 0
    total = 0
    for j in range((len(deg) + 7) // 8):
        dmin = min(deg[8 * j:8 * j + 8])
        total += 8 * ((cum(p - dmin + 1) + 15) // 16 * 16)
    return total


def ncu_traffic(stage):
    import hashlib
    rec = NCU_TRAFFIC.get(stage)
    if rec is None:
        return None
    with open(os.path.join(ROOT, rec["source"]), "rb") as f:
        return rec["bytes"] if hashlib.sha256(f.read()).hexdigest() == rec["sha256"] else None


# Arnoldi steps of a float64 GMRES(30) solve of this workload to 1e-10, as
# this benchmark's float64 form measures them on a GB300 (its gmres_iters);
# used only to extrapolate the CPU oracle's rate to solves (the oracle's
# product is float64 too).  One RHS product plus these steps; the final
# true-residual product is left out, in the oracle's favour.
GMRES_ITERS_CUBE45 = 14


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["f64", "mixed"])
    ap.add_argument("--n", type=int, default=45, help="quads per cube face edge")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-f64", action="store_true", help="skip timing the plain float64 form")
    ap.add_argument("--leaf", type=int, default=0, help="leaf size (0: the autotuner's choice)")
    ap.add_argument("--group", type=int, default=12, help="instances solved as one group (0: skip)")
    ap.add_argument("--group-min-elems", type=int, default=2000)
    ap.add_argument("--group-max-elems", type=int, default=10000)
    ap.add_argument("--group-max-rhs", type=int, default=3)
    ap.add_argument("--serve-requests", type=int, default=8, help="requests in the serving stream (0: skip)")
    ap.add_argument("--serve-max-elems", type=int, default=20000, help="largest mesh of the serving stream")
    ap.add_argument("--serve-kmax", type=float, default=4.0, help="largest Helmholtz wavenumber of the serving stream")
    ap.add_argument("--group-kmax", type=float, default=4.0, help="largest Helmholtz wavenumber of the grouped instances")
    ap.add_argument("--group-f64-rhs", type=int, default=1,
                    help="right-hand sides per grouped instance checked against its float64 solution")
    ap.add_argument("--serve-f64-max-elems", type=int, default=30000,
                    help="largest request of the float64 comparison stream (the subset served by both forms)")
    ap.add_argument("--only", default="", choices=["", "grouped", "serving"],
                    help="run one section alone and print its JSON (not the benchmark line)")
    return ap.parse_args()


def workload(n):
    from paper_0908_0673_gb300 import inputs as I
    m = I.cube(n, I.TRI6, grade=1.2, seed=0)
    phi_ex, chi_e = I.point_source(m, SOURCE)
    return m, phi_ex, chi_e


def chi_vector(chi_idx, n_chi, chi_e):
    out = np.zeros(n_chi)
    out[chi_idx.ravel()] = chi_e.ravel()        # equal inside one index by construction
    return out


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, gpu_index):
        self.p = None
        self.path = os.path.join(tempfile.gettempdir(), f"bem_clocks_{os.getpid()}.csv")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _omp_threads(n):
    """Sets the OpenMP thread count of the oracle's runtime (libgomp is shared
    by the process, so this reaches the oracle's parallel loops)."""
    import ctypes
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(n))
        return True
    except OSError:
        return False


def _oracle_rows(O, m, chi_idx, n_phi, budget_s, seed=0):
    """Rows of the oracle's matrix-free A product on a row sample sized to
    about budget_s seconds: (rows timed, seconds)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n_phi)
    t0 = time.perf_counter()
    rows = rng.choice(n_phi, min(n_phi, 16), replace=False)
    O.apply_rows(m.nodes, m.elems, chi_idx, O.OP_A, x, rows)
    dt = time.perf_counter() - t0
    nrows = int(max(16, min(n_phi, 16 * budget_s / max(dt, 1e-3))))
    rows = rng.choice(n_phi, nrows, replace=False)
    t0 = time.perf_counter()
    O.apply_rows(m.nodes, m.elems, chi_idx, O.OP_A, x, rows)
    return nrows, time.perf_counter() - t0


def oracle_small_problem(O):
    """The paper's first test at full size (level-3 icosphere, 1280 flat
    triangles, 642 nodes, point source inside): the oracle's dense assembly,
    its LU solve and its restarted GMRES(30) solve (tol 1e-10) with the
    direct matrix-free product, on all host cores."""
    from paper_0908_0673_gb300 import inputs as I
    m = I.icosphere(3, I.TRI3)
    ci, n_chi = O.chi_index(m.nodes, m.elems)
    _, chi_e = I.point_source(m, (0.1, 0.2, -0.15))
    chi = O.chi_from_elem(ci, n_chi, chi_e)
    t0 = time.perf_counter()
    A, B, _ = O.operators(m.nodes, m.elems, ci, n_chi)
    t_asm = time.perf_counter() - t0
    b = (B @ chi).real
    t0 = time.perf_counter()
    phi_lu = O.solve_dense(A.real, b)
    t_lu = time.perf_counter() - t0
    # GMRES with the oracle's direct product (the right-hand side from it too)
    t0 = time.perf_counter()
    rhs = O.apply_rows(m.nodes, m.elems, ci, O.OP_B, chi)
    phi_g, it, rel = O.gmres(lambda v: O.apply_rows(m.nodes, m.elems, ci, O.OP_A, v), rhs, restart=30, tol=1e-10)
    t_gm = time.perf_counter() - t0
    return {"workload": "icosphere3-tri3-laplace (1280 elements, 642 nodes)",
            "dense_assembly_s": t_asm, "lu_solve_s": t_lu, "gmres_solve_s": t_gm, "gmres_iters": int(it),
            "gmres_rel_residual": rel,
            "gmres_vs_lu_rel_diff": float(np.linalg.norm(phi_g - phi_lu) / np.linalg.norm(phi_lu))}


def cpu_baseline(m, chi_idx, n_phi, iters, budget_s=15.0, extra_legs=True):
    """The oracle's matrix-free rows of A on a bounded sample of this
    workload, extrapolated to solves/s ((iters + 1) full products per solve:
    one for the right-hand side, one per Arnoldi step).  extra_legs adds the
    same rate on one thread and the oracle's dense assembly, LU and GMRES
    times on the paper's level-3 sphere."""
    import oracle as O
    O.build()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    nrows, dt = _oracle_rows(O, m, chi_idx, n_phi, budget_s)
    rows_per_s = nrows / dt
    matvecs_per_s = rows_per_s / n_phi
    solves_per_s = matvecs_per_s / (iters + 1)
    out = {"value": solves_per_s, "unit": "solves/s", "cores": cores, "kind": "oracle",
           "sample": f"{nrows} of {n_phi} rows of one operator product ({dt:.1f} s), "
                     f"extrapolated to (1 + {iters}) products per solve ({iters} = Arnoldi steps of the "
                     f"float64 GMRES(30) solve of this workload to 1e-10 on the GPU)",
           "matvecs_per_s": matvecs_per_s}
    if extra_legs:
        if _omp_threads(1):
            n1, d1 = _oracle_rows(O, m, chi_idx, n_phi, budget_s / 4, seed=1)
            _omp_threads(cores)
            out["one_thread"] = {"matvecs_per_s": n1 / d1 / n_phi,
                                 "solves_per_s": n1 / d1 / n_phi / (iters + 1),
                                 "sample": f"{n1} rows ({d1:.1f} s), 1 thread",
                                 "parallel_speedup": rows_per_s / (n1 / d1)}
        out["small_problem"] = oracle_small_problem(O)
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    O.build()
    m, _, _ = workload(args.n)
    chi_idx, n_chi = O.chi_index(m.nodes, m.elems)
    n_phi = int(m.n_nodes)
    vals = []
    per = max(3.0, 60.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(m, chi_idx, n_phi, GMRES_ITERS_CUBE45, budget_s=per, extra_legs=False)
        if i >= args.warmup:
            vals.append(cb)
    v = statistics.median([c["value"] for c in vals])
    cb = dict(vals[-1])
    cb["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"cube{args.n}-tri6-laplace", "elements": int(m.n_elems), "nodes": int(n_phi),
                      "solver": "oracle matrix-free rows (CPU, FP64)", "l2": "n/a (CPU)"},
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def time_solves(bem, torch, mesh, stream, dev, prec, chi_d, phi_d, steps, warmup, flush, world, dist, leaf):
    """Device-timed steps (plan build + RHS product + GMRES) in one precision."""
    prm = bem.bem_fmm_params_default(p=10, leaf_size=leaf, eta=2.0, precision=prec)
    sp = bem.bem_solve_params_default(restart=30, tol=1e-10, max_iter=600)

    def step(mid=None):
        plan = bem.bem_plan_create(mesh, bem.BEM_LAPLACE, 0.0, prm, stream)
        if mid is not None:
            mid.record(stream)
        code, info = bem.bem_solve(plan, chi_d, phi_d, 1, sp, stream)
        return plan, info[0]

    for _ in range(warmup):
        plan, info = step()
        stream.synchronize()
        bem.bem_plan_destroy(plan)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = bem.bem_launch_count()
    total_ms, lat, setup_ms, infos = 0.0, [], [], []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, em, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        plan, info = step(em)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        total_ms += ms
        lat.append(ms)
        setup_ms.append(e0.elapsed_time(em))
        infos.append(info)
        bem.bem_plan_destroy(plan)
    torch.cuda.synchronize()
    launches = bem.bem_launch_count() - l0
    t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    max_ms = float(t.item())
    return {"value": world * steps / (max_ms / 1000.0), "ms_per_step": max_ms / steps, "lat": lat,
            "setup_ms": float(np.mean(setup_ms)), "solve_ms": float(np.mean(lat) - np.mean(setup_ms)),
            "infos": infos, "launches": int(launches), "prm": prm, "sp": sp}


def matvec_rate(bem, torch, mesh, stream, dev, prm, n_phi, flush):
    """Back-to-back A products of one built plan, per-stage times, counters."""
    plan = bem.bem_plan_create(mesh, bem.BEM_LAPLACE, 0.0, prm, stream)
    st = bem.bem_plan_stats(plan)
    x_d = torch.randn(n_phi, device=dev, dtype=torch.float64, generator=torch.Generator(device=dev).manual_seed(1))
    y_d = torch.empty_like(x_d)
    for _ in range(3):
        bem.bem_matvec(plan, bem.BEM_OP_A, x_d, y_d, stream)
    with torch.cuda.stream(stream):
        flush.zero_()
    nmv = 30
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(nmv):
        bem.bem_matvec(plan, bem.BEM_OP_A, x_d, y_d, stream)
    e1.record(stream)
    e1.synchronize()
    rate = nmv / (e0.elapsed_time(e1) / 1000.0)
    stages = bem.bem_plan_stage_times(plan, bem.BEM_OP_A, x_d, y_d, reps=10, stream=stream)
    setup_stages = bem.bem_plan_setup_times(plan)
    bem.bem_plan_destroy(plan)
    return rate, stages, setup_stages, st


def solver_compare(bem, torch, mesh, stream, dev, prm, chi_d, n_phi, reps=3):
    """GMRES and BiCGStab on one built plan (solve phase only, same RHS):
    solves/s, iterations, products per solve, and the distance between the
    two solutions."""
    plan = bem.bem_plan_create(mesh, bem.BEM_LAPLACE, 0.0, prm, stream)
    out, phis = {}, {}
    for name, method in (("gmres", bem.BEM_GMRES), ("bicgstab", bem.BEM_BICGSTAB)):
        sp = bem.bem_solve_params_default(restart=30, tol=1e-10, max_iter=600, method=method)
        phi = torch.empty(n_phi, device=dev, dtype=torch.float64)
        bem.bem_solve(plan, chi_d, phi, 1, sp, stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            code, info = bem.bem_solve(plan, chi_d, phi, 1, sp, stream)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        it = info[0].iters
        out[name] = {"solve_ms": ms, "solves_per_s": 1000.0 / ms, "iters": it, "restarts": info[0].restarts,
                     "products_per_solve": 1 + (it if method == bem.BEM_GMRES else 2 * it) + info[0].restarts,
                     "rel_residual": info[0].rel_residual}
        phis[name] = phi
    out["rel_diff_bicgstab_vs_gmres"] = float(torch.linalg.norm(phis["bicgstab"] - phis["gmres"]) /
                                              torch.linalg.norm(phis["gmres"]))
    bem.bem_plan_destroy(plan)
    return out


def serving(args):
    """The same Poisson request stream twice: the mixed form with continuous
    batching, then the plain float64 form one request at a time."""
    from paper_0908_0673_gb300 import bem
    from paper_0908_0673_gb300.serve import CudaEngine, Server, summarize, synthetic_stream
    reqs = synthetic_stream(args.serve_requests, rate_per_s=200.0, elems=(1000, args.serve_max_elems),
                            k_range=(1.0, args.serve_kmax), rhs=(1, 8), seed=0)
    out = {"stream": {"requests": len(reqs), "arrivals": "Poisson, 200 /s, seed 0",
                      "elements": f"log-uniform 1000-{args.serve_max_elems}, 6-node triangles",
                      "geometry": "geodesic sphere | ellipsoid (axes U[0.5,2]) | graded cube",
                      "green": f"50% Laplace, 50% Helmholtz k U[1,{args.serve_kmax:g}]", "rhs": "1-8 interior point sources",
                      "total_solves": sum(len(r.rhs) for r in reqs)}}
    # the whole stream in the mixed form; then the requests up to
    # serve_f64_max_elems elements (same arrival times) in both forms, for the
    # float64 comparison and the speedup on a common set
    sub = [r for r in reqs if r.mesh.n_elems <= args.serve_f64_max_elems]
    out["comparison_subset"] = {"requests": len(sub), "max_elems": args.serve_f64_max_elems,
                                "solves": sum(len(r.rhs) for r in sub)}
    phis = {}
    for name, prec, slots, threads, stream in (("mixed_continuous", bem.BEM_MIXED, 8, 2, reqs),
                                               ("mixed_subset", bem.BEM_MIXED, 8, 2, sub),
                                               ("f64_one_at_a_time", bem.BEM_F64, 1, 1, sub)):
        if not stream or (name == "mixed_subset" and len(sub) == len(reqs)):
            continue
        eng = CudaEngine(precision=prec, max_slots=slots)
        try:
            res = Server(eng, max_inflight=slots, setup_threads=threads, keep_phi=True).run(stream)
        finally:
            eng.close()
        out[name] = summarize(res)
        out[name]["largest_served_elems"] = max((r.n_elems for r in res if r.status in ("ok", "noconv")), default=0)
        bad = [r for r in res if r.status in ("error", "refused")]
        if bad:
            out[name]["failed"] = [{"request": r.rid, "elements": r.n_elems, "k": r.k, "status": r.status,
                                    "why": r.error[:200]} for r in bad[:6]]
        phis[name] = {r.rid: r.phi for r in res if r.phi is not None}
    errs = []
    for rid, ph in phis.get("mixed_continuous", {}).items():
        ref = phis.get("f64_one_at_a_time", {}).get(rid)
        if ref is None:
            continue
        for a, b in zip(ph, ref):
            errs.append(float(np.linalg.norm(a - b) / np.linalg.norm(b)))
    out["rel_err_vs_f64"] = {"max": max(errs) if errs else None,
                             "within_1e-5": int(sum(e <= 1e-5 for e in errs)), "solves": len(errs)}
    mx_sub = out.get("mixed_subset", out["mixed_continuous"] if len(sub) == len(reqs) else None)
    if mx_sub is not None and "f64_one_at_a_time" in out:
        out["speedup_solves_per_s"] = mx_sub["solves_per_s"] / out["f64_one_at_a_time"]["solves_per_s"]
    return out


def grouped(args):
    """Batched instances (meshes of uneven size, Laplace and Helmholtz, several
    right-hand sides each) in the mixed form: plans built, then every
    right-hand-side round solved as one group (one graph launch per restart
    cycle for all members), against the same solves one at a time; each
    solution checked against the instance's own float64 solution."""
    import torch
    from paper_0908_0673_gb300 import bem, tune
    from paper_0908_0673_gb300 import inputs as I
    rng = np.random.default_rng(0)
    n_inst = args.group
    insts = []
    for i in range(n_inst):
        E = rng.uniform(args.group_min_elems, args.group_max_elems)
        kind = int(rng.integers(0, 3))
        if kind == 2:
            m = I.cube(max(2, int(round(math.sqrt(E / 12.0)))), I.TRI6, seed=i)
            rmax = 0.3
        else:
            axes = (1.0, 1.0, 1.0) if kind == 0 else tuple(rng.uniform(0.5, 2.0, 3))
            m = I.geodesic(max(2, int(round(math.sqrt(E / 20.0)))), I.TRI6, axes=axes)
            rmax = 0.3 * min(axes)
        helm = rng.uniform() < 0.5
        k = float(rng.uniform(1.0, args.group_kmax)) if helm else 0.0
        nr = int(rng.integers(1, args.group_max_rhs + 1))
        srcs = []
        for _ in range(nr):
            d = rng.standard_normal(3)
            srcs.append(d / np.linalg.norm(d) * rmax * rng.uniform() ** (1.0 / 3.0))
        insts.append((m, bem.BEM_HELMHOLTZ if helm else bem.BEM_LAPLACE, k, srcs))
    ctx = bem.bem_ctx_create(0)
    sp = bem.bem_solve_params_default(restart=30, tol=1e-10, max_iter=600)

    def build(prec):
        # the float64 references share the mixed form's tree (same leaf size),
        # so that they differ in precision only
        out = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for m, green, k, srcs in insts:
            mh = bem.bem_mesh_create(ctx, m.nodes, m.elems, m.elem_type)
            n_phi, n_chi = bem.bem_mesh_sizes(mh)
            idx = bem.bem_mesh_chi_index(mh, m.n_elems, m.npe)
            prm = tune.choose(m.n_elems, green, bem.BEM_MIXED)
            prm["precision"] = prec
            plan = bem.bem_plan_create(mh, green, k, bem.bem_fmm_params_default(**prm))
            cplx = green == bem.BEM_HELMHOLTZ
            chis = []
            for x in srcs:
                ce = I.helmholtz_point_source(m, x, k)[1] if cplx else I.point_source(m, x)[1]
                c = np.zeros(n_chi, np.complex128 if cplx else np.float64)
                c[idx.ravel()] = np.asarray(ce).ravel()
                chis.append(torch.tensor(c, device="cuda"))
            out.append((mh, plan, n_phi, chis))
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    mx, t_build = build(bem.BEM_MIXED)
    nrhs_max = max(len(s[3]) for s in insts)
    total = sum(len(s[3]) for s in insts)
    group = bem.bem_group_create(ctx, [pl for _, pl, _, _ in mx])
    phis_g = [[torch.empty(npp, device="cuda", dtype=ch[0].dtype) for _ in ch] for _, _, npp, ch in mx]
    # first call captures the graphs: time it apart from the solves
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bem.bem_group_solve(group, [ch[0] for *_, ch in mx], [p[0] for p in phis_g], sp)
    torch.cuda.synchronize()
    t_first = time.perf_counter() - t0
    t0 = time.perf_counter()
    iters, launches, nconv = [], 0, 0
    for r in range(nrhs_max):
        chis = [ch[r] if r < len(ch) else None for *_, ch in mx]
        outs = [p[r] if r < len(p) else None for p in phis_g]
        code, infos, nl = bem.bem_group_solve(group, chis, outs, sp)
        launches += nl
        iters += [inf.iters for inf, c in zip(infos, chis) if c is not None]
        nconv += sum(1 for inf, c in zip(infos, chis) if c is not None and inf.status != bem.BEM_OK)
    torch.cuda.synchronize()
    t_group = time.perf_counter() - t0
    # the same solves one at a time
    t0 = time.perf_counter()
    for (mh, pl, npp, ch) in mx:
        for c in ch:
            out = torch.empty(npp, device="cuda", dtype=c.dtype)
            bem.bem_solve(pl, c, out, 1, sp)
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    bem.bem_group_destroy(group)
    # float64 references (not timed): the first group_f64_rhs right-hand sides
    # of every instance, each instance's float64 plan built and released in turn
    for mh, pl, _, _ in mx:
        bem.bem_plan_destroy(pl)
    errs, worst = [], []
    for i, (mh, _, npp, ch) in enumerate(mx):
        m, green, k, _s = insts[i]
        prm = tune.choose(m.n_elems, green, bem.BEM_MIXED)
        prm["precision"] = bem.BEM_F64
        pl = bem.bem_plan_create(mh, green, k, bem.bem_fmm_params_default(**prm))
        for c, pg in list(zip(ch, phis_g[i]))[:max(0, args.group_f64_rhs)]:
            out = torch.empty(npp, device="cuda", dtype=c.dtype)
            bem.bem_solve(pl, c, out, 1, sp)
            a, b = pg.cpu().numpy(), out.cpu().numpy()
            errs.append(float(np.linalg.norm(a - b) / np.linalg.norm(b)))
            worst.append((errs[-1], {"instance": i, "mesh": m.name, "elements": int(m.n_elems),
                                     "green": "helmholtz" if green == bem.BEM_HELMHOLTZ else "laplace", "k": k,
                                     "rel_err": errs[-1]}))
        bem.bem_plan_destroy(pl)
    worst = [w for _, w in sorted(worst, key=lambda t: -t[0])[:4]]
    for mh, _, _, _ in mx:
        bem.bem_mesh_destroy(mh)
    bem.bem_ctx_destroy(ctx)
    return {"instances": n_inst, "elements": f"uniform {args.group_min_elems}-{args.group_max_elems}, 6-node triangles",
            "geometry": "geodesic sphere | ellipsoid (axes U[0.5,2]) | graded cube",
            "green": f"50% Laplace, 50% Helmholtz k U[1,{args.group_kmax:g}]",
            "rhs": f"1-{args.group_max_rhs} interior point sources", "total_solves": total,
            "total_elements": int(sum(s[0].n_elems for s in insts)),
            "build_s": t_build, "first_call_with_capture_s": t_first,
            "group": {"solves_per_s": total / t_group, "seconds": t_group, "graph_kernels": int(launches)},
            "one_at_a_time": {"solves_per_s": total / t_single, "seconds": t_single},
            "speedup": t_single / t_group, "gmres_iters_mean": float(np.mean(iters)),
            "gmres_iters_max": int(max(iters)), "not_converged": int(nconv),
            "rel_err_vs_own_f64": {"max": max(errs), "within_1e-5": int(sum(e <= 1e-5 for e in errs)), "solves": len(errs),
                                   "checked": f"first {args.group_f64_rhs} right-hand side(s) of every instance",
                                   "worst": worst}}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps(grouped(args) if args.only == "grouped" else serving(args)))
        return
    import torch
    import torch.distributed as dist
    from paper_0908_0673_gb300 import bem

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    prec = bem.BEM_MIXED if args.precision == "mixed" else bem.BEM_F64

    m, phi_ex, chi_e = workload(args.n)
    ctx = bem.bem_ctx_create(local)
    mesh = bem.bem_mesh_create(ctx, m.nodes, m.elems, bem.BEM_TRI6)
    n_phi, n_chi = bem.bem_mesh_sizes(mesh)
    chi_idx = bem.bem_mesh_chi_index(mesh, m.n_elems, 6)
    chi = chi_vector(chi_idx, n_chi, chi_e)
    bem.bem_mesh_upload(mesh, stream)
    chi_d = torch.tensor(chi, device=dev, dtype=torch.float64)
    phi_d = torch.empty(n_phi, device=dev, dtype=torch.float64)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev, dtype=torch.float32)   # > 129 MB L2

    from paper_0908_0673_gb300 import tune
    leaf = args.leaf or tune.choose(int(m.n_elems), bem.BEM_LAPLACE, prec)["leaf_size"]
    leaf64 = args.leaf or tune.choose(int(m.n_elems), bem.BEM_LAPLACE, bem.BEM_F64)["leaf_size"]
    clocks = Clocks(local)
    main_run = time_solves(bem, torch, mesh, stream, dev, prec, chi_d, phi_d, args.steps, args.warmup, flush,
                           world, dist, leaf)
    clk = clocks.stop()
    phi = phi_d.cpu().numpy()
    eps_rms = float(np.sqrt(np.mean((phi - phi_ex) ** 2)))
    prm, sp, infos = main_run["prm"], main_run["sp"], main_run["infos"]

    # the plain float64 form on the same workload, for comparison
    other = None
    if prec == bem.BEM_MIXED and not args.no_f64:
        phi64_d = torch.empty_like(phi_d)
        f = time_solves(bem, torch, mesh, stream, dev, bem.BEM_F64, chi_d, phi64_d, max(1, min(args.steps, 3)),
                        1, flush, world, dist, leaf64)
        phi64 = phi64_d.cpu().numpy()
        mv64 = matvec_rate(bem, torch, mesh, stream, dev, f["prm"], n_phi, flush)
        other = {"solves_per_s": f["value"], "ms_per_step": f["ms_per_step"], "setup_ms": f["setup_ms"],
                 "solve_ms": f["solve_ms"], "gmres_iters": [i.iters for i in f["infos"]], "matvecs_per_s": mv64[0],
                 "stage_ms": mv64[1], "steps": max(1, min(args.steps, 3)), "warmup": 1, "leaf_size": leaf64,
                 "rel_err_of_mixed_solution": float(np.linalg.norm(phi - phi64) / np.linalg.norm(phi64))}

    matvecs_per_s, stages, setup_stages, st = matvec_rate(bem, torch, mesh, stream, dev, prm, n_phi, flush)

    # roofline of the dominant kernel
    dom = max(stages, key=stages.get)
    kind = 0 if prec == bem.BEM_MIXED else 1
    peak = bem.bem_measure_peak(kind, stream)
    if dom == "near_l2p":
        flops = st["near_pairs"] * FLOPS_PER_PAIR["A"]
        achieved = flops / (stages[dom] * 1e-3) / 1e12
        roof = {"kernel": "k_near_f32 (near-field regular quadrature + L2P)" if kind == 0 else
                "k_near (near-field regular quadrature + L2P)", "bound": "alu",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": ncu_traffic("near_l2p") if kind == 0 else None, "traffic_unit": "bytes per launch",
                "peak_source": f"measured {'FP32' if kind == 0 else 'FP64'} FMA throughput (bem_measure_peak)",
                "work": f"{st['near_pairs']} target-source pairs x {FLOPS_PER_PAIR['A']:.0f} flops"}
    elif dom == "m2l":
        cpp6 = math.comb(10 + 6, 6)
        flops = st["n_inter"] * 2.0 * cpp6
        achieved = flops / (stages[dom] * 1e-3) / 1e12
        roof = {"kernel": "k_m2l (multipole-to-local, Tausch derivatives + contraction)", "bound": "alu",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": f"measured {'FP32' if kind == 0 else 'FP64'} FMA throughput (bem_measure_peak)",
                "work": f"{st['n_inter']} interaction pairs x 2 x C(p+6,6)={cpp6} flops (algorithmic, p=10)"}
    else:
        roof = {"kernel": dom, "bound": "alu", "achieved": None, "peak": peak, "unit": "TFLOP/s", "frac": None,
                "traffic": None}

    m2l_tensor = None
    if prec == bem.BEM_MIXED:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
        tf32 = 0.5 * peaks["bf16_tflops"]
        t = stages["m2l"] * 1e-3
        alg = st["n_inter"] * 2.0 * math.comb(10 + 6, 6) / t / 1e12
        issued = st["n_inter"] * 3 * 2.0 * tc_issued_macs(10) / t / 1e12
        m2l_tensor = {"kernel": "k_m2l_permute + k_m2l_tc + k_m2l_gather_sym (tcgen05 kind::tf32, hi/lo split, 3 products)",
                      "bound": "tensor", "unit": "TFLOP/s", "peak": tf32,
                      "peak_source": "TF32 = 0.5 x measured BF16 (MEASURED_PEAKS.json, nominal ratio)",
                      "achieved_algorithmic": alg, "frac_algorithmic": alg / tf32,
                      "achieved_issued": issued, "frac_issued": issued / tf32,
                      "stage_ms": stages["m2l"], "traffic": ncu_traffic("m2l"),
                      "traffic_unit": "DRAM bytes per M2L stage (permute + tcgen05 + gather launches)",
                      "work": f"{st['n_inter']} pairs x 2 x C(16,6) algorithmic; x 3 x {tc_issued_macs(10)} MACs issued"}

    # end to end through the public API from pinned host buffers
    nodes_h = torch.from_numpy(np.ascontiguousarray(m.nodes)).pin_memory()
    elems_h = torch.from_numpy(np.ascontiguousarray(m.elems)).pin_memory()
    chi_h = torch.from_numpy(chi).pin_memory()
    phi_h = torch.empty(n_phi, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for i in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mh = bem.bem_mesh_create(ctx, nodes_h.numpy(), elems_h.numpy(), bem.BEM_TRI6)
        plan = bem.bem_plan_create(mh, bem.BEM_LAPLACE, 0.0, prm, stream)
        with torch.cuda.stream(stream):
            c_d = chi_h.to(dev, non_blocking=True)
            p_d = torch.empty(n_phi, device=dev, dtype=torch.float64)
        bem.bem_solve(plan, c_d, p_d, 1, sp, stream)
        with torch.cuda.stream(stream):
            phi_h.copy_(p_d, non_blocking=True)
        stream.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1000.0)
        bem.bem_plan_destroy(plan)
        bem.bem_mesh_destroy(mh)
    h2d = nodes_h.numel() * 8 + 2 * elems_h.numel() * 4 + chi_h.numel() * 8
    d2h = phi_h.numel() * 8
    e2e_value = world * 1000.0 / statistics.mean(e2e_ms)

    iters = [i.iters for i in infos]
    lat = main_run["lat"]
    out = {
        "metric": METRIC, "value": main_run["value"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main_run["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == bem.BEM_MIXED else "f64", "data": "synthetic",
        "config": {"workload": f"cube{args.n}-tri6-laplace", "elements": int(m.n_elems), "nodes": int(n_phi), "chi": int(n_chi),
                   "p": 10, "leaf_size": leaf, "leaf_size_source": "argument" if args.leaf else "autotuner table",
                   "eta": 2.0, "precision": args.precision, "gmres": "restart 30, tol 1e-10",
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}",
                   "step": "device plan build + RHS product + GMRES solve"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "setup_ms": main_run["setup_ms"], "solve_ms": main_run["solve_ms"],
        "gmres_iters": iters, "rel_residual": infos[-1].rel_residual if infos else None,
        "eps_rms_vs_point_source": eps_rms,
        "matvecs_per_s": matvecs_per_s, "stage_ms": stages, "setup_stage_ms": setup_stages, "plan_stats": st,
        "roofline": roof, "m2l_tensor": m2l_tensor, "clocks": clk, "gpu_launches": main_run["launches"],
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
    }
    if other is not None:
        out["f64_form"] = other
    if rank == 0 and world == 1:
        out["solvers"] = solver_compare(bem, torch, mesh, stream, dev, prm, chi_d, n_phi)
    if rank == 0 and world == 1 and args.serve_requests > 0:
        out["serving"] = serving(args)
    if rank == 0 and world == 1 and args.group > 0:
        out["grouped"] = grouped(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(m, chi_idx, n_phi, GMRES_ITERS_CUBE45)
    if rank == 0:
        print(json.dumps(out))
    bem.bem_mesh_destroy(mesh)
    bem.bem_ctx_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
