#!/usr/bin/env python
"""Throughput of the SSP-RK3 step of the Hermite finite-difference method on one GB300.

Workload (default): the 2D four-quadrant Riemann problem on a 1024 x 1024 jittered, randomly
split triangulation of the unit square with 5 transmissive ghost layers (1,048,576 physical
vertices, 1,069,156 stored, ~3.2 M flux edges), device CFL time step (CFL 0.3).  Synthetic
seeded inputs (synth/), no dataset.

Metric: vertex-stage updates per second = physical vertices x 3 RK stages x steps / time.
The primary line is the FP64 path; the FP32-bulk path is timed in the same run and reported
under "variants".  Per-kernel times come from CUDA events around every launch in a second pass
of the same steps (hfd_steps_profiled); the roofline object describes the dominant kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--n 1024]

--impl reference times the FP64 CPU oracle (the reference arm of this comparison) on a bounded
patch of the same workload on one host core.  The default line's cpu_baseline reports the same
oracle on one core and, under "all_cores", one oracle process per host core at once.

Other workloads (--workload): batched, adjoint, tgv, conservative, circular-sod, vortex-order.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "vertex-stage updates/s"
CPU_PATCH_N = 32                 # bounded oracle sample: 32 x 32 patch of the same workload
# DRAM bytes (read + write) per launch of each kernel on the default 1024 x 1024 workload, from
# one ncu capture per kernel (one launch, one-pass metrics; profiles/traffic_four_quadrant_1024x1024.md),
# valid for the kernel and data-layout sources they were taken on: when either file's hash
# differs the figures are stale and the line reports traffic as null
TRAFFIC_SOURCES = ("paper_2109_01286_gb300/csrc/kernels.cu", "paper_2109_01286_gb300/csrc/api.cu")
TRAFFIC_SHA = "40d96e012190e243"
DRAM_TRAFFIC_1024 = {"k_div<double>": 3263.0e6, "k_div<float>": 1795.1e6, "k_div_df": 2923.6e6}


def sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-div", default="plain", choices=["plain", "folded"],
                    help="arithmetic of the FP64 divergence (hfd_mesh_set_fp64_div)")
    ap.add_argument("--fp32-div", default="unstaged", choices=["unstaged", "staged", "gathers"],
                    help="divergence kernel of the FP32-bulk path (hfd_mesh_set_div_staged)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the bounded batched / adjoint / Taylor-Green passes of the default line")
    ap.add_argument("--workload", default="four-quadrant",
                    choices=["four-quadrant", "batched", "adjoint", "tgv", "conservative", "couette",
                             "circular-sod", "vortex-order", "three-d"],
                    help="batched: 256 uneven isentropic-vortex meshes advanced together; "
                         "adjoint: gradient of a 200-step vortex run, checked by differences; "
                         "conservative: the four-quadrant line with median-dual value rows; "
                         "circular-sod: Sec. 3.3 on embedded-circle Delaunay meshes; "
                         "vortex-order: Sec. 3.1 density error at 50-150 segments per side; "
                         "three-d: the 3D extension on an n^3 tetrahedral box (--n, default 40 "
                         "for this workload)")
    ap.add_argument("--directions", type=int, default=64)
    ap.add_argument("--batch", type=int, default=256)
    return ap.parse_args()


def workload(n):
    mesh = synth.jittered_box_with_ghosts(n, n, (0.0, 1.0), (0.0, 1.0), 5, seed=2)
    return mesh, synth.four_quadrant(mesh)


def workload_name(n):
    return f"four-quadrant Riemann, {n}x{n} jittered random-split mesh, 5 ghost layers"


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, val in zip(names, r[5:9]):
                    if val.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ roofline bookkeeping
def algorithmic_costs(stats, T):
    """Algorithmic bytes and FP64/FP32 flops of one launch of each kernel (one RK stage), from
    the mesh's actual sizes.  T = bytes of the bulk type.  Per-unit figures:
      vertex : 96 B state read + 12T AoS copy + 8T fluxes written, ~30 flop  per vertex
      edge   : 24 B stencil + 2T normal + 48T weights + 4T flux written     per flux edge,
               + 12T state copy read once per vertex; 480 bulk-precision flop per edge on the
               smooth branch (5-node sums in conservative variables 240, Roe flux ~200, end-state
               differences 24, positivity 12; a division or square root counts as one flop)
      div    : 8 B row pointers + (4 B + 6T) per stencil vertex + (4 B + 3T) per stencil edge
               + 96 B stage state + 96 B base state (2 of 3 stages) + 96 B written per vertex,
               + 8T fluxes per vertex and 4T per edge read once; 48 flop per stencil vertex,
               24 per stencil edge, 48 for the stage update."""
    V, A, Ef = stats["nv"], stats["nactive"], stats["nflux_edges"]
    nv, ne = stats["div_nv_total"], stats["div_ne_total"]
    return {
        "vertex": {"bytes": V * (96 + 20 * T), "flops": 30 * V},
        "edge": {"bytes": Ef * (24 + 54 * T) + V * 12 * T, "flops": 480 * Ef},
        "div": {"bytes": A * (8 + 96 * (1 + 2.0 / 3.0) + 96) + nv * (4 + 6 * T) + ne * (4 + 3 * T)
                + V * 8 * T + Ef * 4 * T, "flops": 48 * nv + 24 * ne + 48 * A},
        "ghost": {"bytes": (V - A) * (12 + 96 + 96), "flops": 0},
    }


def fma_peaks():
    """FP64 and FP32 FMA throughput of this device, measured by the library's hand-written FMA
    loops (hfd_measure_fma_peaks) at the clocks it runs now, before any timed region."""
    from paper_2109_01286_gb300 import measure_fma_peaks
    m = measure_fma_peaks()
    return {"fp64_tflops": m["fp64_flops"] / 1e12, "fp32_tflops": m["fp32_flops"] / 1e12,
            "sm_count": m["sm_count"],
            "source": f"measured: hand-written FP64 FMA loop on all {m['sm_count']} SMs "
                      "(hfd_measure_fma_peaks), best of 3 launches"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ CPU oracle timing
def time_oracle(seconds=12.0, steps=None, warmup=0):
    """Times the FP64 oracle's SSP-RK3 step on a bounded patch of the workload; returns
    (vertex-stage/s, effective cores, sample description, per-step seconds list)."""
    import oracle
    mesh, U = workload(CPU_PATCH_N)
    P = oracle.prepare(mesh)
    A = len(P.active)
    dt = 0.5 * oracle.cfl_dt(mesh, P, U)
    # every timed step advances the initial state, as on the GPU (the state of this shock
    # problem turns non-finite within a few steps of the method as read)
    for _ in range(warmup):
        oracle.step(mesh, P, U, dt)
    times = []
    c0, w0 = time.process_time(), time.perf_counter()
    while True:
        t = time.perf_counter()
        oracle.step(mesh, P, U, dt)
        times.append(time.perf_counter() - t)
        if steps is not None and len(times) >= steps:
            break
        if steps is None and time.perf_counter() - w0 > seconds:
            break
    cores = (time.process_time() - c0) / max(time.perf_counter() - w0, 1e-9)
    value = A * 3 * len(times) / sum(times)
    sample = (f"oracle SSP-RK3 steps on a {CPU_PATCH_N}x{CPU_PATCH_N} patch of the same workload "
              f"({A} physical vertices, 5 ghost layers), {len(times)} steps, each from the "
              f"initial state")
    return value, max(1, round(cores)), sample, times


def _oracle_worker(seconds):
    """One all-cores worker: the oracle timed as above, with the wall-clock window of its timed
    steps (for the union over the workers)."""
    t0 = time.time()
    v, _, _, times = time_oracle(seconds=seconds)
    t1 = time.time()
    return v * sum(times), t1 - sum(times), t1, len(times)


def time_oracle_all_cores(seconds=8.0):
    """The same oracle steps in one process per host core, all at once (the oracle is
    single-threaded numpy): total vertex-stages over the union of the workers' timed windows.
    A spawn pool, because the calling process may hold a CUDA context."""
    import multiprocessing as mp
    n = len(os.sched_getaffinity(0))
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    pool = mp.get_context("spawn").Pool(n)
    try:
        # bounded: workers that cannot start (or hang) must not hold the bench
        res = pool.map_async(_oracle_worker, [seconds] * n).get(timeout=4 * seconds + 120)
    finally:
        pool.terminate()
        pool.join()
    work = sum(r[0] for r in res)
    window = max(r[2] for r in res) - min(r[1] for r in res)
    return work / window, n, sum(r[3] for r in res)


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    value, cores, sample, times = time_oracle(steps=args.steps, warmup=args.warmup)
    ms = 1000.0 * sum(times) / len(times)
    line = {
        "metric": METRIC, "value": value, "unit": "vertex-stage/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": workload_name(CPU_PATCH_N) + " (bounded CPU sample)",
                   "precision": "fp64", "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "vertex-stage/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "vertex-stage/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ native arm
def run_native(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2109_01286_gb300 import Prep, replicas
    mesh, U = workload(args.n)
    t0 = time.perf_counter()
    conservative = args.workload == "conservative"
    prep = Prep(mesh, conservative=conservative)
    prep_s = time.perf_counter() - t0
    U_dev = torch.from_numpy(U).cuda()
    stream = torch.cuda.current_stream()
    results = {}
    clocks_main = None
    peak_hbm, peak_src = load_peaks()
    fpk = fma_peaks()
    for prec in ("fp64", "fp32"):
        dm = prep.upload(prec)
        if prec == "fp32" and args.fp32_div == "staged":
            dm.set_div_staged(1)
        if prec == "fp32" and args.fp32_div == "gathers":
            dm.set_div_staged(2)
        if prec == "fp64" and args.fp64_div == "folded":
            dm.set_fp64_div(1)
        st = dm.stats_dict()
        Ui = dm.import_state(U_dev)
        # Every timed step advances the initial state of the workload: the method as read here
        # is unstable on this problem and its state turns non-finite within a few steps, after
        # which the sensor takes its re-decision path everywhere.  The device copy that resets
        # the state is inside the timed region.
        X = torch.empty_like(Ui)
        for _ in range(args.warmup):
            X.copy_(Ui)
            dm.steps(X, 0.0, 1)
        torch.cuda.synchronize()
        barrier()
        clk = Clocks(local) if prec == "fp64" else None
        if clk:
            clk.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            X.copy_(Ui)
            dm.steps(X, 0.0, 1)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        if clk:
            clocks_main = clk.stop()
        A = st["nactive"]
        value, _, ms = replicas.whole_job_rate(A * 3 * args.steps, ev0.elapsed_time(ev1), dist,
                                               device="cuda")
        finite = True
        try:
            dm.check()
        except Exception:
            finite = False
        # second pass: the same steps launched kernel by kernel with events
        kms = {k: 0.0 for k in ("ghost", "vertex", "edge", "div", "dt")}
        nl = 0
        for _ in range(args.steps):
            X.copy_(Ui)
            km, n = dm.steps_profiled(X, 0.0, 1)
            nl += n
            for k in kms:
                kms[k] += km[k]
        T = 8 if prec == "fp64" else 4
        costs = algorithmic_costs(st, T)
        launches_per_kind = {"vertex": 3 * args.steps, "edge": 3 * args.steps,
                             "div": 3 * args.steps, "ghost": 4 * args.steps}
        kern = {}
        for k in ("vertex", "edge", "div", "ghost"):
            n = launches_per_kind[k]
            avg_s = kms[k] / 1000.0 / n
            kern[k] = {"ms_total": kms[k], "launches": n, "avg_ms": 1000 * avg_s,
                       "share": kms[k] / max(sum(kms.values()), 1e-12),
                       "gbs": costs[k]["bytes"] / avg_s / 1e9,
                       "tflops": costs[k]["flops"] / avg_s / 1e12}
        results[prec] = {"ms": ms, "value": value, "finite": finite, "kernels": kern,
                         "profiled_ms": sum(kms.values()), "launches": nl, "stats": st}
        # one step from the initial state, for the FP32-bulk vs FP64 comparison
        X.copy_(Ui)
        dm.step(X, 0.0)
        results[prec]["one_step"] = dm.export_state(X)[0:4].cpu().numpy()
        # the FP64 divergence in its folded double-float form (hfd_mesh_set_fp64_div), the same
        # steps from the initial state
        if prec == "fp64" and not args.no_variants and args.fp64_div == "plain":
            dm.set_fp64_div(1)
            for _ in range(args.warmup):
                X.copy_(Ui)
                dm.steps(X, 0.0, 1)
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(args.steps):
                X.copy_(Ui)
                dm.steps(X, 0.0, 1)
            ev1.record(stream)
            torch.cuda.synchronize()
            fv, _, fms = replicas.whole_job_rate(A * 3 * args.steps, ev0.elapsed_time(ev1), dist,
                                                 device="cuda")
            fk = {k: 0.0 for k in ("ghost", "vertex", "edge", "div", "dt")}
            for _ in range(args.steps):
                X.copy_(Ui)
                km, _ = dm.steps_profiled(X, 0.0, 1)
                for k in fk:
                    fk[k] += km[k]
            X.copy_(Ui)
            R_f = dm.residual(X.clone())
            dm.set_fp64_div(0)
            R_p = dm.residual(X.clone())
            rel = float(torch.linalg.norm(R_f - R_p) / torch.linalg.norm(R_p))
            results[prec]["folded"] = {
                "value": fv, "ms_per_step": fms / args.steps,
                "kernel_avg_ms": {k: fk[k] / (3 * args.steps) for k in ("vertex", "edge", "div")},
                "residual_rel_l2_vs_plain": rel,
                "form": "FP64 divergence with edge-row endpoint averages folded into the vertex "
                        "rows, centre-vertex differences in FP64, products in double-float on the "
                        "FP32 pipe (hfd_mesh_set_fp64_div(1))"}
        # the same steps timed from a developed state: the state after two steps (the method's
        # growth makes later states of this problem inadmissible), with the branch mix of both
        if not args.no_variants:
            D = Ui.clone()
            dm.steps(D, 0.0, 2)
            torch.cuda.synchronize()
            finite2 = bool(torch.isfinite(D).all())
            weno = {"initial": int(np.unpackbits(dm.edge_branches(Ui)).sum()),
                    "after_2_steps": int(np.unpackbits(dm.edge_branches(D)).sum())}
            for _ in range(args.warmup):
                X.copy_(D)
                dm.steps(X, 0.0, 1)
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(args.steps):
                X.copy_(D)
                dm.steps(X, 0.0, 1)
            ev1.record(stream)
            torch.cuda.synchronize()
            dv, _, dms = replicas.whole_job_rate(A * 3 * args.steps, ev0.elapsed_time(ev1), dist,
                                                 device="cuda")
            results[prec]["developed"] = {
                "value": dv, "ms_per_step": dms / args.steps, "state_finite": finite2,
                "weno_sides_and_components": weno,
                "step_input": "every timed step advances the state after two steps"}
        if prec == "fp64":
            e2e = None
            if not args.no_e2e:
                hin = torch.from_numpy(U.copy()).pin_memory()
                hout = torch.empty_like(hin).pin_memory()
                dm.steps_host(hin, hout, 0.0, 1)         # warm the e2e buffers and graph
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    dm.steps_host(hin, hout, 0.0, 1)
                e1.record(stream)
                torch.cuda.synchronize()
                barrier()
                ev, _, ems = replicas.whole_job_rate(A * 3 * args.steps, e0.elapsed_time(e1), dist,
                                                     device="cuda")
                nbytes = hin.numel() * 8
                e2e = {"value": ev, "unit": "vertex-stage/s",
                       "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                       "ms_per_step": ems / args.steps}
            results[prec]["e2e"] = e2e
        del dm
        torch.cuda.empty_cache()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    r = results["fp64"]
    dom = max(r["kernels"], key=lambda k: r["kernels"][k]["share"])
    kd = r["kernels"][dom]
    fresh = TRAFFIC_SHA is not None and sources_sha() == TRAFFIC_SHA

    def traffic(name):
        return DRAM_TRAFFIC_1024.get(name) if (args.n == 1024 and fresh) else None

    def dram(name, avg_ms):
        # the % of HBM by DRAM bytes: measured bytes per launch over the live launch time
        t = traffic(name)
        return (None, None) if t is None else (t / (avg_ms / 1000.0) / 1e9, t / (avg_ms / 1000.0) / 1e9 / peak_hbm)
    roof = {"kernel": f"k_{dom}<double>", "bound": "alu", "achieved": kd["tflops"],
            "peak": fpk["fp64_tflops"], "unit": "TFLOP/s",
            "frac": kd["tflops"] / fpk["fp64_tflops"], "traffic": traffic(f"k_{dom}<double>"),
            "traffic_unit": "bytes per launch (ncu DRAM read + write)",
            "peak_source": fpk["source"],
            "hbm_gbs": kd["gbs"], "hbm_frac": kd["gbs"] / peak_hbm,
            "dram_gbs": dram(f"k_{dom}<double>", kd["avg_ms"])[0],
            "dram_frac": dram(f"k_{dom}<double>", kd["avg_ms"])[1],
            "hbm_peak_source": peak_src}
    folded = r.get("folded")
    if folded is not None:
        folded["div_traffic"] = traffic("k_div_df")
        folded["div_dram_gbs"] = dram("k_div_df", folded["kernel_avg_ms"]["div"])[0]
    f32 = results["fp32"]
    dom32 = max(f32["kernels"], key=lambda k: f32["kernels"][k]["share"])
    k32 = f32["kernels"][dom32]
    line = {
        "metric": METRIC, "value": r["value"], "unit": "vertex-stage/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args.n) + (", conservative variant (median-dual "
                                                        "value rows)" if conservative else ""),
                   "precision": "fp64",
                   "step_input": "every timed step advances the initial state (device reset "
                                 "copy inside the timed region)",
                   "physical_vertices": r["stats"]["nactive"], "stored_vertices": r["stats"]["nv"],
                   "flux_edges": r["stats"]["nflux_edges"], "time_step": "device CFL 0.3",
                   "l2": "no flush: per-stage working set (state, coefficients) is several GB, "
                         "far larger than the 129 MB L2",
                   "parallelism": f"replicas x{world}", "prep_seconds": prep_s},
        "roofline": roof,
        "kernels_fp64": r["kernels"],
        "variants": {"fp32_bulk": {
            "value": f32["value"], "ms_per_step": f32["ms"] / args.steps, "dtype": "f32",
            "state_finite": f32["finite"],
            "roofline": {"kernel": f"k_{dom32}<float>", "bound": "hbm", "achieved": k32["gbs"],
                         "peak": peak_hbm, "unit": "GB/s", "frac": k32["gbs"] / peak_hbm,
                         "traffic": traffic(f"k_{dom32}<float>"),
                         "traffic_unit": "bytes per launch (ncu DRAM read + write)",
                         "dram_gbs": dram(f"k_{dom32}<float>", k32["avg_ms"])[0],
                         "dram_frac": dram(f"k_{dom32}<float>", k32["avg_ms"])[1],
                         "peak_source": peak_src},
            "kernels": f32["kernels"]}},
        "state_finite": r["finite"],
        "developed_state": {"fp64": r.get("developed"), "fp32_bulk": f32.get("developed")},
        "fp64_folded_divergence": folded,
        "fma_peaks": fpk,
        "gpu_launches": int(r["launches"]),
        "e2e": r.get("e2e"),
        "clocks": clocks_main,
    }
    # FP32-bulk against FP64 after one step from the same state: per-variable relative L1 over
    # the physical vertices, and over those at least 0.05 away from the initial discontinuities
    a64, a32 = results["fp64"]["one_step"], results["fp32"]["one_step"]
    xm, ym = mesh["x"], mesh["y"]
    phys = np.ones(len(xm), bool)
    phys[mesh["ghost_ids"]] = False
    away = phys & (np.abs(xm - 0.5) > 0.05) & (np.abs(ym - 0.5) > 0.05)
    def rl1(mask):
        return [float(np.abs(a32[q, mask] - a64[q, mask]).sum() / np.abs(a64[q, mask]).sum())
                for q in range(4)]
    line["fp32_vs_fp64_one_step_rel_l1"] = {"variables": ["rho", "rho u", "rho v", "E"],
                                            "all": rl1(phys), "away_from_discontinuities": rl1(away)}
    if args.gpus == 1 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample, _ = time_oracle()
        line["cpu_baseline"] = {"value": v, "unit": "vertex-stage/s", "cores": cores,
                                "kind": "oracle", "sample": sample}
        try:
            va, na, steps = time_oracle_all_cores()
            line["cpu_baseline"]["all_cores"] = {
                "value": va, "unit": "vertex-stage/s", "cores": na,
                "sample": f"the same patch stepped by {na} oracle processes at once, "
                          f"{steps} steps in all, over the union of their timed windows"}
        except Exception as e:                        # the single-core figure stands alone
            line["cpu_baseline"]["all_cores"] = {"unavailable": str(e)[:200]}
    if not args.no_variants:
        # bounded passes of the batched, adjoint and viscous configurations (after the timed
        # regions of the line's own workload)
        for key, fn in (("batched_subset", lambda: variant_batched(fpk, steps=min(args.steps, 10))),
                        ("adjoint_cost", variant_adjoint), ("tgv_mixed_precision", variant_tgv),
                        ("three_d", lambda: variant_3d(fpk, peak_hbm, steps=min(args.steps, 10)))):
            try:
                line["variants"][key] = fn()
            except Exception as e:                    # reported, never fatal to the line
                line["variants"][key] = {"error": str(e)[:300]}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ short variants of the other configs
def variant_batched(fpk, members_n=32, steps=10, warmup=3):
    """A bounded pass of the batched configuration in the default line: the first `members_n`
    of the 256 uneven isentropic-vortex meshes (host preprocessing of all 256 takes minutes;
    --workload batched runs them all)."""
    from paper_2109_01286_gb300 import Prep
    every = synth.batched_vortices(n=256, seed=4)
    members = every[:members_n]
    t0 = time.perf_counter()
    preps = [Prep(x["mesh"]) for x in members]
    prep_s = time.perf_counter() - t0
    out = batched_pass(members, preps, steps, warmup, fpk)
    keys = ("value", "ms_per_step", "speedup_vs_looped", "looped_singles_value", "launch", "roofline")
    return {"workload": f"first {members_n} of the 256 batched isentropic vortices "
                        "(log-uniform 2e3-6.4e4 vertices, aspect 1-4), each its own CFL step",
            "physical_vertices": int(sum(x["U"].shape[1] for x in members)), "steps": steps,
            "prep_seconds": prep_s,
            "fp64": {k: out["fp64"][k] for k in keys},
            "fp32_bulk": {k: out["fp32"][k] for k in keys}}


def variant_adjoint(reps=10, horizon=20, every=4):
    """Cost of the discrete adjoint on the adjoint configuration's mesh (256 x 256 periodic
    vortex, FP64, device CFL step of the initial state): one hfd_adjoint against one hfd_step,
    and a checkpointed rollout's backward pass against its forward pass."""
    import torch
    from paper_2109_01286_gb300 import Mesh
    from paper_2109_01286_gb300.autograd import rollout
    m = synth.jittered_grid(256, 256, 10.0, 10.0, seed=5)
    mesh = Mesh(m)
    U0 = mesh.import_state(torch.from_numpy(synth.isentropic_vortex(m, beta=5.0)).cuda())
    probe = U0.clone()
    mesh.step(probe, 0.0)
    dt = float(mesh.last_dt())
    stream = torch.cuda.current_stream()
    lam = torch.ones_like(U0)
    X = U0.clone()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    step_ms = timed(lambda: mesh.step(X.copy_(U0), dt))
    adj_ms = timed(lambda: mesh.adjoint(U0, lam, dt=dt))
    Ui = U0.clone().requires_grad_(True)
    rolls = []
    for ev in (every, 1):          # checkpoints every `every` steps, and every step (no recompute)
        t_fwd = timed(lambda: rollout(Ui, mesh, dt, horizon, ev))

        def fwd_bwd():
            Ui.grad = None
            rollout(Ui, mesh, dt, horizon, ev)[0].sum().backward()
        t_both = timed(fwd_bwd)
        rolls.append({"steps": horizon, "checkpoint_every": ev, "forward_ms": t_fwd,
                      "backward_ms": t_both - t_fwd,
                      "backward_over_forward": (t_both - t_fwd) / t_fwd})
    mesh.check()
    return {"workload": "256x256 periodic isentropic vortex, FP64, fixed step (device CFL 0.3 of "
                        "the initial state)",
            "step_ms": step_ms, "adjoint_ms": adj_ms, "adjoint_over_step": adj_ms / step_ms,
            "rollouts": rolls}


def variant_3d(fpk, peak_hbm, n=40, steps=10, warmup=3):
    """The three-dimensional extension (include/hfd3d.h) on an n^3 periodic Kuhn-split
    tetrahedral box with the vortex tube along z, FP64: vertex-stage updates per second over
    `steps` timed steps, each from the initial state (the reset copy is inside the timed
    region, as in the line's own workload), the per-kernel split, and the divergence kernel's
    arithmetic against the measured FP64 peak.  Algorithmic work of one k3_div launch: 60 FMA
    per vertex entry (4 rows x 3 fluxes x 5 components), 20 per edge entry, the stage update;
    its bytes: 4 + 96 per vertex entry, 4 + 32 per edge entry, state in and out."""
    import torch
    from paper_2109_01286_gb300 import hfd3d
    from synth import three_d as T3
    m = T3.periodic_tet_box(n, n, n, 10.0, 10.0, 10.0, seed=3)
    t0 = time.perf_counter()
    mesh = hfd3d.Mesh3(m)
    prep_s = time.perf_counter() - t0
    info = mesh.info()
    U0 = torch.from_numpy(T3.vortex_tube(m)).cuda()
    V = info["nv"]
    # fixed step: CFL 0.3 of the initial state, the shortest edge over the largest |u| + c
    w = U0[0:5].cpu().numpy()
    p = 0.4 * (w[4] - 0.5 * (w[1] ** 2 + w[2] ** 2 + w[3] ** 2) / w[0])
    speed = np.sqrt((w[1] ** 2 + w[2] ** 2 + w[3] ** 2) / w[0] ** 2) + np.sqrt(1.4 * p / w[0])
    dt = 0.3 * 0.7 * (10.0 / n) / float(speed.max())
    X = U0.clone()
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        mesh.steps(X.copy_(U0), dt, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        mesh.steps(X.copy_(U0), dt, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    mesh.check()
    finite = bool(torch.isfinite(X).all())
    km = {"vertex": 0.0, "edge": 0.0, "div": 0.0}
    for _ in range(steps):
        t = mesh.steps_profiled(X.copy_(U0), dt, 1)
        for k in km:
            km[k] += t[k] / (3 * steps)
    # the divergence gather at one lane per vertex, for comparison with the default four
    mesh.set_lanes(1)
    k1 = 0.0
    for _ in range(steps):
        k1 += mesh.steps_profiled(X.copy_(U0), dt, 1)["div"] / (3 * steps)
    mesh.set_lanes(4)
    nv_t, ne_t = info["div_nv_total"], info["div_ne_total"]
    flops = 2.0 * (60 * nv_t + 20 * ne_t) + 3.0 * 20 * V
    nbytes = (4 + 96) * nv_t + (4 + 32) * ne_t + 8 * 4 + 3 * 20 * 8 * V
    div_s = km["div"] / 1000.0
    return {"workload": f"3D extension: {n}^3 periodic Kuhn-split tetrahedral box (jitter 0.15), "
                        "vortex tube along z (beta 5, mean flow (1, 1, 0.5)), FP64, fixed step",
            "vertices": V, "edges": info["nedges"], "div_entries_per_vertex":
                [nv_t / V, ne_t / V], "prep_seconds": prep_s,
            "value": V * 3 / (ms / 1000.0), "unit": "vertex-stage/s", "ms_per_step": ms,
            "state_finite": finite, "kernel_avg_ms": km, "div_ms_one_lane": k1,
            "roofline": {"kernel": "k3_div", "bound": "alu", "achieved": flops / div_s / 1e12,
                         "peak": fpk["fp64_tflops"], "unit": "TFLOP/s",
                         "frac": flops / div_s / 1e12 / fpk["fp64_tflops"],
                         "hbm_gbs": nbytes / div_s / 1e9, "hbm_frac": nbytes / div_s / 1e9 / peak_hbm,
                         "peak_source": fpk["source"]}}


def variant_tgv(steps=(1, 5, 20)):
    """Mixed-precision accuracy on the viscous Taylor-Green configuration (512 x 512, Re 100,
    Mach 0.1, Pr 0.72): FP32 bulk against FP64 after a few steps, and each path's velocity
    against the incompressible decay exp(-2 nu t)."""
    import torch
    from paper_2109_01286_gb300 import Prep
    n, mach, re = 512, 0.1, 100.0
    p0 = 1.0 / (1.4 * mach * mach)
    m = synth.jittered_grid(n, n, 2 * np.pi, 2 * np.pi, seed=3)
    U0 = synth.taylor_green(m, mach=mach)
    prep = Prep(m, viscous=True, mu=1.0 / re, R_gas=p0, prandtl=0.72)
    dt = 0.3 * (2 * np.pi / n) / (1.0 + np.sqrt(1.4 * p0))
    got = {}
    for prec in ("fp64", "fp32"):
        mesh = prep.upload(prec)
        X = mesh.import_state(torch.from_numpy(U0).cuda())
        done, got[prec] = 0, {}
        for k in steps:
            mesh.steps(X, dt, k - done)
            done = k
            got[prec][k] = mesh.export_state(X).cpu().numpy()
        del mesh
    decay = lambda t: np.exp(-2.0 * t / re)

    def vel_err(U, t):
        uex = np.sin(m["x"]) * np.cos(m["y"]) * decay(t)
        vex = -np.cos(m["x"]) * np.sin(m["y"]) * decay(t)
        u, v = U[1] / U[0], U[2] / U[0]
        return float(np.sqrt(np.mean((u - uex) ** 2 + (v - vex) ** 2) / np.mean(uex ** 2 + vex ** 2)))
    rows = []
    for k in steps:
        a, b = got["fp64"][k], got["fp32"][k]
        rows.append({"step": k,
                     "fp32_vs_fp64_rel_l2_all_rows": float(np.linalg.norm(a - b) / np.linalg.norm(a)),
                     "fp32_vs_fp64_rel_l2_w": float(np.linalg.norm(a[:4] - b[:4]) / np.linalg.norm(a[:4])),
                     "velocity_vs_decay_fp64": vel_err(a, k * dt),
                     "velocity_vs_decay_fp32": vel_err(b, k * dt)})
    return {"workload": f"viscous Taylor-Green {n}x{n}, Re {re:g}, Mach {mach}, Pr 0.72, steps of "
                        f"{dt:.4g}", "checkpoints": rows}


# ------------------------------------------------------------------ batched workload
def batched_pass(members, preps, steps, warmup, fpk, dist=None):
    """The batch of `members` (with their preps) advanced as one device mesh (autotuned launch
    shape, CUDA graph of RK steps, every member its own CFL step) for `steps` timed steps, and
    the same meshes looped one at a time; FP64 and FP32 bulk.  Returns per precision the rates,
    the speed-up over the loop, the launch choice, the per-kernel times and the roofline of the
    dominant kernel."""
    import torch
    from paper_2109_01286_gb300 import Prep, replicas
    args = argparse.Namespace(steps=steps, warmup=warmup)
    Ub = np.concatenate([x["U"] for x in members], axis=1)
    stream = torch.cuda.current_stream()
    out = {}
    for prec in ("fp64", "fp32"):
        batch = Prep.concat(preps).upload(prec)
        A = batch.stats.nactive
        U0 = batch.import_state(torch.from_numpy(Ub).cuda())
        choice = batch.autotune(U0)
        W = U0.clone()
        batch.steps(W, 0.0, args.warmup)
        X = U0.clone()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.steps(X, 0.0, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        value, units, ms = replicas.whole_job_rate(A * 3 * args.steps, e0.elapsed_time(e1), dist,
                                                   device="cuda")
        kms, nl = batch.steps_profiled(U0.clone(), 0.0, args.steps)
        # roofline of the dominant kernel (per-launch averages of the profiled steps)
        T = 8 if prec == "fp64" else 4
        costs = algorithmic_costs(batch.stats_dict(), T)
        dom = max(("vertex", "edge", "div"), key=lambda k: kms[k])
        avg_s = kms[dom] / 1000.0 / (3 * args.steps)
        peak_hbm, peak_src = load_peaks()
        if prec == "fp64":
            roof = {"kernel": f"k_{dom}<double>", "bound": "alu",
                    "achieved": costs[dom]["flops"] / avg_s / 1e12, "peak": fpk["fp64_tflops"],
                    "unit": "TFLOP/s", "traffic": None, "peak_source": fpk["source"],
                    "hbm_gbs": costs[dom]["bytes"] / avg_s / 1e9}
            roof["frac"] = roof["achieved"] / roof["peak"]
        else:
            roof = {"kernel": f"k_{dom}<float>", "bound": "hbm",
                    "achieved": costs[dom]["bytes"] / avg_s / 1e9, "peak": peak_hbm,
                    "unit": "GB/s", "traffic": None, "peak_source": peak_src}
            roof["frac"] = roof["achieved"] / peak_hbm
        del batch, W, X
        torch.cuda.empty_cache()
        # the same meshes one at a time
        singles = [p.upload(prec) for p in preps]
        states = [s.import_state(torch.from_numpy(x["U"]).cuda()) for s, x in zip(singles, members)]
        for s, u in zip(singles, states):
            s.steps(u.clone(), 0.0, args.warmup)
        torch.cuda.synchronize()
        e0.record(stream)
        for s, u in zip(singles, states):
            s.steps(u, 0.0, args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        loop_value, _, ms_loop = replicas.whole_job_rate(A * 3 * args.steps, e0.elapsed_time(e1),
                                                         dist, device="cuda")
        del singles, states
        torch.cuda.empty_cache()
        out[prec] = {"value": value, "ms_per_step": ms / args.steps,
                     "looped_singles_value": loop_value,
                     "looped_singles_ms_per_step": ms_loop / args.steps,
                     "speedup_vs_looped": ms_loop / ms,
                     "launch": {"persistent": choice[0], "grid": choice[1], "lanes": choice[2], "staged_div": choice[3]},
                     "kernels_ms": kms, "launches": nl, "roofline": roof}
    return out


def run_batched(args):
    """Many uneven meshes advanced together (one union mesh, autotuned launch shape, graph of RK
    stages) against looping the same meshes one at a time (one graph per mesh).  Under torchrun
    the meshes are partitioned over the ranks (no data-path collective); the whole-job rate is
    all ranks' vertex-stage updates over the slowest rank's time."""
    import torch
    from paper_2109_01286_gb300 import Prep, replicas
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    every = synth.batched_vortices(n=args.batch, seed=4)
    members = [every[i] for i in replicas.shard(len(every), rank, world)]
    t0 = time.perf_counter()
    preps = [Prep(x["mesh"]) for x in members]
    prep_s = time.perf_counter() - t0
    fpk = fma_peaks()
    out = batched_pass(members, preps, args.steps, args.warmup, fpk, dist)
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return
    r = out["fp64"]
    line = {
        "metric": METRIC, "value": r["value"], "unit": "vertex-stage/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "workload": "batched",
        "config": {"workload": f"{args.batch} isentropic vortices, vertex counts log-uniform in "
                               "[2e3, 6.4e4], aspect 1-4, jittered random-split periodic meshes",
                   "physical_vertices": int(sum(x["U"].shape[1] for x in every)),
                   "parallelism": f"meshes partitioned over {world} rank(s)",
                   "prep_seconds": prep_s, "time_step": "device CFL 0.3 per member"},
        "fp64": out["fp64"], "fp32_bulk": out["fp32"], "gpu_launches": int(r["launches"]),
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ adjoint workload
def run_adjoint(args):
    """Discrete adjoint of an isentropic-vortex run on a 256 x 256 jittered mesh (FP64,
    checkpointed): objective J = sum_v A_v (rho - rho_exact)^2 at the final time; gradients with
    respect to the initial state (and its derivatives), checked against central differences
    (step 1e-6) on random directions, and to the vortex strength beta, checked against
    fourth-order differences.  200 steps are requested; the longest horizon of 200, 100, 50, 20,
    10 steps on which the run stays finite and 4 directions agree to 1e-5 is used.  Reports the
    cost of the backward pass relative to the forward pass."""
    import torch
    from paper_2109_01286_gb300 import Mesh
    from paper_2109_01286_gb300.autograd import rollout
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n, nsteps, every, beta = 256, 200, 20, 5.0
    m = synth.jittered_grid(n, n, 10.0, 10.0, seed=5)
    mesh = Mesh(m)
    U0 = synth.isentropic_vortex(m, beta=beta)
    # fixed step: the device CFL step (CFL 0.3) of the initial state
    probe = mesh.import_state(torch.from_numpy(U0).cuda())
    mesh.step(probe, 0.0)
    dt = float(mesh.last_dt())
    del probe
    T = nsteps * dt
    perm = torch.from_numpy(mesh.perm.astype(np.int64)).cuda()
    area = torch.from_numpy(synth.vertex_areas(m)).cuda()[perm]
    rho_ex = torch.from_numpy(synth.isentropic_vortex(m, beta=beta, t=T)[0]).cuda()[perm]

    # The method as read amplifies perturbations exponentially (its linearised residual has
    # eigenvalues with positive real part on these meshes), and central differences lose their
    # meaning once the amplification swamps the step.  Horizons from the
    # requested one downwards are checked on 4 directions, then on all directions; the longest
    # horizon whose differences agree with the adjoint to 1e-5 on every direction is used.
    requested = nsteps
    horizons = [h for h in (200, 100, 50, 40, 30, 20, 10) if h <= requested]
    scan = []
    def make_J(ns, ev, rho_t):
        def J(Ui):
            UN = rollout(Ui, mesh, dt, ns, ev)
            return torch.sum(area * (UN[0] - rho_t) ** 2)
        return J

    def fd_check(J, g, k, seed):
        rng = np.random.default_rng(seed)
        rel = []
        with torch.no_grad():
            for _ in range(k):
                d = mesh.import_state(torch.from_numpy(rng.standard_normal(U0.shape)).cuda())
                d = d / torch.linalg.norm(d)
                eps = 1e-6
                fd = (J(U0i.detach() + eps * d).item() - J(U0i.detach() - eps * d).item()) / (2 * eps)
                ad = torch.sum(g * d).item()
                rel.append(abs(fd - ad) / max(abs(fd), abs(ad), 1e-300))
        return rel

    U0i = mesh.import_state(torch.from_numpy(U0).cuda()).requires_grad_(True)
    chosen, rel_chosen = None, None
    for hz in horizons:
        ev = min(every, max(1, hz // 5))
        rho_t = torch.from_numpy(synth.isentropic_vortex(m, beta=beta, t=hz * dt)[0]).cuda()[perm]
        Jh = make_J(hz, ev, rho_t)
        U0i.grad = None
        val = Jh(U0i)
        if not bool(torch.isfinite(val)):
            scan.append({"steps": hz, "finite": False})
            continue
        val.backward()
        rel = fd_check(Jh, U0i.grad.detach(), 4, 11)
        entry = {"steps": hz, "finite": True, "fd_rel_err_max_4dirs": max(rel)}
        scan.append(entry)
        if max(rel) <= 1e-5:
            rel_all = fd_check(Jh, U0i.grad.detach(), args.directions, 5)
            entry["fd_rel_err_max_all_dirs"] = max(rel_all)
            if max(rel_all) <= 1e-5:
                chosen, rel_chosen = hz, rel_all
                break
    nsteps = chosen if chosen else horizons[-1]
    every = min(every, max(1, nsteps // 5))
    T = nsteps * dt
    rho_ex = torch.from_numpy(synth.isentropic_vortex(m, beta=beta, t=T)[0]).cuda()[perm]
    J = make_J(nsteps, every, rho_ex)
    U0i.grad = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    val = J(U0i)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    val.backward()
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    g = U0i.grad.detach()
    # per-step cost: forward step against one adjoint step (same state)
    X = U0i.detach().clone()
    lam = torch.randn_like(X)
    out = torch.empty_like(X)
    for _ in range(3):
        mesh.step(X.clone(), dt)
        mesh.adjoint(X, lam, out, dt)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        mesh.step(X, dt)
    e1.record()
    torch.cuda.synchronize()
    ms_step = e0.elapsed_time(e1) / 20
    e0.record()
    for _ in range(20):
        mesh.adjoint(X, lam, out, dt)
    e1.record()
    torch.cuda.synchronize()
    ms_adj = e0.elapsed_time(e1) / 20
    # central differences on random directions of the initial state (already taken for the
    # chosen horizon)
    rel = rel_chosen if rel_chosen is not None else fd_check(J, g, args.directions, 5)
    # vortex strength: dJ/dbeta = <g, dU0/dbeta> - 2 sum A (rho - rho_ex) drho_ex/dbeta, with the
    # beta derivatives of the (synthetic) exact states by 4th-order central differences
    db = 1e-3
    def ic(bb, t=0.0):
        return synth.isentropic_vortex(m, beta=bb, t=t)
    dU0 = (-ic(beta + 2 * db) + 8 * ic(beta + db) - 8 * ic(beta - db) + ic(beta - 2 * db)) / (12 * db)
    drho = (-ic(beta + 2 * db, T)[0] + 8 * ic(beta + db, T)[0] - 8 * ic(beta - db, T)[0]
            + ic(beta - 2 * db, T)[0]) / (12 * db)
    with torch.no_grad():
        UN = rollout(U0i.detach(), mesh, dt, nsteps, every)
        resid = UN[0] - rho_ex
    dJdb = torch.sum(g * mesh.import_state(torch.from_numpy(dU0).cuda())).item() \
        - 2.0 * torch.sum(area * resid * torch.from_numpy(drho).cuda()[perm]).item()
    with torch.no_grad():
        def Jb(bb):
            Ub = mesh.import_state(torch.from_numpy(ic(bb)).cuda())
            re = torch.from_numpy(ic(bb, T)[0]).cuda()[perm]
            return torch.sum(area * (rollout(Ub, mesh, dt, nsteps, every)[0] - re) ** 2).item()
        # fourth-order central differences with the step of dU0/dbeta: a step of 1e-6 would
        # leave a change in J of ~1e-16 against the rounding noise of a 50-step rollout
        fd_b = (-Jb(beta + 2 * db) + 8 * Jb(beta + db) - 8 * Jb(beta - db) + Jb(beta - 2 * db)) / (12 * db)
    line = {
        "metric": "adjoint check and cost", "workload": "adjoint",
        "config": {"workload": f"isentropic vortex beta={beta}, {n}x{n} jittered random-split "
                               f"periodic mesh, FP64, {nsteps} SSP-RK3 steps, dt={dt:.5g}, "
                               f"checkpoint every {every}",
                   "objective": "sum_v A_v (rho - rho_exact)^2 at t_final"},
        "J": val.item(), "t_final": T, "steps_requested": requested, "steps_used": nsteps,
        "checkpoint_every": every, "horizon_scan": scan,
        "forward_s": t_fwd, "backward_s": t_bwd, "backward_over_forward": t_bwd / t_fwd,
        "ms_step": ms_step, "ms_adjoint_step": ms_adj, "adjoint_over_step": ms_adj / ms_step,
        "fd_directions": args.directions, "fd_rel_err_max": max(rel),
        "fd_rel_err_median": float(np.median(rel)),
        "dJ_dbeta_adjoint": dJdb, "dJ_dbeta_fd": fd_b,
        "dJ_dbeta_rel_err": abs(dJdb - fd_b) / abs(fd_b),
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ viscous accuracy workload
def run_tgv(args):
    """Decaying Taylor-Green vortex (Re 100, Mach 0.1, Pr 0.72) on a 512 x 512 jittered
    periodic mesh to t = 1, FP64 and FP32 bulk: relative L2 difference of the two paths and the
    velocity error of each against the incompressible decay exp(-2 nu t)."""
    import torch
    from paper_2109_01286_gb300 import Prep
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n, mach, re, tend = args.n if args.n != 1024 else 512, 0.1, 100.0, 1.0
    p0 = 1.0 / (1.4 * mach * mach)
    m = synth.jittered_grid(n, n, 2 * np.pi, 2 * np.pi, seed=3)
    U0 = synth.taylor_green(m, mach=mach)
    prep = Prep(m, viscous=True, mu=1.0 / re, R_gas=p0, prandtl=0.72)
    h = 2 * np.pi / n
    dt = 0.3 * h / (1.0 + np.sqrt(1.4 * p0))
    nsteps = int(np.ceil(tend / dt))
    dt = tend / nsteps
    # checkpoints in steps (the state of this method as read turns non-finite within a few tens
    # of steps at this resolution; each checkpoint is reported while both paths are finite)
    marks = [k for k in (1, 2, 5, 10, 20, 50, 100, 200, 500, 1000, 2000) if k < nsteps] + [nsteps]
    states = {"fp64": {}, "fp32": {}}
    walls = {}
    for prec in ("fp64", "fp32"):
        mesh = prep.upload(prec)
        X = mesh.import_state(torch.from_numpy(U0).cuda())
        done = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for mk in marks:
            mesh.steps(X, dt, mk - done)
            done = mk
            S = mesh.export_state(X).cpu().numpy()
            if not np.all(np.isfinite(S)):
                break
            states[prec][mk] = S
        walls[prec] = time.perf_counter() - t0
    decay = lambda t: np.exp(-2.0 * (1.0 / re) * t)

    def vel_err(U, t):
        uex = np.sin(m["x"]) * np.cos(m["y"]) * decay(t)
        vex = -np.cos(m["x"]) * np.sin(m["y"]) * decay(t)
        u, v = U[1] / U[0], U[2] / U[0]
        return float(np.sqrt(np.mean((u - uex) ** 2 + (v - vex) ** 2) / np.mean(uex ** 2 + vex ** 2)))
    table = []
    for mk in marks:
        if mk not in states["fp64"] or mk not in states["fp32"]:
            break
        a, b = states["fp64"][mk], states["fp32"][mk]
        t = mk * dt
        table.append({"step": mk, "t": t, "fp32_vs_fp64_rel_l2": float(np.linalg.norm(a - b) / np.linalg.norm(a)),
                      "fp32_vs_fp64_rel_l2_w": float(np.linalg.norm(a[:4] - b[:4]) / np.linalg.norm(a[:4])),
                      "velocity_rel_l2_vs_exp_decay_fp64": vel_err(a, t),
                      "velocity_rel_l2_vs_exp_decay_fp32": vel_err(b, t)})
    finite_until = {p: (max(states[p]) * dt if states[p] else 0.0) for p in states}
    line = {
        "metric": "mixed-precision accuracy", "workload": "tgv",
        "config": {"workload": f"Taylor-Green vortex Re {re:g}, Mach {mach}, Pr 0.72, {n}x{n} "
                               f"jittered periodic mesh, to t = {tend}, steps of {dt:.4g}"},
        "checkpoints": table, "finite_until_t": finite_until, "wall_s": walls,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ vortex accuracy workload
def run_vortex_order(args):
    """Accuracy test of Sec. 3.1 at the paper's resolutions: the isentropic vortex (beta 5,
    gamma 1.4) advected by the mean flow (1, 1) on the periodic [-10, 10]^2, on meshes of 50,
    75, 100 and 150 segments per side (jittered random-split grids standing in for the paper's
    Delaunay meshes), FP64 SSP-RK3.  Each mesh takes a fixed step: its CFL-0.3 step rounded
    down so that the checkpoints t = 0.25, 0.5, 1, 2 fall on steps.  Reports the area-weighted
    L2 and the max density error against the exact translated vortex at each checkpoint and the
    observed order between consecutive meshes."""
    import torch
    from paper_2109_01286_gb300 import Mesh
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    Ns, marks, quantum = (50, 75, 100, 150), (0.25, 0.5, 1.0, 2.0), 0.25
    vortex = dict(beta=5.0, center=(0.0, 0.0), mean=(1.0, 1.0))
    rows = []
    for N in Ns:
        m = synth.jittered_grid(N, N, 20.0, 20.0, seed=1, x0=-10.0, y0=-10.0)
        mesh = Mesh(m)
        X = mesh.import_state(torch.from_numpy(synth.isentropic_vortex(m, **vortex)).cuda())
        probe = X.clone()
        mesh.step(probe, 0.0)
        dt = quantum / np.ceil(quantum / mesh.last_dt())
        del probe
        A = synth.vertex_areas(m)
        done, t0 = 0, time.perf_counter()
        errs = {}
        for T in marks:
            k = int(round(T / dt))
            mesh.steps(X, dt, k - done)
            done = k
            rho = mesh.export_state(X)[0].cpu().numpy()
            ex = synth.isentropic_vortex(m, t=T, **vortex)[0]
            d = rho - ex
            errs[T] = {"l2": float(np.sqrt(np.sum(A * d * d) / np.sum(A))),
                       "max": float(np.abs(d).max()), "finite": bool(np.all(np.isfinite(rho)))}
        rows.append({"segments": N, "vertices": len(m["x"]), "h": 20.0 / N, "dt": dt,
                     "steps": done, "errors": {str(T): e for T, e in errs.items()},
                     "wall_s": time.perf_counter() - t0})
    orders = {}
    for T in marks:
        o = []
        for a, b in zip(rows[:-1], rows[1:]):
            ea, eb = a["errors"][str(T)]["l2"], b["errors"][str(T)]["l2"]
            o.append(float(np.log(ea / eb) / np.log(b["segments"] / a["segments"]))
                     if ea > 0 and eb > 0 and np.isfinite(ea) and np.isfinite(eb) else None)
        orders[str(T)] = o
    line = {"metric": "density error order", "workload": "vortex-order", "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "isentropic vortex beta 5, mean flow (1,1), periodic "
                                   "[-10,10]^2, jittered random-split meshes of 50/75/100/150 "
                                   "segments per side, FP64, CFL <= 0.3"},
            "runs": rows, "l2_orders_between_consecutive_meshes": orders}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ circular Sod workload
def run_couette(args):
    """Compressible Couette flow of Sec. 3.2 marched in time: walls at y = -5 and +5 moving at
    -u0 and +u0 held by 6 fixed ghost layers each (the exact solution), x periodic on [-5, 5),
    gamma 1.4, c_p 10, conductivity 1/100, viscosity 1/10 (the paper's constants; the wall
    speed and temperatures it leaves out are u0 = 1, T = 10 and 12, p = 10).  Jittered
    random-split meshes with the paper's 35, 70, 105 and 140 segments per side, FP64, started
    from the exact steady solution with a fixed step proportional to h (CFL 0.3 of the finest
    mesh scaled by h): the area-weighted L2 density error against the exact solution at
    checkpoints, and the order between consecutive meshes, while the states stay finite."""
    import torch
    from paper_2109_01286_gb300 import Mesh
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    Ns, marks = (35, 70, 105, 140), (0.05, 0.1, 0.2, 0.5, 1.0, 2.0)
    visc = dict(viscous=True, mu=0.1, prandtl=100.0, R_gas=0.4 * 10.0 / 1.4)
    quantum = 0.05
    errs, meshes = {}, []
    for N in Ns:
        m = synth.couette_channel(N, N + 1, 6, seed=7)
        U0 = synth.couette(m)
        mesh = Mesh(m, **visc)
        phys = np.ones(len(m["x"]), bool)
        phys[m["ghost_ids"]] = False
        A = synth.vertex_areas(m)[phys]
        X = mesh.import_state(torch.from_numpy(U0).cuda())
        probe = X.clone()
        mesh.step(probe, 0.0)
        dt_cfl = float(mesh.last_dt())
        k = int(np.ceil(quantum / dt_cfl))          # steps per quantum: checkpoints on steps
        dt = quantum / k
        done, errs[N] = 0.0, {}
        for t in marks:
            nsteps = int(round((t - done) / dt))
            mesh.steps(X, dt, nsteps)
            done = t
            U = mesh.export_state(X).cpu().numpy()
            if not np.all(np.isfinite(U[:, phys])):
                break
            errs[N][t] = float(np.sqrt(np.sum(A * (U[0, phys] - U0[0, phys]) ** 2) / A.sum()))
        meshes.append({"segments": N, "vertices": len(m["x"]), "physical": int(phys.sum()),
                       "dt": dt, "finite_until": max(errs[N]) if errs[N] else 0.0})
        del mesh
    table = []
    for t in marks:
        row = {"t": t, "rho_l2": [errs[N].get(t) for N in Ns]}
        e = row["rho_l2"]
        row["orders"] = [float(np.log(e[i] / e[i + 1]) / np.log(Ns[i + 1] / Ns[i]))
                         if e[i] and e[i + 1] else None for i in range(len(Ns) - 1)]
        table.append(row)
    line = {"metric": "density error vs exact", "workload": "couette", "data": "synthetic",
            "config": {"workload": "compressible Couette flow (Sec. 3.2), walls at y = +-5 "
                                   "with 6 fixed ghost layers, x periodic, 35/70/105/140 "
                                   "segments per side, FP64, from the exact solution"},
            "meshes": meshes, "checkpoints": table}
    print(json.dumps(line), flush=True)


def run_circular_sod(args):
    """Circular Sod problem (Sec. 3.3) on embedded-circle Delaunay meshes of [-1, 1]^2 whose
    sides are split into 50, 100 and 150 segments: FP64 SSP-RK3 steps at CFL 0.3 (device time
    step) toward t = 0.2, stopping at the first step whose state is not finite or has a
    non-positive density or pressure; then the step rate on the largest mesh, timed over the
    steps that stay admissible, each timed pass restarting from the initial state (the device
    copy is inside the timed region)."""
    import torch
    from paper_2109_01286_gb300 import Mesh
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    g1 = synth.GAMMA - 1.0
    runs, last = [], None
    for n in (50, 100, 150):
        m = synth.embedded_circle_box(n, seed=8)
        U0 = torch.from_numpy(synth.circular_sod(m)).cuda()
        mesh = Mesh(m)
        A = mesh.stats_dict()["nactive"]
        X = mesh.import_state(U0)
        t, steps, first_bad = 0.0, 0, None
        while t < 0.2 and steps < 5000:
            mesh.step(X, 0.0)
            t += mesh.last_dt()
            steps += 1
            w = X[:4]
            p = g1 * (w[3] - 0.5 * (w[1] * w[1] + w[2] * w[2]) / w[0])
            if not (bool(torch.isfinite(w).all()) and bool((w[0] > 0).all()) and bool((p > 0).all())):
                first_bad = steps
                break
        runs.append({"segments": n, "vertices": len(m["x"]), "active": A,
                     "triangles": len(m["tri"]), "steps_admissible": steps - (first_bad is not None),
                     "t_admissible": t if first_bad is None else t - mesh.last_dt(),
                     "first_inadmissible_step": first_bad, "t_target": 0.2})
        last = (mesh, A, U0, steps - (first_bad is not None))
    mesh, A, U0, K = last
    K = max(1, min(K, 5))
    Ui = mesh.import_state(U0)
    X = torch.empty_like(Ui)
    stream = torch.cuda.current_stream()

    def timed():
        for _ in range(args.warmup):
            X.copy_(Ui)
            mesh.steps(X, 0.0, K)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            X.copy_(Ui)
            mesh.steps(X, 0.0, K)
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / (K * args.steps)

    ms_default = timed()
    choice = mesh.autotune(Ui)
    ms = timed()
    line = {
        "metric": "vertex-stage updates/s", "workload": "circular-sod",
        "value": A * 3 / (ms / 1000.0), "unit": "vertex-stage/s",
        "ms_per_step": ms, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "circular Sod (Sec. 3.3), embedded-circle Delaunay meshes of "
                               "[-1,1]^2 with 50/100/150 segments per side, 5 ghost layers, "
                               "CFL 0.3; rate on the 150-segment mesh over "
                               f"{K} steps per pass from the initial state, autotuned launch"},
        "launch": {"persistent": choice[0], "grid": choice[1], "lanes": choice[2], "staged_div": choice[3]},
        "ms_per_step_default_launch": ms_default,
        "runs": runs,
    }
    print(json.dumps(line), flush=True)


def run_three_d(args):
    """The 3D extension alone (variant_3d at the size --n, 40 when --n is left at the 2D
    default), as one JSON line."""
    n = 40 if args.n == 1024 else args.n
    peak_hbm, _ = load_peaks()
    r = variant_3d(fma_peaks(), peak_hbm, n=n, steps=args.steps, warmup=args.warmup)
    line = {"metric": "vertex-stage updates/s", "workload": "three-d", "value": r["value"],
            "unit": "vertex-stage/s", "ms_per_step": r["ms_per_step"], "steps": args.steps,
            "warmup": args.warmup, "dtype": "f64", "data": "synthetic",
            "config": {"workload": r["workload"]}, "roofline": r["roofline"], "detail": r}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "tgv":
        run_tgv(args)
    elif args.workload == "couette":
        run_couette(args)
    elif args.workload == "circular-sod":
        run_circular_sod(args)
    elif args.workload == "vortex-order":
        run_vortex_order(args)
    elif args.workload == "three-d":
        run_three_d(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
