"""Benchmark: PCG solves/s of the multiscreen hypersingular BEM hot path on GB300.

One step = one pass of the whole hot path on the three-page book workload
(h = 1/64, 12,033 dofs, 24,576 triangles, 48 jittered patches, coarse H = 1/4,
g = (1, 0.5, 0.25)): assembly of W (far field, near field, contraction),
set-up of the two-level additive Schwarz preconditioner, and the PCG solve to
relative residual 1e-8.  The geometry's topology is built once at upload
(per-geometry setup); it is inside the end-to-end number, which also copies
the mesh from pinned host memory and reads the density back every step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank solves its own replica (no data-path
collective: the solves are independent), timing is max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG solves/s and p50/p99 latency at rel. residual 1e-8 vs plain FP64 GPU PCG"
UNIT = "solves/s"
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# double-float far-field kernel: FP32-pipe operations per unordered pair
# (36 evaluations x 76 + 6 x 36 per-point updates), counted from far_df.cu
FP32_OPS_PER_FAR_PAIR = 36 * 76 + 6 * 36
# DRAM bytes (read + write) of one far_df_kernel launch, from an ncu capture of
# the h=1/32 book (6,144 triangles: 1.21 MB read + 257.52 MB written), scaled
# to the h=1/64 book by the number of triangle pairs (x16).  Valid for the
# kernel as captured; reset to None when the kernel changes.
FAR_DF_TRAFFIC_BOOK64 = 16 * (1.211904e6 + 257.520640e6)
# double-float multiply-add on the FP32 pipe (df.cuh df_fma_acc)
FP32_OPS_PER_DF_FMA = 13


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return 6800.0, "fallback 6.8 TB/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--far-kernel", type=int, default=0, help="0 double-float (default), 1 native FP64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-modes", action="store_true", help="skip the solve-mode comparison")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving simulation")
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--serve-precision", default="mixed", choices=["mixed", "mixed-tc", "mixed-fp16", "df", "tc"])
    ap.add_argument("--serve-config", default="mix", choices=["mix", "c5"],
                    help="mix: 300-request stream of small geometries (default); c5: the serving configuration "
                         "(2000 requests, squares / cubes / panels up to 40k dofs, 160 GB budget; minutes)")
    ap.add_argument("--no-cube", action="store_true", help="skip the cube-with-mid-planes section")
    ap.add_argument("--no-panels", action="store_true",
                    help="skip the sixteen hinged-panel instances (grouped factorisation, batched solves)")
    ap.add_argument("--workload", default="book64", choices=["book64", "book48", "book32", "flat"],
                    help="book64 is the measured workload; book48, book32 and flat are for profiling")
    ap.add_argument("--matvec", type=int, default=0,
                    help="microbenchmark only: time the product kernel on K vectors (msbem_apply)")
    ap.add_argument("--matvec-precision", default="df", choices=["df", "fp32", "fp64", "tc", "fp16-tc"])
    return ap.parse_args()


BOOK64_TEXT = ("three-page book h=1/64, N=12033 dofs, 24576 triangles, 48 jittered patches (seed 0), "
               "coarse H=1/4 (33 dofs), g=(1,0.5,0.25), rtol 1e-8")


def workload_text(name: str, geom) -> str:
    """The config.workload string both arms print for the same --workload."""
    return BOOK64_TEXT if name == "book64" else f"{geom.name} (profiling case)"


def make_workload(name):
    from paper_2310_09204_gb300 import workloads as WL
    if name == "book64":
        return WL.book_config()
    if name == "book32":
        return WL.book(32, 4, jitter=True, seed=0)
    if name == "book48":
        return WL.book(48, 4, jitter=True, seed=0)
    return WL.flat_config()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x: float, device=None) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def aggregate(pg, world: int, steps: int, local_seconds: float, device=None):
    """Whole-job throughput of N independent replicas: every rank ran `steps`
    solves; the job time is the slowest rank's.  Returns (solves/s, seconds)."""
    t = max_over_ranks(pg, local_seconds, device)
    return world * steps / t, t


# --------------------------------------------------------------------------
# oracle timing (cpu_baseline and the reference arm)
# --------------------------------------------------------------------------

def oracle_step_seconds(geom, state: dict) -> tuple[float, dict]:
    """One oracle solve of the workload on the host cores.  The pair matrix V
    (the dominant phase) is timed on a sample of 1/8 of its rows and scaled;
    topology, contraction, preconditioner set-up and PCG run in full on the
    oracle's own W (assembled once, untimed, the first time)."""
    from oracle import core, solver
    from oracle.topology import Topology
    t0 = time.perf_counter()
    top = Topology(geom.xyz, geom.tri)
    t_topo = time.perf_counter() - t0
    nt = geom.nt
    frac = 8
    rows = np.arange(state.get("row_offset", 0), nt, frac, dtype=np.int64)
    state["row_offset"] = (state.get("row_offset", 0) + 1) % frac
    R = np.repeat(rows, nt)
    C = np.tile(np.arange(nt, dtype=np.int64), rows.size)
    t0 = time.perf_counter()
    core.V_entries(geom.xyz, geom.tri, R, C)
    t_V = (time.perf_counter() - t0) * nt / rows.size / 2.0      # upper half of V suffices
    del R, C
    if "pb" not in state:
        state["pb"] = solver.Problem(geom)
    pb = state["pb"]
    t0 = time.perf_counter()
    solver.assemble_W(top, pb.V)
    t_W = time.perf_counter() - t0
    t0 = time.perf_counter()
    pb.factor()
    t_f = time.perf_counter() - t0
    t0 = time.perf_counter()
    res = pb.solve(rtol=1e-8)
    t_s = time.perf_counter() - t0
    total = t_topo + t_V + t_W + t_f + t_s
    return total, {"topology_s": t_topo, "V_s_scaled": t_V, "contract_s": t_W, "factor_s": t_f,
                   "solve_s": t_s, "iters": res.iters}


def cores_used() -> int:
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


def run_reference(args, world, rank, pg):
    if rank != 0:
        return
    from oracle import core
    core.build()
    geom = make_workload(args.workload)
    state = {}
    for _ in range(args.warmup):
        # untimed warm-up: the topology and one V row (cheap) plus the one-time W
        from oracle import solver
        if "pb" not in state:
            state["pb"] = solver.Problem(geom)
    times, details = [], []
    for _ in range(args.steps):
        t, d = oracle_step_seconds(geom, state)
        times.append(t)
        details.append(d)
    total = sum(times)
    value = args.steps / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_text(args.workload, geom), "global_batch": 1,
                       "seq_len": int(state["pb"].top.ndof), "parallelism": "rank 0 only (host cores)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
                             "sample": "V on 1/8 of its rows (scaled); topology, contraction, "
                                       "preconditioner and PCG in full", "phases": details[-1]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def run_ours(args, world, rank, local, pg):
    import torch
    import paper_2310_09204_gb300 as M
    from paper_2310_09204_gb300 import build as B
    from paper_2310_09204_gb300 import workloads as WL

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    geom = make_workload(args.workload)
    g = geom.g

    S = M.Solver(geom, device=local, stream=stream.cuda_stream)
    N = S.n
    dens = torch.empty(N, dtype=torch.float64, device=dev)

    def step():
        S.assemble(far_kernel=args.far_kernel)
        S.factor()
        return S.solve(g, rtol=1e-8, out=dens)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    launches0 = S.counters()["launches"]
    clocks = Clocks(local)
    barrier(pg)
    torch.cuda.synchronize()
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    far_ms, phase, iters = [], [], []
    for k in range(args.steps):
        out = step()
        ev[k + 1].record(stream)
        t = S.timings()
        far_ms.append(t["far_ms"])
        phase.append(t)
        iters.append(out["iters"])
    torch.cuda.synchronize()
    barrier(pg)
    ck = clocks.stop()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    launches = (S.counters()["launches"] - launches0) / args.steps
    value, total_s = aggregate(pg, world, args.steps, sum(step_ms) / 1e3, dev)
    far_pairs = S.counters()["far_pairs"]
    far_avg_s = statistics.mean(far_ms) / 1e3
    ops = far_pairs * FP32_OPS_PER_FAR_PAIR
    peak = SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6
    achieved = ops / far_avg_s
    kernel = "far_df_kernel (double-float on FP32 pipe)" if args.far_kernel == 0 else "far_fp64_kernel"

    # solve modes on the resident geometry (W and M already built by the last
    # step): the plain FP64 comparator request by request, the double-float
    # path, and the batched / mixed-precision forms on the same 16 requests
    modes = None
    if rank == 0 and not args.no_modes:
        modes = solve_modes(S, geom, stream)
    roof_mv = matvec_rooflines(S, N, stream) if rank == 0 and not args.no_modes else None

    serving = None
    if rank == 0 and not args.no_serve:
        if args.serve_config == "c5":
            serving = serve_bench(2000 if args.serve_requests == 300 else args.serve_requests, local, stream,
                                  precision=args.serve_precision, config="c5", budget=160e9)
        else:
            serving = serve_bench(args.serve_requests, local, stream, precision=args.serve_precision)
    cube = None
    if rank == 0 and not args.no_cube:
        cube = cube_bench(local, stream)
    panels = None
    if rank == 0 and not args.no_panels:
        panels = panels_bench(local, stream)

    # end to end through the C ABI with host buffers: upload (host topology +
    # H2D from pinned memory) + assemble + factor + solve + D2H of the density
    e2e = None
    if not args.no_e2e:
        pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy()
               for k, v in (("xyz", geom.xyz), ("tri", geom.tri.astype(np.int32)),
                            ("cxyz", geom.coarse_xyz), ("ctri", geom.coarse_tri.astype(np.int32)),
                            ("parent", geom.parent.astype(np.int32)), ("patch", geom.patch.astype(np.int32)))}
        host_out = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
        h2d = sum(a.nbytes for a in pin.values())
        E = M.Solver(None, device=local, stream=stream.cuda_stream)

        def e2e_step():
            E.upload(pin["xyz"], pin["tri"], pin["cxyz"], pin["ctri"], pin["parent"], pin["patch"])
            E.assemble(far_kernel=args.far_kernel)
            E.factor()
            r = E.solve(g, rtol=1e-8, out=host_out)
            E.free_geometry()
            return r

        e2e_step()
        barrier(pg)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        barrier(pg)
        e2e_value, _ = aggregate(pg, world, args.steps, time.perf_counter() - t0, dev)
        E.close()
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(N * 8)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import core
        core.build()
        t, d = oracle_step_seconds(geom, {})
        cpu = {"value": 1.0 / t, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
               "sample": "one solve of the same workload; V timed on 1/8 of its rows and scaled, "
                         "topology, contraction, preconditioner set-up and PCG in full",
               "phases": d}

    if rank == 0:
        lat = sorted(step_ms)
        p50 = lat[len(lat) // 2]
        p99 = lat[min(len(lat) - 1, int(round(0.99 * (len(lat) - 1))))]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 (double-float far field)" if args.far_kernel == 0 else "f64",
            "data": "synthetic",
            "config": {"workload": workload_text(args.workload, geom),
                       "global_batch": world, "seq_len": N, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (W 1.16 GB, V 4.8 GB)"},
            "latency_ms": {"p50": p50, "p99": p99},
            "phases_ms": {k: statistics.mean(p[k] for p in phase) for k in phase[0]},
            "pcg_iters": iters[-1],
            "roofline": {"kernel": kernel, "bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": (FAR_DF_TRAFFIC_BOOK64 if (args.far_kernel == 0 and args.workload == "book64")
                                     else None),
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz (FP32-pipe ops/s)",
                         "ops_per_launch": ops, "launch_ms": far_avg_s * 1e3},
            "roofline_matvec": roof_mv,
            "solve_modes": modes,
            "serving": serving,
            "cube": cube,
            "panels16": panels,
            "clocks": ck,
            "gpu_launches": int(launches),
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    S.close()


def _events(stream, f):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    out = f()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b), out


def solve_modes(S, geom, stream, nreq=16, seed=7):
    """Solves/s and per-request latency of the solve forms on the same nreq
    requests (seeded Neumann data, the first one the workload's g) on the
    resident geometry.  The plain FP64 comparator runs request by request;
    the batched forms take all nreq requests in one call.  Every result is
    checked against the comparator's: its true relative residual (double-float
    product) and its relative l2 difference."""
    rng = np.random.default_rng(seed)
    G = rng.uniform(-1.0, 1.0, (nreq, 3))
    G[0] = geom.g
    batch_forms = (("df_batch", "df"), ("mixed_batch", "mixed"), ("tc_batch", "tc"), ("mixed_tc_batch", "mixed-tc"),
                   ("mixed_fp16_batch", "mixed-fp16"))
    for prec in ("fp64", "df", "mixed", "tc", "mixed-tc"):   # warm-up (graphs, FP64 copy and slices of W)
        S.solve(G[0], precision=prec)
    for _, prec in batch_forms:
        S.solve_batch(G, precision=prec)
    out = {"requests": nreq, "rtol": 1e-8, "data": "g_c uniform in [-1,1]^3 (seed 7), g_0 = workload g",
           "forms": {"df": "double-float products (CUDA cores)", "mixed": "FP32 inner PCG, double-float residual",
                     "tc": "double-float products on the tensor cores (integer slices)",
                     "mixed_tc": "FP32 inner PCG, tensor-core double-float residual",
                     "mixed_fp16": "scaled-FP16 tensor-core inner PCG, tensor-core double-float residual"}}
    ref = np.empty((nreq, S.n))
    for name, prec in (("plain_fp64", "fp64"), ("df", "df"), ("mixed", "mixed"), ("tc", "tc"),
                       ("mixed_tc", "mixed-tc")):
        lat, it = [], []
        for c in range(nreq):
            ms, r = _events(stream, lambda: S.solve(G[c], rtol=1e-8, precision=prec))
            lat.append(ms)
            it.append(r["iters"])
            if prec == "fp64":
                ref[c] = r["density"]
            else:
                d = np.linalg.norm(r["density"] - ref[c]) / np.linalg.norm(ref[c])
                out.setdefault(name + "_maxdiff_vs_fp64", 0.0)
                out[name + "_maxdiff_vs_fp64"] = max(out[name + "_maxdiff_vs_fp64"], float(d))
        lat.sort()
        out[name] = {"solves_per_s": 1e3 * nreq / sum(lat), "p50_ms": lat[nreq // 2], "p99_ms": lat[-1],
                     "iters": [int(min(it)), int(max(it))], "mode": "one request per call"}
    for name, prec in batch_forms:
        ms, r = _events(stream, lambda: S.solve_batch(G, rtol=1e-8, precision=prec))
        diff = max(float(np.linalg.norm(r["density"][c] - ref[c]) / np.linalg.norm(ref[c])) for c in range(nreq))
        # true residuals with the double-float product
        Y, _ = S.apply(r["density"])
        L = np.stack([S.rhs(G[c]) for c in range(nreq)])
        rel = float(max(np.linalg.norm(L[c] - Y[c]) / np.linalg.norm(L[c]) for c in range(nreq)))
        out[name] = {"solves_per_s": 1e3 * nreq / ms, "batch_ms": ms, "iters": [int(r["iters"].min()),
                     int(r["iters"].max())], "max_true_relres": rel, "maxdiff_vs_fp64": diff,
                     "mode": f"{nreq} requests in one call"}
    base = out["plain_fp64"]["solves_per_s"]
    out["speedup_vs_plain_fp64"] = {k: out[k]["solves_per_s"] / base
                                    for k in ("df", "mixed", "tc", "mixed_tc") + tuple(n for n, _ in batch_forms)}
    return out


# bytes of W read per entry by each product: double-float planes, FP32 hi
# plane, the six bf16 slices of the tensor-core double-float product, the
# fp16 copy of the scaled-FP16 product
MATVEC_BYTES = {"df": 8, "fp32": 4, "tc": 12, "fp16-tc": 2}


def matvec_rooflines(S, N, stream, reps=5):
    """Device time of the matrix-vector products (msbem_apply reports the
    product kernels' own CUDA-event time) against their bound: HBM for the
    products that read W once per call (double-float and FP32 for one vector,
    the tensor-core products for any count: 12 or 2 bytes an entry), the FP32
    pipe for 16 double-float vectors (13 FP32 operations per entry and
    vector)."""
    hbm, src = measured_peaks()
    fp32_peak = SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6
    rng = np.random.default_rng(3)
    out = {}
    for name, prec, k in (("df_k1", "df", 1), ("fp32_k1", "fp32", 1), ("df_k16", "df", 16), ("fp32_k16", "fp32", 16),
                          ("tc_k1", "tc", 1), ("tc_k16", "tc", 16), ("fp16tc_k1", "fp16-tc", 1),
                          ("fp16tc_k16", "fp16-tc", 16)):
        X = rng.standard_normal((k, N))
        S.apply(X, precision=prec)
        ms = sorted(S.apply(X, precision=prec)[1] for _ in range(reps))[reps // 2]
        if name == "df_k16":
            ops = FP32_OPS_PER_DF_FMA * 16 * float(N) * N
            ach = ops / (ms * 1e-3)
            out[name] = {"bound": "alu", "achieved": ach / 1e12, "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
                         "frac": ach / fp32_peak, "launch_ms": ms, "algorithmic": "13 x 16 x N^2 FP32 ops"}
        else:
            b = MATVEC_BYTES[prec] * float(N) * N
            ach = b / (ms * 1e-3) / 1e9
            out[name] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                         "launch_ms": ms, "algorithmic": f"{MATVEC_BYTES[prec]} B x N^2 (W read once)",
                         "peak_source": src}
    return out


def cube_bench(device, stream, reps: int = 3):
    """The cube with its three mid-planes at h = 1/96 (N = 83,817; W 56 GB as
    two FP32 planes; V, 220 GB, assembled in row panels; eight closed cells):
    set-up phases, solves per form (median of `reps`), and the product
    kernel's rooflines at this size (W far larger than L2)."""
    import torch
    import paper_2310_09204_gb300 as M
    from paper_2310_09204_gb300 import workloads as WL
    geom = WL.cube_config()
    out = {"workload": "cube + 3 mid-planes, h=1/96, N=83817, N_T=165888, 324 patches, coarse 387, 8 cells, "
                       "g seeded"}
    with M.Solver(None, device=device) as S:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.upload(geom.xyz, geom.tri, geom.coarse_xyz, geom.coarse_tri, geom.parent, geom.patch)
        torch.cuda.synchronize()
        out["upload_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        S.assemble()
        torch.cuda.synchronize()
        out["assemble_s"] = time.perf_counter() - t0
        t = S.timings()
        out["phases_ms"] = {k: t[k] for k in ("far_ms", "near_ms", "contract_ms")}
        t0 = time.perf_counter()
        S.factor()
        torch.cuda.synchronize()
        out["factor_s"] = time.perf_counter() - t0
        out["split"] = S.split_info()
        rng = np.random.default_rng(0)
        G = rng.uniform(-1.0, 1.0, (16, 3))
        G[0] = geom.g
        S.solve(G[0], precision="fp64")              # makes the FP64 copy of W
        S.solve(G[0], precision="mixed-tc")          # makes the slices of W
        forms = {}
        for name, prec in (("plain_fp64", "fp64"), ("df", "df"), ("mixed", "mixed"), ("mixed_tc", "mixed-tc")):
            ms, it = [], 0
            for r in range(reps):
                m, o = _events(stream, lambda: S.solve(G[r], rtol=1e-8, precision=prec))
                ms.append(m)
                it = o["iters"]
            forms[name] = {"solves_per_s": 1e3 / sorted(ms)[reps // 2], "iters": it}
        for name, prec in (("mixed_batch16", "mixed"), ("mixed_tc_batch16", "mixed-tc"), ("tc_batch16", "tc")):
            m, o = _events(stream, lambda: S.solve_batch(G, rtol=1e-8, precision=prec))
            forms[name] = {"solves_per_s": 16e3 / m, "iters": int(o["iters"].max())}
        base = forms["plain_fp64"]["solves_per_s"]
        for v in forms.values():
            v["vs_plain_fp64"] = v["solves_per_s"] / base
        out["solves"] = forms
        hbm, src = measured_peaks()
        N = float(S.n)
        roof = {}
        for name, prec, k in (("df_k1", "df", 1), ("fp32_k1", "fp32", 1), ("df_k16", "df", 16),
                              ("fp32_k16", "fp32", 16), ("tc_k16", "tc", 16)):
            X = rng.standard_normal((k, S.n))
            S.apply(X, precision=prec)
            ms = sorted(S.apply(X, precision=prec)[1] for _ in range(reps))[reps // 2]
            if name == "df_k16":
                a = FP32_OPS_PER_DF_FMA * 16 * N * N / (ms * 1e-3)
                pk = SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6
                roof[name] = {"bound": "alu", "achieved": a / 1e12, "peak": pk / 1e12, "unit": "TFLOP/s",
                              "frac": a / pk, "launch_ms": ms}
            else:
                b = MATVEC_BYTES[prec] * N * N / (ms * 1e-3) / 1e9
                roof[name] = {"bound": "hbm", "achieved": b, "peak": hbm, "unit": "GB/s", "frac": b / hbm,
                              "launch_ms": ms, "peak_source": src}
        out["roofline_matvec"] = roof
    return out


def panels_bench(device, stream, nreq: int = 4):
    """The sixteen hinged-panel multiscreens (2-6 unit squares at seeded
    dihedral angles, h in {1/24, 1/32, 1/48}) resident in one context: the
    preconditioners factored one geometry per call and then all sixteen in one
    grouped inversion (msbem_factor_group), and nreq seeded requests per
    instance solved by the plain FP64 comparator (request by request) and by
    the batched mixed-precision forms (nreq per call).  Errors are per
    instance: the relative l2 difference from the plain FP64 density and the
    true relative residual with the double-float product."""
    import torch
    import paper_2310_09204_gb300 as M
    from paper_2310_09204_gb300 import workloads as WL
    geoms = WL.panels_config()
    first = M.Solver(geoms[0], device=device)
    group = [first] + [M.Solver(g, share=first) for g in geoms[1:]]
    out = {"workload": "16 hinged-panel multiscreens (seeds 0-15), 2-6 unit squares, h in {1/24,1/32,1/48}, "
                       f"{nreq} requests each (g_0 = workload g, then uniform in [-1,1]^3)",
           "dofs": [int(S.n) for S in group]}
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for S in group:
            S.assemble()
        torch.cuda.synchronize()
        out["assemble_s"] = time.perf_counter() - t0
        for S in group:                              # warm-up (pool)
            S.factor()
        t0 = time.perf_counter()
        for S in group:
            S.factor()
        torch.cuda.synchronize()
        out["factor_one_by_one_s"] = time.perf_counter() - t0
        M.msbem_factor_group(group)                  # warm-up
        t0 = time.perf_counter()
        M.msbem_factor_group(group)
        torch.cuda.synchronize()
        out["factor_grouped_s"] = time.perf_counter() - t0
        forms = {"plain_fp64": [], "mixed_tc_batch": [], "mixed_fp16_batch": []}
        per_inst = []
        for i, (S, geom) in enumerate(zip(group, geoms)):
            rng = np.random.default_rng(geom.meta["seed"])
            G = rng.uniform(-1.0, 1.0, (nreq, 3))
            G[0] = geom.g
            for prec in ("fp64", "mixed-tc"):
                S.solve(G[0], precision=prec)        # FP64 copy and slices of W, graphs
            S.solve_batch(G, precision="mixed-fp16")
            ref = np.empty((nreq, S.n))
            for c in range(nreq):
                ms, r = _events(stream, lambda: S.solve(G[c], rtol=1e-8, precision="fp64"))
                forms["plain_fp64"].append(ms)
                ref[c] = r["density"]
            L = np.stack([S.rhs(G[c]) for c in range(nreq)])
            row = {"n": int(S.n)}
            for name, prec in (("mixed_tc_batch", "mixed-tc"), ("mixed_fp16_batch", "mixed-fp16")):
                ms, r = _events(stream, lambda: S.solve_batch(G, rtol=1e-8, precision=prec))
                forms[name].append(ms)
                Y, _ = S.apply(r["density"])
                row[name] = {"maxdiff_vs_fp64": max(float(np.linalg.norm(r["density"][c] - ref[c]) /
                                                          np.linalg.norm(ref[c])) for c in range(nreq)),
                             "max_true_relres": max(float(np.linalg.norm(L[c] - Y[c]) / np.linalg.norm(L[c]))
                                                    for c in range(nreq)),
                             "iters": int(r["iters"].max())}
            per_inst.append(row)
        total = len(geoms) * nreq
        res = {k: {"solves_per_s": 1e3 * total / sum(v), "total_ms": sum(v)} for k, v in forms.items()}
        for v in res.values():
            v["vs_plain_fp64"] = v["solves_per_s"] / res["plain_fp64"]["solves_per_s"]
        out["solves"] = res
        out["per_instance"] = per_inst
        out["worst"] = {k: {"maxdiff_vs_fp64": max(r[k]["maxdiff_vs_fp64"] for r in per_inst),
                            "max_true_relres": max(r[k]["max_true_relres"] for r in per_inst)}
                        for k in ("mixed_tc_batch", "mixed_fp16_batch")}
    finally:
        for S in reversed(group):
            S.close()
    return out


def serving_workload(R: int, seed: int = 0, new_fraction: float = 0.3):
    """Seeded request stream: each request names a geometry and constant
    Neumann data g in [-1,1]^3; with probability new_fraction (always for the
    first) the geometry is a new one -- the next of a seeded sequence drawn
    from the square (h = 1/24 .. 1/96), three-page book (h = 1/32, 1/48) and
    panel families (500 - 13.5k dofs) -- else one used before."""
    from paper_2310_09204_gb300 import workloads as WL
    rng = np.random.default_rng(seed)
    geoms, reqs = {}, []

    def new_geom(k):
        f = k % 4
        if f == 0:
            n = int(rng.choice([24, 32, 40, 48, 56, 64, 80, 96]))
            return WL.unit_square(n, 2, "square")
        if f == 1:
            n = int(rng.choice([32, 48]))
            return WL.book(n, 4, jitter=True, seed=int(rng.integers(1 << 30)))
        return WL.panels(1000 + k)

    for i in range(R):
        if i == 0 or rng.random() < new_fraction:
            key = len(geoms) + 1
            geoms[key] = new_geom(key)
        else:
            key = int(rng.integers(1, len(geoms) + 1))
        reqs.append((key, rng.uniform(-1.0, 1.0, 3)))
    return geoms, reqs


# the request-stream configuration of the serving row: squares (h = 1/24 ..
# 1/200), cubes with mid-planes (h = 1/12 .. 1/66) and hinged-panel screens,
# 500 - 40k dofs; patches of 100 - 400 dofs
C5_SQUARES = ((24, 2), (32, 2), (48, 3), (64, 4), (96, 6), (128, 8), (160, 10), (192, 12), (200, 10))
C5_CUBES = tuple((n, 6) for n in range(12, 67, 6))


def _c5_geometry(spec):
    """One geometry of the C5 stream from its (family, parameters) spec (a
    top-level function: it runs in the generator pool)."""
    from paper_2310_09204_gb300 import workloads as WL
    fam, a, b = spec
    if fam == "square":
        return WL.unit_square(a, b, "square")
    if fam == "cube":
        return WL.cube_midplanes(a, b, seed=b)
    return WL.panels(a)


def serving_workload_c5(R: int = 2000, seed: int = 0, new_fraction: float = 0.3, small: bool = False):
    """The serving configuration's stream: R requests; with probability
    new_fraction (always for the first) a new geometry, drawn evenly from the
    square, cube and panel families, else one used before; g in [-1,1]^3.
    small: the three smallest squares and two smallest cubes only (a warm-up
    stream).  Geometries are generated in a pool of processes (spawned)."""
    import multiprocessing as mp
    rng = np.random.default_rng(seed)
    squares = C5_SQUARES[:3] if small else C5_SQUARES
    cubes = C5_CUBES[:2] if small else C5_CUBES
    specs, reqs = [], []
    for i in range(R):
        if i == 0 or rng.random() < new_fraction:
            f = int(rng.integers(2 if small else 3))
            if f == 0:
                n, nc = squares[int(rng.integers(len(squares)))]
                specs.append(("square", n, nc))
            elif f == 1:
                n, nc = cubes[int(rng.integers(len(cubes)))]
                specs.append(("cube", n, nc))
            else:
                specs.append(("panels", 5000 + len(specs), 0))
            key = len(specs)
        else:
            key = int(rng.integers(1, len(specs) + 1))
        reqs.append((key, rng.uniform(-1.0, 1.0, 3)))
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        built = pool.map(_c5_geometry, specs, chunksize=4)
    return {k + 1: g for k, g in enumerate(built)}, reqs


def serve_bench(R: int, device: int, stream, load: float = 1.5, precision: str = "mixed", config: str = "mix",
                budget: float = 0.0):
    """Serving: the plain FP64 comparator (one request at a time in arrival
    order, geometries cached once assembled) against the serving engine in
    mixed precision (continuous batching), on the same seeded requests.

    The comparator runs its requests back to back: that gives its capacity
    and every request's service time; requests then arrive as a Poisson
    stream at `load` x that capacity, and the comparator's latencies follow
    from the FIFO recurrence done_i = max(arrival_i, done_{i-1}) + service_i
    (exact for a one-at-a-time server).  The engine serves the same arrivals
    in real time; a second, saturated run (every request queued at once)
    measures its capacity.  Every engine density is checked against the
    comparator's."""
    import torch
    import paper_2310_09204_gb300 as M
    geoms, reqs = serving_workload(R) if config == "mix" else serving_workload_c5(R)
    R = len(reqs)

    def plain(far_kernel):
        """The comparator, back to back: (service times, densities).  Its
        geometry cache evicts the least recently used geometries beyond the
        HBM budget (W as float pairs, its FP64 copy, the preconditioner)."""
        cache, ref, service, used = {}, [], [], {}
        lim = budget if budget > 0 else float("inf")
        home = M.Solver(None, device=device)   # one context (and memory pool) for all cached geometries

        def bytes_of(key):
            n = float(cache[key].n)
            return 16.0 * n * n + 8.0 * n * 2000
        for i, (key, g) in enumerate(reqs):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if key not in cache:
                cache[key] = M.Solver(geoms[key], device=device, share=home)
                while sum(bytes_of(k) for k in cache) > lim and len(cache) > 1:
                    old = min((k for k in cache if k != key), key=lambda k: used.get(k, -1))
                    cache.pop(old).close()
                cache[key].assemble(far_kernel=far_kernel).factor()
            used[key] = i
            out = cache[key].solve(g, rtol=1e-8, precision="fp64")
            torch.cuda.synchronize()
            service.append(time.perf_counter() - t0)
            ref.append(out["density"].copy())
        for S in cache.values():
            S.close()
        home.close()
        return service, ref

    def fifo(service, arr):
        done, lat = 0.0, []
        for a, sv in zip(arr, service):
            done = max(a, done) + sv
            lat.append(done - a)
        lat.sort()
        return {"capacity_solves_per_s": R / sum(service), "solves_per_s": R / (done - arr[0]),
                "p50_ms": 1e3 * lat[R // 2], "p99_ms": 1e3 * lat[min(R - 1, int(0.99 * R))]}

    service, ref = plain(1)            # FP64 pair integrals, FP64 W copy, FP64 PCG
    service_df, _ = plain(0)           # the same with the double-float assembly
    cap_plain = R / sum(service)
    rate = load * cap_plain
    rng = np.random.default_rng(1)
    arr = np.cumsum(rng.exponential(1.0 / rate, R))

    def run_engine(arrivals):
        with M.Server(device=device, precision=precision, hbm_budget=budget) as E:
            for key, gm in geoms.items():
                E.add_geometry(key, gm)
            outs = [np.empty(E.ndof[k]) for k, _ in reqs]
            ids = [0] * R
            t0 = E.now() + 0.01
            i, completed = 0, 0
            while completed < R:
                now = E.now()
                while i < R and t0 + arrivals[i] <= now:
                    ids[i] = E.submit(reqs[i][0], reqs[i][1], outs[i], t_arrival=t0 + arrivals[i])
                    i += 1
                completed += E.progress(block=False)
                if completed == i and i < R:
                    time.sleep(max(0.0, t0 + arrivals[i] - E.now()))
            t_end = E.now()
            res = [E.result(x) for x in ids]
            st = E.stats()
            ndofs = [E.ndof[k] for k in geoms]
        lat = sorted(r["latency_ms"] for r in res)
        diff = max(float(np.linalg.norm(o - r) / max(np.linalg.norm(r), 1e-300)) for o, r in zip(outs, ref))
        return {"solves_per_s": R / (t_end - t0 - arrivals[0]), "p50_ms": lat[R // 2],
                "p99_ms": lat[min(R - 1, int(0.99 * R))], "max_relres": max(r["relres"] for r in res),
                "all_ok": all(r["status"] == 0 for r in res), "maxdiff_vs_plain_fp64": diff,
                "admissions": st["admissions"], "evictions": st["evictions"], "ndofs": ndofs}

    eng = run_engine(arr)
    sat = run_engine(np.zeros(R))
    pl = fifo(service, arr)
    pl["mode"] = ("FP64 pair integrals (far_kernel 1), FP64 copy of W, FP64 PCG; one request at a time, FIFO, "
                  "geometry cache; latencies by the FIFO recurrence")
    pld = fifo(service_df, arr)
    pld["mode"] = "as plain_fp64 but with the double-float assembly of W"
    ndofs = eng.pop("ndofs")
    sat.pop("ndofs")
    return {
        "config": config, "requests": R, "distinct_geometries": len(geoms), "new_geometry_fraction": len(geoms) / R,
        "families": ("squares h=1/24..1/96, three-page books h=1/32,1/48, panel screens (500-13.5k dofs)"
                     if config == "mix" else
                     "squares h=1/24..1/200, cubes with mid-planes h=1/12..1/66, hinged panel screens "
                     "(500-40k dofs)"),
        "dofs_range": [int(min(ndofs)), int(max(ndofs))],
        "hbm_budget_bytes": budget if budget > 0 else "80% of free",
        "arrivals": f"Poisson, rate {rate:.1f}/s = {load} x plain FP64 capacity (seed 1)",
        "plain_fp64": pl,
        "plain_fp64_df_assembly": pld,
        "engine_precision": precision,
        "engine_mixed": eng,
        "engine_mixed_saturated": {"capacity_solves_per_s": sat["solves_per_s"], "p50_ms": sat["p50_ms"],
                                   "p99_ms": sat["p99_ms"], "all_ok": sat["all_ok"]},
        "capacity_vs_plain_fp64": sat["solves_per_s"] / cap_plain,
        "capacity_vs_plain_df_assembly": sat["solves_per_s"] * sum(service_df) / R,
    }


def run_matvec(args):
    """Microbenchmark for profiling: msbem_apply on K seeded vectors of the
    workload's W (warm-up, then `steps` timed products); one JSON line with
    the product kernels' median device time and their HBM rate."""
    import torch
    import paper_2310_09204_gb300 as M
    from paper_2310_09204_gb300 import build as B
    B.build()
    geom = make_workload(args.workload)
    with M.Solver(geom) as S:
        S.assemble()
        X = np.random.default_rng(5).standard_normal((args.matvec, S.n))
        for _ in range(max(args.warmup, 1)):
            S.apply(X, precision=args.matvec_precision)
        ms = sorted(S.apply(X, precision=args.matvec_precision)[1] for _ in range(max(args.steps, 1)))
        torch.cuda.synchronize()
        med = ms[len(ms) // 2]
        hbm, src = measured_peaks()
        nb = MATVEC_BYTES.get(args.matvec_precision, 8) * float(S.n) ** 2
        print(json.dumps({"matvec": args.matvec_precision, "k": args.matvec, "workload": geom.name, "N": S.n,
                          "median_ms": med, "hbm_gbs": nb / (med * 1e-3) / 1e9, "hbm_peak_gbs": hbm,
                          "peak_source": src}), flush=True)


def main():
    args = parse()
    if args.matvec:
        run_matvec(args)
        return
    world, rank, local, pg = dist_setup(args)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank, pg)
        else:
            run_ours(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    main()
