"""Benchmark: PCG solves/s and p50/p99 latency of the multiscreen hypersingular
BEM hot path on GB300, against the plain FP64 GPU PCG.

Default workload (the bench line): the serving configuration -- a stream of
2000 solve requests (30% new geometries: squares, cubes with mid-planes and
hinged panel screens, 500-40k dofs) served by the engine (msbem_server_*)
under a 160 GB HBM budget, each request solved by mixed-precision PCG to
relative residual 1e-8 with the refinement's density test.  One step = 2000/K
requests (K = --steps); the timed region serves all of them queued at once
(the engine's capacity, `value`).  Beside it: the same stream end to end
(meshes registered as their first request arrives, densities to pinned host
memory; `e2e`), the engine's observed p50/p99 under Poisson arrivals, the
plain FP64 comparator request by request (two forms), and secondary sections
(the three-page book step with its solve forms, the cube, sixteen panel
screens) and the oracle on the host cores.

--workload book64: one step = assembly + preconditioner set-up + PCG solve
of the three-page book (h = 1/64, 12,033 dofs).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank serves its own replica of the stream (no
data-path collective: the solves are independent); timing is max over ranks.
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
# double-float far-field kernel: thread instructions issued per unordered
# separated pair, from an ncu capture of the h=1/32 book (smsp__inst_executed
# x active threads per instruction / pairs: 1.5236e9 x 29.48 / 1.88e7)
FP32_OPS_PER_FAR_PAIR = 2389
# DRAM bytes (read + write) of one far_df_kernel launch, from an ncu capture of
# the h=1/32 book (6,144 triangles: 2.15 MB read + 307.85 MB written), scaled
# to the h=1/64 book by the number of triangle pairs (x16).  Valid for the
# kernel as captured; reset to None when the kernel changes.
FAR_DF_TRAFFIC_BOOK64 = 16 * (2.151168e6 + 307.84512e6)
# the method's work per far pair (the unit of the far-field roofline): 36
# evaluations of w_p w_q / |x_p - y_q| at about 13 FP64 operations each (3
# subtractions, r^2, an rsqrt from an FP32 seed and two Newton steps, one
# accumulate)
METHOD_OPS_PER_FAR_PAIR = 36 * 13
# FP64 FMA rate of this GB300 (instructions per second), measured by a probe
# of this build: the FP64 pipe the method's count refers to
FP64_FMA_PER_S = 0.50e12
# double-float multiply-add on the FP32 pipe (df.cuh df_fma_acc)
FP32_OPS_PER_DF_FMA = 13


C5_REQUESTS = 2000
C5_BUDGET = 160e9
C5_TEXT = ("serving stream: 2000 solve requests (arrival order seed 0; 30% new geometries drawn evenly from "
           "squares h=1/24..1/200, cubes with mid-planes h=1/12..1/66 and hinged panel screens, 500-40k dofs), "
           "g uniform in [-1,1]^3, HBM budget 160 GB, mixed-precision PCG (FP32 inner, double-float residual) "
           "to rel. residual 1e-8 and estimated density error 1e-9")
# the refinement's density target of the engine (msbem_server_opts.density_tol)
C5_DENSITY_TOL = 1e-9
# the oracle's bounded sample of the stream: geometries of at most this many
# triangles (about 6k dofs; the oracle needs seconds for one, minutes for the
# largest of the stream)
C5_CPU_MAX_NT = 12000


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
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving stream (c5: the configuration's 2000; book64: the mix's stream)")
    ap.add_argument("--fp64-prefix", type=int, default=200,
                    help="c5: requests of the stream the all-FP64 comparator is timed on")
    ap.add_argument("--cpu-seconds", type=float, default=25.0,
                    help="c5: seconds of oracle work in the CPU baseline")
    ap.add_argument("--serve-precision", default="mixed", choices=["mixed", "mixed-tc", "mixed-fp16", "df", "tc"])
    ap.add_argument("--no-cube", action="store_true", help="skip the cube-with-mid-planes section")
    ap.add_argument("--no-setup", action="store_true",
                    help="skip the preconditioner set-up section (grouped SPD inverse, double-float and FP32)")
    ap.add_argument("--setup-only", type=int, default=0,
                    help="only invert one synthetic SPD matrix of this order (double-float, then FP32) and print "
                         "the times (for profiling the set-up kernels)")
    ap.add_argument("--no-panels", action="store_true",
                    help="skip the sixteen hinged-panel instances (grouped factorisation, batched solves)")
    ap.add_argument("--workload", default="c5", choices=["c5", "book64", "book48", "book32", "flat"],
                    help="c5: the serving configuration (the bench line); book64: one assembly + set-up + "
                         "solve of the three-page book per step; book48, book32 and flat are for profiling")
    ap.add_argument("--matvec", type=int, default=0,
                    help="microbenchmark only: time the product kernel on K vectors (msbem_apply)")
    ap.add_argument("--matvec-precision", default="df", choices=["df", "fp32", "fp64", "tc", "fp16-tc"])
    return ap.parse_args()


BOOK64_TEXT = ("three-page book h=1/64, N=12033 dofs, 24576 triangles, 48 jittered patches (seed 0), "
               "coarse H=1/4 (33 dofs), g=(1,0.5,0.25), rtol 1e-8")


def book_config(name: str, geom, world: int) -> dict:
    """config of a --workload book64 / profiling line (the same in both arms)."""
    cfg = {"workload": workload_text(name, geom), "parallelism": f"replicas x{world}"}
    if name == "book64":
        cfg["l2"] = "inputs larger than L2 (W 1.16 GB, V 4.8 GB)"
    return cfg


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

def cores_used() -> int:
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)


def c5_config(R: int, K: int, world: int) -> dict:
    """config of the serving line (the same in both arms)."""
    return {"workload": C5_TEXT, "requests": R, "requests_per_step": R // K, "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (W up to 12.7 GB per geometry, 160 GB resident)"}


def c5_small_requests(geoms, reqs, max_nt: int = C5_CPU_MAX_NT):
    """Requests of the stream, in arrival order, whose geometry has at most
    max_nt triangles: the bounded sample the oracle is timed on."""
    return [(k, g) for k, g in reqs if geoms[k].nt <= max_nt]


def run_reference(args, world, rank, pg):
    """The reference arm: the oracle on the host cores, rank 0 only, each step
    one full oracle solve (every phase timed in full).  c5: the requests of the
    serving stream, in arrival order, whose geometry has at most
    C5_CPU_MAX_NT triangles (larger ones take the oracle minutes each);
    book64: the book itself."""
    if rank != 0:
        return
    from oracle import core
    core.build()
    K, W = max(args.steps, 1), max(args.warmup, 0)
    if args.workload == "c5":
        per = max(1, args.serve_requests // K)
        R = per * K
        geoms, reqs = serving_workload_c5(R)
        small = c5_small_requests(geoms, reqs)
        jobs = [(geoms[k], g) for k, g in small]
        config = c5_config(R, K, args.gpus)
        sample = (f"each step one request of the stream: the requests in arrival order whose geometry has at most "
                  f"{C5_CPU_MAX_NT} triangles ({len(small)} of {R}), cycled; every phase in full")
    else:
        geom = make_workload(args.workload)
        jobs = [(geom, geom.g)]
        config = book_config(args.workload, geom, args.gpus)
        sample = "each step one solve of the workload, every phase in full (topology, V, W, set-up, PCG)"
    for w in range(W):
        oracle_solve_seconds(*jobs[w % len(jobs)])
    times, details = [], []
    for k in range(K):
        t, d = oracle_solve_seconds(*jobs[(W + k) % len(jobs)])
        times.append(t)
        details.append(d)
    total = sum(times)
    value = K / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": K,
            "warmup": W, "ms_per_step": 1e3 * total / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
                             "sample": sample, "phases_last": details[-1]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def run_ours(args, world, rank, local, pg):
    if args.workload == "c5":
        run_serving(args, world, rank, local, pg)
    else:
        run_book(args, world, rank, local, pg)


def run_book(args, world, rank, local, pg, secondary=False):
    """One step = assembly + preconditioner set-up + PCG solve of the book (or
    a profiling case).  secondary: the book section of the serving line (no
    serving, cube, panel, end-to-end or CPU sections; returns the dict)."""
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
    roof = far_roofline(far_pairs, statistics.mean(far_ms), "CUDA events around each launch on its stream, "
                                                            "mean over the timed steps")
    if args.far_kernel == 0 and args.workload == "book64":
        roof["traffic"] = FAR_DF_TRAFFIC_BOOK64
    if args.far_kernel == 1:
        roof["kernel"] = "far_fp64_kernel"

    # solve modes on the resident geometry (W and M already built by the last
    # step): the plain FP64 comparator request by request, the double-float
    # path, and the batched / mixed-precision forms on the same 16 requests
    modes = side = None
    if rank == 0 and not args.no_modes:
        modes = solve_modes(S, geom, stream)
        side = modes.pop("_dens")
    roof_mv = matvec_rooflines(S, N, stream) if rank == 0 and not args.no_modes else None

    serving = None
    if rank == 0 and not args.no_serve and not secondary:
        serving = serve_bench(300, local, stream, precision=args.serve_precision)
    cube = None
    if rank == 0 and not args.no_cube and not secondary:
        cube = cube_bench(local, stream)
    panels = None
    if rank == 0 and not args.no_panels and not secondary:
        panels = panels_bench(local, stream)

    # end to end through the C ABI with host buffers: upload (host topology +
    # H2D from pinned memory) + assemble + factor + solve + D2H of the density
    e2e = None
    if not args.no_e2e and not secondary:
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
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not secondary:
        from oracle import core
        core.build()
        t, d = oracle_solve_seconds(geom, g)
        cpu = {"value": 1.0 / t, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
               "sample": "one solve of the same workload, every phase in full (topology, V, W, "
                         "preconditioner set-up, PCG)", "phases": d}

    line = None
    if rank == 0:
        lat = sorted(step_ms)
        p50 = lat[len(lat) // 2]
        p99 = lat[min(len(lat) - 1, int(round(0.99 * (len(lat) - 1))))]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("double-float (2^-48) W, far field and PCG products; FP64 near field and coarse solve "
                      "(FP64 tolerances met)" if args.far_kernel == 0 else "f64"),
            "data": "synthetic",
            "config": book_config(args.workload, geom, world),
            "ndof": N,
            "latency_ms": {"p50": p50, "p99": p99},
            "phases_ms": {k: statistics.mean(p[k] for p in phase) for k in phase[0]},
            "pcg_iters": iters[-1],
            "roofline": roof,
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
        if side is not None:
            line["_dens"] = {"geom": geom, "G": side["G"], "dens": side["dens"]}
            if not secondary and world == 1 and not args.no_cpu_baseline:
                book_oracle_errors(line)
            if not secondary:
                line.pop("_dens", None)
        if not secondary:
            print(json.dumps(line), flush=True)
    S.close()
    return line


def _events(stream, f):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    out = f()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b), out


def solve_modes(S, geom, stream, nreq=16, seed=7, dtol=1e-9):
    """Solves/s and per-request latency of the solve forms on the same nreq
    requests (seeded Neumann data, the first one the workload's g) on the
    resident geometry.  The plain FP64 comparator runs request by request;
    the batched forms take all nreq requests in one call.  The mixed forms
    run with the refinement's density test (density_tol = dtol).  Every result
    is checked by its true relative residual (double-float product), by its
    relative l2 difference from the comparator's, and by its relative l2 error
    against the double-float PCG run to rel. residual 1e-13 (err_vs_tight_df);
    the densities are kept (under '_dens') for the error against the oracle's
    direct solution, computed after the GPU work."""
    rng = np.random.default_rng(seed)
    G = rng.uniform(-1.0, 1.0, (nreq, 3))
    G[0] = geom.g
    batch_forms = (("df_batch", "df"), ("mixed_batch", "mixed"), ("tc_batch", "tc"), ("mixed_tc_batch", "mixed-tc"),
                   ("mixed_fp16_batch", "mixed-fp16"))
    mixed = ("mixed", "mixed-tc", "mixed-fp16")
    for prec in ("fp64", "df", "mixed", "tc", "mixed-tc"):   # warm-up (graphs, FP64 copy and slices of W)
        S.solve(G[0], precision=prec)
    for _, prec in batch_forms:
        S.solve_batch(G, precision=prec)
    tight = S.solve_batch(G, rtol=1e-13, maxit=4000)["density"].copy()
    out = {"requests": nreq, "rtol": 1e-8, "density_tol_mixed": dtol,
           "data": "g_c uniform in [-1,1]^3 (seed 7), g_0 = workload g",
           "forms": {"df": "double-float products (CUDA cores)", "mixed": "FP32 inner PCG, double-float residual",
                     "tc": "double-float products on the tensor cores (integer slices)",
                     "mixed_tc": "FP32 inner PCG, tensor-core double-float residual",
                     "mixed_fp16": "scaled-FP16 tensor-core inner PCG, tensor-core double-float residual"},
           "err_vs_tight_df": {}}
    dens = {}
    ref = np.empty((nreq, S.n))

    def err(D):
        return max(float(np.linalg.norm(D[c] - tight[c]) / np.linalg.norm(tight[c])) for c in range(nreq))
    for name, prec in (("plain_fp64", "fp64"), ("df", "df"), ("mixed", "mixed"), ("tc", "tc"),
                       ("mixed_tc", "mixed-tc")):
        lat, it = [], []
        D = np.empty((nreq, S.n))
        kw = {"density_tol": dtol} if prec in mixed else {}
        for c in range(nreq):
            ms, r = _events(stream, lambda: S.solve(G[c], rtol=1e-8, precision=prec, **kw))
            lat.append(ms)
            it.append(r["iters"])
            D[c] = r["density"]
            if prec == "fp64":
                ref[c] = r["density"]
            else:
                d = np.linalg.norm(r["density"] - ref[c]) / np.linalg.norm(ref[c])
                out.setdefault(name + "_maxdiff_vs_fp64", 0.0)
                out[name + "_maxdiff_vs_fp64"] = max(out[name + "_maxdiff_vs_fp64"], float(d))
        lat.sort()
        dens[name] = D
        out["err_vs_tight_df"][name] = err(D)
        out[name] = {"solves_per_s": 1e3 * nreq / sum(lat), "p50_ms": lat[nreq // 2], "p99_ms": lat[-1],
                     "iters": [int(min(it)), int(max(it))], "mode": "one request per call"}
    for name, prec in batch_forms:
        kw = {"density_tol": dtol} if prec in mixed else {}
        ms, r = _events(stream, lambda: S.solve_batch(G, rtol=1e-8, precision=prec, **kw))
        diff = max(float(np.linalg.norm(r["density"][c] - ref[c]) / np.linalg.norm(ref[c])) for c in range(nreq))
        # true residuals with the double-float product
        Y, _ = S.apply(r["density"])
        L = np.stack([S.rhs(G[c]) for c in range(nreq)])
        rel = float(max(np.linalg.norm(L[c] - Y[c]) / np.linalg.norm(L[c]) for c in range(nreq)))
        dens[name] = r["density"].copy()
        out["err_vs_tight_df"][name] = err(r["density"])
        out[name] = {"solves_per_s": 1e3 * nreq / ms, "batch_ms": ms, "iters": [int(r["iters"].min()),
                     int(r["iters"].max())], "max_true_relres": rel, "maxdiff_vs_fp64": diff,
                     "mode": f"{nreq} requests in one call"}
    # the residual test alone (no density test), for the cost of the density test
    ms, r = _events(stream, lambda: S.solve_batch(G, rtol=1e-8, precision="mixed-tc"))
    out["mixed_tc_batch_residual_only"] = {"solves_per_s": 1e3 * nreq / ms, "batch_ms": ms,
                                           "err_vs_tight_df": err(r["density"])}
    base = out["plain_fp64"]["solves_per_s"]
    out["speedup_vs_plain_fp64"] = {k: out[k]["solves_per_s"] / base
                                    for k in ("df", "mixed", "tc", "mixed_tc") + tuple(n for n, _ in batch_forms)}
    out["_dens"] = {"G": G, "dens": dens}
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


SETUP_ORDER = 7407   # the wire basket of the cube with mid-planes at h = 1/66


def setup_bench(n: int = SETUP_ORDER, reps: int = 3) -> dict:
    """The preconditioner set-up's inversion alone (msbem_spd_inverse_group,
    Sec. 5 eq. jumpSplit: the blocks of M(H;h) inverted explicitly) on one
    synthetic SPD matrix of the order of the cube's wire basket: B B^T / n + I,
    B uniform in (-1, 1), seed 1.  Double-float: n / 32 steps of pivot, panel,
    slicing and the tensor-core update (orders >= 2048); FP32: the CUDA-core
    update.  Times are CUDA events around the call on its stream (best of
    `reps`); `update_roofline` relates the double-float steps to the pass over
    the FP64 matrix that every step makes (16 n^2 bytes read and written)."""
    import math
    import torch
    import paper_2310_09204_gb300 as M
    dev = torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device=dev).manual_seed(1)
    B = torch.rand(n, n, dtype=torch.float64, device=dev, generator=g) * 2 - 1
    A0 = B @ B.T / n + torch.eye(n, dtype=torch.float64, device=dev)
    del B
    eye = torch.eye(n, dtype=torch.float64, device=dev)
    out = {"order": n, "matrix": "B B^T / n + I, B uniform(-1, 1), seed 1 (cube h=1/66 wire-basket order)"}
    for prec in ("df", "fp32"):
        best, st, A = None, None, None
        for _ in range(reps):
            A = A0.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = M.msbem_spd_inverse_group([A], precision=prec)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        err = (A @ A0 - eye).abs().max().item()
        out[prec] = {"ms": best, "status": st[0], "max_abs_AX_minus_I": err}
    steps = math.ceil(n / 32)
    peak, src = measured_peaks()
    bound_ms = steps * 16.0 * n * n / (peak * 1e9) * 1e3
    out["update_roofline"] = {"steps": steps, "bytes_per_step": 16.0 * n * n, "hbm_gbs": peak, "peak_source": src,
                              "hbm_bound_ms": bound_ms, "df_frac_of_hbm_bound": bound_ms / out["df"]["ms"]}
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


# --------------------------------------------------------------------------
# the serving configuration: the default workload of the bench line
# --------------------------------------------------------------------------



def engine_run(geoms, ndof, reqs, device, precision="mixed", budget=C5_BUDGET, arrivals=None, out="device",
               register="all", density_tol=C5_DENSITY_TOL, sample=(), admission_threads=0):
    """Serve `reqs` [(key, g)] on a fresh engine.

    arrivals None: every request is queued at once (saturated: the engine's
    capacity); else Poisson arrival offsets in seconds, submitted in real time.
    out "device": densities into one device buffer; "host": into pinned host
    memory.  register "all": every geometry registered before the timed region
    (host copies held by the engine); "lazy": a geometry is registered when its
    first request arrives, inside the timed region.  The timed region is
    bracketed by a device-wide synchronize and CUDA events on both sides.
    Returns the measurements, the engine's statistics and the densities of the
    requests listed in `sample` (host copies, taken after the timed region)."""
    import torch
    import paper_2310_09204_gb300 as M
    R = len(reqs)
    offs = np.zeros(R + 1, np.int64)
    offs[1:] = np.cumsum([ndof[k] for k, _ in reqs])
    if out == "device":
        buf = torch.empty(int(offs[-1]), dtype=torch.float64, device=f"cuda:{device}")
    else:
        buf = torch.empty(int(offs[-1]), dtype=torch.float64).pin_memory()
    views = [buf[int(offs[i]):int(offs[i + 1])] for i in range(R)]
    gpin = torch.from_numpy(np.array([g for _, g in reqs], np.float64)).pin_memory().numpy()
    E = M.Server(device=device, precision=precision, hbm_budget=budget, density_tol=density_tol,
                 admission_threads=admission_threads)
    registered = set()
    try:
        if register == "all":
            for key, gm in geoms.items():
                E.add_geometry(key, gm, ndof=ndof[key])
                registered.add(key)
        st0 = E.stats()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        t0 = E.now()
        ids = []
        i = completed = 0
        while completed < R:
            now = E.now()
            while i < R and (arrivals is None or t0 + arrivals[i] <= now):
                key = reqs[i][0]
                if key not in registered:
                    E.add_geometry(key, geoms[key], ndof=ndof[key])
                    registered.add(key)
                ta = t0 + (arrivals[i] if arrivals is not None else 0.0)
                ids.append(E.submit(key, gpin[i], views[i], t_arrival=ta))
                i += 1
            completed += E.progress(block=False)
            if arrivals is not None and completed == i and i < R:
                time.sleep(max(0.0, t0 + arrivals[i] - E.now()))
        torch.cuda.synchronize()
        ev1.record()
        ev1.synchronize()
        wall = E.now() - t0
        res = [E.result(x) for x in ids]
        st1 = E.stats()
    finally:
        E.close()
    lat = sorted(r["latency_ms"] for r in res)
    dens = {i: views[i].cpu().numpy().copy() for i in sample}
    h2d = sum(geoms[k].xyz.nbytes + 4 * geoms[k].tri.size + geoms[k].coarse_xyz.nbytes +
              4 * geoms[k].coarse_tri.size + 8 * geoms[k].nt for k in registered) + 24 * R
    return {"seconds": ev0.elapsed_time(ev1) / 1e3, "wall_seconds": wall, "solves_per_s": R / (ev0.elapsed_time(ev1) / 1e3),
            "p50_ms": lat[R // 2], "p99_ms": lat[min(R - 1, int(0.99 * R))],
            "max_relres": max(r["relres"] for r in res), "all_ok": all(r["status"] == 0 for r in res),
            "statuses": sorted({r["status"] for r in res}),
            "refinements": [int(min(r["refinements"] for r in res)), int(max(r["refinements"] for r in res))],
            "admissions": int(st1["admissions"] - st0["admissions"]),
            "evictions": int(st1["evictions"] - st0["evictions"]),
            "far_ms": st1["far_ms"] - st0["far_ms"], "far_pairs": int(st1["far_pairs"] - st0["far_pairs"]),
            "assemble_ms": st1["assemble_ms"] - st0["assemble_ms"], "factor_ms": st1["factor_ms"] - st0["factor_ms"],
            "launches": int(st1["launches"] - st0["launches"]),
            "h2d_bytes": int(h2d), "d2h_bytes": int(8 * offs[-1]) if out == "host" else 0}, dens


def comparator_run(geoms, reqs, device, far_kernel, budget=C5_BUDGET, tight=()):
    """The plain FP64 comparator, request by request in arrival order: a
    geometry is assembled (far_kernel 1: FP64 pair integrals; 0: the
    double-float pair integrals) and factored on its first use and cached
    under the HBM budget (least recently used evicted first), then each request
    is solved by FP64 PCG (FP64 copy of W, FP64 block inverses) to rel.
    residual 1e-8.  Returns every request's service time and the densities of
    the requests in `tight`, each re-solved after its timed service by the
    double-float PCG to rel. residual 1e-13 (the reference the densities of
    both arms are measured against; untimed)."""
    import torch
    import paper_2310_09204_gb300 as M
    cache, service, used, refs, plain = {}, [], {}, {}, {}
    home = M.Solver(None, device=device)

    def bytes_of(key):
        n = float(cache[key].n)
        return 16.0 * n * n + 8.0 * n * 2000
    try:
        for i, (key, g) in enumerate(reqs):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if key not in cache:
                cache[key] = M.Solver(geoms[key], device=device, share=home)
                while sum(bytes_of(k) for k in cache) > budget and len(cache) > 1:
                    old = min((k for k in cache if k != key), key=lambda k: used.get(k, -1))
                    cache.pop(old).close()
                cache[key].assemble(far_kernel=far_kernel).factor()
            used[key] = i
            out = cache[key].solve(g, rtol=1e-8, precision="fp64")
            torch.cuda.synchronize()
            service.append(time.perf_counter() - t0)
            if i in tight:
                plain[i] = out["density"].copy()
                refs[i] = cache[key].solve(g, rtol=1e-13, maxit=4000)["density"].copy()
    finally:
        for S in cache.values():
            S.close()
        home.close()
    return service, refs, plain


def fifo_latency(service, arr):
    """Latencies of a one-at-a-time server with the given service times at the
    given arrival offsets: done_i = max(arrival_i, done_{i-1}) + service_i."""
    done, lat = 0.0, []
    for a, sv in zip(arr, service):
        done = max(a, done) + sv
        lat.append(done - a)
    lat.sort()
    R = len(lat)
    return {"p50_ms": 1e3 * lat[R // 2], "p99_ms": 1e3 * lat[min(R - 1, int(0.99 * R))]}


def oracle_solve_seconds(geom, g) -> tuple[float, dict]:
    """One oracle solve on the host cores, as the oracle stands and every phase
    in full: topology (fine and coarse), assembly (the pair matrix V, the
    contraction to W, closed cells), preconditioner set-up, PCG to rel.
    residual 1e-8."""
    from oracle import solver
    t = {}
    t0 = time.perf_counter()
    P = solver.Problem(geom, assemble=False)
    t1 = time.perf_counter()
    P.assemble()
    t2 = time.perf_counter()
    P.factor()
    t3 = time.perf_counter()
    res = P.solve(g, rtol=1e-8)
    t4 = time.perf_counter()
    t = {"topology_s": t1 - t0, "assemble_s": t2 - t1, "factor_s": t3 - t2, "solve_s": t4 - t3,
         "iters": int(res.iters), "ndof": int(P.ndof)}
    return t4 - t0, t


def c5_ndof(geoms):
    """Dof count of every geometry (host topology, threads: the C call
    releases the interpreter lock)."""
    import concurrent.futures as cf
    import paper_2310_09204_gb300 as M
    keys = list(geoms)
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        n = list(ex.map(lambda k: M.msbem_mesh_dofs(geoms[k].xyz, geoms[k].tri)[0], keys))
    return dict(zip(keys, n))


def far_roofline(far_pairs: int, far_ms: float, source: str) -> dict:
    """Roofline of the far-field kernel from its unit count (unordered pairs
    sharing no vertex) and its event-timed duration.  achieved counts the
    method's work, 36 evaluations x 13 operations per pair (an FP64 rsqrt by
    two Newton steps from an FP32 seed, 3 subtractions, r^2, one accumulate);
    frac_pipe counts the FP32 instructions the double-float kernel issues."""
    peak = SM_COUNT * FP32_LANES * SM_MAX_MHZ * 1e6
    sec = far_ms / 1e3
    method = far_pairs * METHOD_OPS_PER_FAR_PAIR
    issued = far_pairs * FP32_OPS_PER_FAR_PAIR
    return {"kernel": "far_df_kernel (double-float on the FP32 pipe)", "bound": "alu",
            "achieved": method / sec / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s", "frac": method / sec / peak,
            "traffic": None,
            "traffic_note": "per launch it varies with the geometry; the ncu capture of the h=1/32 book measured "
                            "16.5 DRAM bytes per unit (2.15 MB read + 307.8 MB written for 1.88e7 pairs: the V "
                            "output only)",
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz (no FP32 entry in MEASURED_PEAKS.json)",
            "work_per_unit": f"{METHOD_OPS_PER_FAR_PAIR} method operations per pair (36 x 13)",
            "frac_pipe": issued / sec / peak,
            "pipe_ops_per_unit": FP32_OPS_PER_FAR_PAIR,
            "vs_fp64_pipe": method / sec / FP64_FMA_PER_S,
            "units": int(far_pairs), "kernel_ms": far_ms, "timing": source}


def run_serving(args, world, rank, local, pg):
    """The bench line: the serving engine on the serving configuration's
    stream.  One step = R/K requests of the stream (K = --steps); the timed
    region serves all K steps' requests at once (saturated: the engine's
    capacity).  W = --warmup steps of a separate warm-up stream of small
    geometries run on another engine first."""
    import torch
    import paper_2310_09204_gb300 as M
    from paper_2310_09204_gb300 import build as B
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    K, W = max(args.steps, 1), max(args.warmup, 0)
    per = max(1, args.serve_requests // K)
    R = per * K
    geoms, reqs = serving_workload_c5(R)
    ndof = c5_ndof(geoms)
    sample = sorted(np.random.default_rng(11).choice(R, min(40, R), replace=False).tolist())
    if W:
        wg, wr = serving_workload_c5(W * per, seed=7, small=True)
        engine_run(wg, c5_ndof(wg), wr, local)
    clocks = Clocks(local)
    barrier(pg)
    clocks.start()
    run, dens = engine_run(geoms, ndof, reqs, local, sample=sample)
    barrier(pg)
    ck = clocks.stop()
    value, total_s = aggregate(pg, world, R, run["seconds"], dev)
    e2e = None
    if not args.no_e2e:
        erun, _ = engine_run(geoms, ndof, reqs, local, out="host", register="lazy")
        e2e_value, _ = aggregate(pg, world, R, erun["seconds"], dev)
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(erun["h2d_bytes"] / K),
               "d2h_bytes_per_step": int(erun["d2h_bytes"] / K),
               "how": "the same stream through the engine's C ABI: each geometry registered (host copy and dof "
                      "count) when its first request arrives, its mesh uploaded at admission, every density "
                      "copied to pinned host memory; bytes are the meshes, g and densities",
               "max_relres": erun["max_relres"], "all_ok": erun["all_ok"]}
    if rank != 0:
        return
    serving = {"requests": R, "distinct_geometries": len(geoms), "dofs_range": [min(ndof.values()), max(ndof.values())],
               "engine_saturated": run}
    comp = {}
    book = cube = panels = None
    if not args.no_serve:
        svc, refs, plain = comparator_run(geoms, reqs, local, 0, tight=set(sample))
        cap_df = R / sum(svc)
        # the comparator given the order that suits a one-at-a-time server best
        # (requests grouped by geometry, in order of first appearance), as the
        # engine's offline run may reorder
        first = {}
        for i, (k, _) in enumerate(reqs):
            first.setdefault(k, i)
        grouped = sorted(range(R), key=lambda i: (first[reqs[i][0]], i))
        svc_g, _, _ = comparator_run(geoms, [reqs[i] for i in grouped], local, 0)
        cap_df_g = R / sum(svc_g)
        P = min(R, args.fp64_prefix)
        svc64, _, _ = comparator_run(geoms, reqs[:P], local, 1)
        cap64_prefix = P / sum(svc64)
        # all-FP64 capacities estimated from the double-float-assembly ones by
        # the ratio measured on the same first P requests
        r64 = cap64_prefix / (P / sum(svc[:P]))
        rate = cap_df
        arr = np.cumsum(np.random.default_rng(1).exponential(1.0 / rate, R))
        pois, _ = engine_run(geoms, ndof, reqs, local, arrivals=arr)
        eng_err = max(float(np.linalg.norm(dens[i] - refs[i]) / np.linalg.norm(refs[i])) for i in sample)
        pl_err = max(float(np.linalg.norm(plain[i] - refs[i]) / np.linalg.norm(refs[i])) for i in sample)
        comp = {
            "plain_fp64_df_assembly": {
                "capacity_solves_per_s": cap_df, **fifo_latency(svc, arr),
                "mode": "FP64 PCG (FP64 copy of W, FP64 block inverses) request by request in arrival order, "
                        "W from the double-float pair integrals, LRU geometry cache under 160 GB; latencies by "
                        "the FIFO recurrence of a one-at-a-time server from its measured service times"},
            "plain_fp64_df_assembly_grouped": {
                "capacity_solves_per_s": cap_df_g,
                "mode": "as plain_fp64_df_assembly with the requests grouped by geometry (order of first "
                        "appearance): each geometry assembled once"},
            "plain_fp64": {
                "capacity_solves_per_s_estimated": cap_df * r64,
                "capacity_solves_per_s_grouped_estimated": cap_df_g * r64,
                "measured_on_first_requests": {"requests": P, "capacity_solves_per_s": cap64_prefix,
                                               "df_assembly_capacity_solves_per_s": P / sum(svc[:P]),
                                               **fifo_latency(svc64, arr[:P])},
                "mode": f"as plain_fp64_df_assembly with FP64 pair integrals (far_kernel 1); timed on the first "
                        f"{P} requests of the stream only (the whole stream takes ~16 min): its capacities are the "
                        f"double-float-assembly ones times the ratio measured on those requests ({r64:.3f})"}}
        serving.update({
            "engine_at_load": pois, "arrivals": f"Poisson, rate {rate:.2f}/s = the plain_fp64_df_assembly "
                                                f"capacity (seed 1)",
            "comparators": comp,
            "speedup_vs_plain_fp64_df_assembly": value / world / cap_df,
            "speedup_vs_plain_fp64_df_assembly_grouped": value / world / cap_df_g,
            "speedup_vs_plain_fp64": value / world / (cap_df * r64),
            "speedup_vs_plain_fp64_grouped": value / world / (cap_df_g * r64),
            "offline_vs_online": "value: every request queued at once (offline; the engine batches the requests of "
                                 "a resident geometry); engine_at_load: requests submitted as they arrive",
            "err_vs_tight_df": {"engine_max": eng_err, "plain_fp64_max": pl_err, "requests": len(sample),
                                "reference": "double-float PCG to rel. residual 1e-13 on the same W (the path "
                                             "held to the oracle by the parity tests), 40 seeded requests"}})
    if not args.no_modes:
        import copy
        bargs = copy.copy(args)
        bargs.workload = "book64"
        book = run_book(bargs, 1, 0, local, None, secondary=True)
    if not args.no_cube:
        cube = cube_bench(local, torch.cuda.current_stream(dev))
    if not args.no_panels:
        panels = panels_bench(local, torch.cuda.current_stream(dev))
    setup = None if args.no_setup else setup_bench()
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = c5_cpu_baseline(geoms, reqs, budget_s=args.cpu_seconds)
        if book is not None:
            book_oracle_errors(book)
    if book is not None:
        book.pop("_dens", None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * total_s / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "mixed: FP32 inner PCG; double-float (2^-48) W, far field, refinement residual and block "
                 "inverses; FP64 near field and coarse solve (FP64 tolerances met)",
        "data": "synthetic",
        "config": c5_config(R, K, world),
        "latency_ms": ({"p50": serving["engine_at_load"]["p50_ms"], "p99": serving["engine_at_load"]["p99_ms"],
                        "at": serving["arrivals"]} if "engine_at_load" in serving else None),
        "vs_plain_fp64_gpu_pcg": ({k: serving[k] for k in ("speedup_vs_plain_fp64_df_assembly",
                                                           "speedup_vs_plain_fp64_df_assembly_grouped",
                                                           "speedup_vs_plain_fp64",
                                                           "speedup_vs_plain_fp64_grouped")} if comp else None),
        "roofline": far_roofline(run["far_pairs"], run["far_ms"],
                                 "CUDA events inside each assembly on its stream, summed over the timed region"),
        "serving": serving, "book": book, "cube": cube, "panels16": panels, "setup_inverse": setup,
        "clocks": ck, "gpu_launches": run["launches"], "e2e": e2e, "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def c5_cpu_baseline(geoms, reqs, budget_s: float = 25.0) -> dict:
    """The oracle on the host cores on a bounded sample of the stream: the
    requests in arrival order whose geometry has at most C5_CPU_MAX_NT
    triangles, each a full oracle solve (no phase sampled or scaled), until
    budget_s seconds of work or 20 requests."""
    from oracle import core
    core.build()
    times, phases = [], []
    for key, g in c5_small_requests(geoms, reqs):
        t, d = oracle_solve_seconds(geoms[key], g)
        times.append(t)
        phases.append(d)
        if sum(times) >= budget_s or len(times) >= 20:
            break
    return {"value": len(times) / sum(times), "unit": UNIT, "cores": cores_used(), "kind": "oracle",
            "sample": f"the first {len(times)} requests of the stream (arrival order) whose geometry has at most "
                      f"{C5_CPU_MAX_NT} triangles ({min(p['ndof'] for p in phases)}-{max(p['ndof'] for p in phases)}"
                      f" dofs); each a full oracle solve: topology, V, W, preconditioner set-up, PCG (larger "
                      f"geometries take the oracle minutes each, so the sample favours it)",
            "seconds": sum(times), "phases_last": phases[-1]}


def book_oracle_errors(book: dict) -> None:
    """Relative l2 error of every solve form's densities on the book against
    the oracle's direct (Cholesky) solution of its own W (untimed, after the
    GPU work); fills book['solve_modes']['err_vs_oracle']."""
    from oracle import solver
    side = book.pop("_dens", None)
    if not side:
        return
    import scipy.linalg as sla
    P = solver.Problem(side["geom"])
    cf = sla.cho_factor(P.W, lower=True)
    X = np.stack([sla.cho_solve(cf, P.rhs(g)) for g in side["G"]])
    err = {}
    for name, D in side["dens"].items():
        err[name] = max(float(np.linalg.norm(D[c] - X[c]) / np.linalg.norm(X[c])) for c in range(len(X)))
    book["solve_modes"]["err_vs_oracle"] = {
        "max_relative_l2": err, "reference": "oracle: FP64 W from its own quadrature, dense Cholesky solve"}


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
    if args.setup_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"setup_inverse": setup_bench(args.setup_only, reps=1)}), flush=True)
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
