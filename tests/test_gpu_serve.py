"""Serving engine (msbem_server_*): resident geometries, admission by HBM
budget with eviction, continuous batching.

The bar, per request: the density a request gets in the mix of other
requests (other data on its geometry in neighbouring slots, slots refilled
while it runs, other geometries on other streams) is bit for bit the one it
gets alone; and it is the solve of msbem_solve_batch in the same precision
(same per-column arithmetic) -- which the batch tests hold to the oracle.
"""
import numpy as np
import pytest

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import build as B
from paper_2310_09204_gb300 import workloads as WL
from oracle import solver

pytestmark = pytest.mark.gpu

GEOMS = {1: WL.flat_config(), 2: WL.book(8, 2, jitter=True, seed=3), 3: WL.bowtie(6, 2)}


@pytest.fixture(scope="module", autouse=True)
def _build():
    B.build()
    M.lib()


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    keys = rng.choice(sorted(GEOMS), size=n)
    G = rng.uniform(-1, 1, (n, 3))
    return list(zip(keys.tolist(), G))


def _serve(reqs, precision, interleave=False, budget=0.0):
    """Submit reqs (all at once, or a few per progress pass) and run to the end."""
    with M.Server(precision=precision, hbm_budget=budget) as S:
        for k, g in GEOMS.items():
            S.add_geometry(k, g)
        outs, ids = [], []
        for i, (k, g) in enumerate(reqs):
            out = np.full(S.ndof[k], np.nan)
            outs.append(out)
            ids.append(S.submit(k, g, out))
            if interleave and i % 3 == 2:
                S.progress(block=False)
        S.progress(block=True)
        res = [S.result(i) for i in ids]
        return outs, res, S.stats()


@pytest.mark.parametrize("precision", ["df", "mixed", "tc", "mixed-tc", "mixed-fp16"])
def test_alone_and_in_the_mix(precision):
    reqs = _requests(40, 31)       # > 16 on some geometry: slots are refilled
    mix, res, st = _serve(reqs, precision, interleave=True)
    assert st["completed"] == len(reqs) and st["admissions"] == 3
    for i in (0, 7, 19, 33):
        alone, ra, _ = _serve([reqs[i]], precision)
        assert ra[0]["status"] == 0 and res[i]["status"] == 0
        assert np.array_equal(alone[0], mix[i]), i
        assert ra[0]["iters"] == res[i]["iters"]
    for r in res:
        assert r["status"] == 0 and r["relres"] <= 1e-8 and r["latency_ms"] >= 0.0


@pytest.mark.parametrize("precision", ["df", "mixed", "tc", "mixed-tc", "mixed-fp16"])
def test_matches_batch_solve_and_oracle(precision):
    reqs = _requests(12, 32)
    outs, res, _ = _serve(reqs, precision)
    for k, geom in GEOMS.items():
        idx = [i for i, (kk, _) in enumerate(reqs) if kk == k]
        if not idx:
            continue
        G = np.stack([reqs[i][1] for i in idx])
        with M.Solver(geom) as S:
            # the engine sets up the mixed precisions' preconditioner in FP32
            S.assemble().factor(precision="fp32" if precision.startswith("mixed") else "df")
            bt = S.solve_batch(G, precision=precision)
        pb = solver.Problem(geom)
        for j, i in enumerate(idx):
            assert np.linalg.norm(outs[i] - bt["density"][j]) <= 1e-12 * np.linalg.norm(bt["density"][j])
            L = pb.rhs(G[j])
            assert np.linalg.norm(L - pb.W @ outs[i]) <= 1.05e-8 * np.linalg.norm(L)


def test_budget_forces_eviction():
    # room for one geometry at a time: every switch of geometry evicts
    reqs = [(1, np.array([0.0, 0.0, 1.0])), (2, np.array([1.0, 0.5, 0.25])), (3, np.array([0.0, 1.0, 0.0])),
            (1, np.array([0.3, -0.2, 1.0]))]
    with M.Server(precision="df") as S:
        for k, g in GEOMS.items():
            S.add_geometry(k, g)
        fp = sorted(S.footprint(k) for k in GEOMS)
        assert fp[0] > 0 and S.footprint(42) == -1.0
    budget = fp[-1] * 1.01
    assert fp[0] + fp[1] > budget
    outs, res, st = _serve(reqs, "df", budget=budget)
    assert all(r["status"] == 0 for r in res)
    assert st["evictions"] >= 2 and st["admissions"] >= 3
    ref, rr, _ = _serve(reqs, "df")
    for a, b in zip(outs, ref):
        assert np.array_equal(a, b)


def test_errors():
    with M.Server(precision="df") as S:
        S.add_geometry(1, GEOMS[1])
        with pytest.raises(M.MsbemError):
            S.add_geometry(1, GEOMS[1])
        with pytest.raises(M.MsbemError):
            S.submit(99, [0, 0, 1])
        rid = S.submit(1, [0.0, 0.0, 0.0])          # no data: zero density, no iterations
        S.progress(block=True)
        r = S.result(rid)
        assert r["status"] == 0 and r["iters"] == 0


def test_concurrent_contexts_assemble_independently():
    """Two contexts assembling at the same time on two host threads, with
    different singular orders: each W is bit for bit its sequential one
    (the quadrature tables travel with each launch)."""
    import threading
    jobs = [(GEOMS[2], 3), (GEOMS[3], 8), (GEOMS[1], 5)]
    seq = []
    for geom, order in jobs:
        with M.Solver(geom) as S:
            S.assemble(ss_order=order)
            seq.append(S.matrix())
    for _ in range(3):
        out = [None] * len(jobs)

        def work(i):
            geom, order = jobs[i]
            with M.Solver(geom) as S:
                for _ in range(3):
                    S.assemble(ss_order=order)
                out[i] = S.matrix()

        th = [threading.Thread(target=work, args=(i,)) for i in range(len(jobs))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for a, b in zip(out, seq):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["mixed", "mixed-tc"])
def test_density_bar_in_the_engine(precision):
    """With density_tol the engine's mixed-precision results (FP32 set-up of
    the preconditioner, FP32 inner PCG, double-float refinement) meet the 1e-8
    density bar against the oracle's direct solution, and each is still bit
    for bit the result it gets alone."""
    reqs = _requests(24, 41)
    with M.Server(precision=precision, density_tol=1e-9) as S:
        for k, g in GEOMS.items():
            S.add_geometry(k, g)
        outs = [np.full(S.ndof[k], np.nan) for k, _ in reqs]
        ids = [S.submit(k, g, o) for (k, g), o in zip(reqs, outs)]
        S.progress(block=True)
        res = [S.result(i) for i in ids]
    pbs = {k: solver.Problem(g) for k, g in GEOMS.items()}
    for (k, g), x, r in zip(reqs, outs, res):
        assert r["status"] == 0 and r["refinements"] >= 2
        xs = pbs[k].direct(g)
        assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
    with M.Server(precision=precision, density_tol=1e-9) as S:
        k, g = reqs[5]
        S.add_geometry(k, GEOMS[k])
        alone = np.full(S.ndof[k], np.nan)
        S.submit(k, g, alone)
        S.progress(block=True)
    assert np.array_equal(alone, outs[5])
