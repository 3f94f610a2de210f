"""The serving benchmark's request streams (host only): seeded and
reproducible, geometries of the stated families and sizes."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
import paper_2310_09204_gb300 as M  # noqa: E402


def test_c5_stream_is_seeded_and_sized():
    g1, r1 = bench.serving_workload_c5(40, seed=3)
    g2, r2 = bench.serving_workload_c5(40, seed=3)
    assert len(r1) == 40 and sorted(g1) == sorted(g2)
    for (k1, a), (k2, b) in zip(r1, r2):
        assert k1 == k2 and np.array_equal(a, b)
        assert np.all(np.abs(a) <= 1.0)
    for k in g1:
        assert np.array_equal(g1[k].xyz, g2[k].xyz) and np.array_equal(g1[k].tri, g2[k].tri)
    # every request names a geometry seen at or before it; new ones appear in key order
    seen = 0
    for k, _ in r1:
        assert 1 <= k <= seen + 1
        seen = max(seen, k)
    fams = {g.meta.get("family", "panels") for g in g1.values()}
    assert fams <= {"square", "cube", "panels"}
    for g in g1.values():
        n = M.msbem_mesh_dofs(g.xyz, g.tri)[0]
        assert 500 <= n <= 40000, (g.name, n)


def test_mix_stream_is_seeded():
    g1, r1 = bench.serving_workload(30, seed=5)
    g2, r2 = bench.serving_workload(30, seed=5)
    assert [k for k, _ in r1] == [k for k, _ in r2]
    assert all(np.array_equal(a, b) for (_, a), (_, b) in zip(r1, r2))
    assert all(np.array_equal(g1[k].tri, g2[k].tri) for k in g1)


def test_fifo_latency_recurrence():
    """A one-at-a-time server: done_i = max(arrival_i, done_{i-1}) + service_i."""
    lat = bench.fifo_latency([1.0, 1.0, 1.0, 1.0], [0.0, 0.5, 5.0, 5.0])
    # latencies 1.0, 1.5, 1.0, 2.0 -> sorted 1.0, 1.0, 1.5, 2.0
    assert lat["p50_ms"] == 1500.0 and lat["p99_ms"] == 2000.0


def test_small_request_sample_and_warmup_stream():
    geoms, reqs = bench.serving_workload_c5(60, seed=0)
    small = bench.c5_small_requests(geoms, reqs)
    assert small and all(geoms[k].nt <= bench.C5_CPU_MAX_NT for k, _ in small)
    # arrival order is kept
    pos = [next(i for i, r in enumerate(reqs) if r[0] == k and np.array_equal(r[1], g)) for k, g in small]
    assert pos == sorted(pos)
    wg, wr = bench.serving_workload_c5(30, seed=7, small=True)
    for g in wg.values():
        assert g.meta.get("family", "panels") in ("square", "cube")
        assert M.msbem_mesh_dofs(g.xyz, g.tri)[0] <= 7000


def test_c5_config_is_the_same_in_both_arms():
    assert bench.c5_config(2000, 20, 1) == bench.c5_config(2000, 20, 1)
    cfg = bench.c5_config(2000, 20, 1)
    assert cfg["requests"] == 2000 and cfg["requests_per_step"] == 100 and cfg["workload"] == bench.C5_TEXT
