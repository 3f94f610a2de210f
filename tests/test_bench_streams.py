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
