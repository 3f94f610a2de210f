"""Multiscreens of unit squares hinged at random dihedral angles (the batched
+ mixed-precision workload family): parity with the oracle on small
instances (junction lines of up to four squares, with and without a coarse
space), and the sixteen full-size instances solved in the mixed precision
against the double-float path, with the error reported per instance."""
import math

import numpy as np
import pytest

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import build as B
from paper_2310_09204_gb300 import workloads as WL
from oracle import solver

pytestmark = pytest.mark.gpu

SMALL = [WL.panels(7, n=8, n_coarse=2), WL.panels(5, n=8, n_coarse=2), WL.panels(11, n=12),
         WL.panels(2, n=6, angle_range=(30.0, 45.0))]


@pytest.fixture(scope="module", autouse=True)
def _build():
    B.build()
    M.lib()


def _energy_rel(x, ref, W):
    e = x - ref
    return math.sqrt(max(e @ W @ e, 0.0)) / math.sqrt(ref @ W @ ref)


@pytest.mark.parametrize("geom", SMALL, ids=lambda g: g.name)
def test_panels_against_oracle(geom):
    pb = solver.Problem(geom)
    pb.factor()
    ref = pb.solve(rtol=1e-8)
    with M.Solver(geom) as S:
        v, s = S.dof_map()
        assert np.array_equal(v, pb.top.dof_vertex) and np.array_equal(s, pb.top.dof_sector)
        S.assemble()
        Wg = S.matrix()
        scale = np.abs(pb.W).max()
        assert np.abs(Wg - pb.W).max() <= 1e-12 * scale
        d = np.abs(np.diag(Wg) - np.diag(pb.W)) / np.abs(np.diag(pb.W))
        assert d.max() <= 1e-12
        S.factor()
        out = S.solve(geom.g, rtol=1e-8)
        assert abs(out["iters"] - ref.iters) <= 1
        fx = S.solve(geom.g, rtol=0.0, maxit=ref.iters, fixed=True)
        assert np.linalg.norm(fx["density"] - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
        assert _energy_rel(fx["density"], ref.x, pb.W) <= 1e-8
        mx = S.solve(geom.g, rtol=1e-8, precision="mixed")
        L = pb.rhs(geom.g)
        assert np.linalg.norm(L - pb.W @ mx["density"]) <= 1.05e-8 * np.linalg.norm(L)


def test_sixteen_instances_mixed_vs_double_float():
    errs = []
    for geom in WL.panels_config():
        rng = np.random.default_rng(geom.meta["seed"])
        G = rng.uniform(-1, 1, (4, 3))
        G[0] = geom.g
        with M.Solver(geom) as S:
            S.assemble().factor()
            mx = S.solve_batch(G, rtol=1e-8, precision="mixed")
            df = S.solve_batch(G, rtol=1e-10)
            Y, _ = S.apply(mx["density"])
            for c in range(len(G)):
                L = S.rhs(G[c])
                assert np.linalg.norm(L - Y[c]) <= 1.05e-8 * np.linalg.norm(L)
                e = np.linalg.norm(mx["density"][c] - df["density"][c]) / np.linalg.norm(df["density"][c])
                errs.append(e)
                assert e <= 1e-6, (geom.name, c, e)
    print("mixed vs double-float, max relative l2 error per request:", max(errs))
