"""The cube with its three mid-planes (eight closed cells): the library
assembles W + rho Z Z^T (closed-cell reading), and its solves are held to the
oracle's augmented system."""
import math

import numpy as np
import pytest

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import build as B
from paper_2310_09204_gb300 import workloads as WL
from oracle import solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    B.build()
    M.lib()


def _energy_rel(x, ref, W):
    e = x - ref
    return math.sqrt(max(e @ W @ e, 0.0)) / math.sqrt(ref @ W @ ref)


@pytest.mark.parametrize("n", [4, 6, 12])
def test_cube_against_oracle(n):
    geom = WL.cube_midplanes(n, 2 if n < 12 else 6)
    pb = solver.Problem(geom)
    pb.factor()
    with M.Solver(geom) as S:
        S.assemble()
        Z, rho = S.cells()
        assert Z.shape[1] == 8 and np.array_equal(Z, pb.Z)
        assert abs(rho - pb.rho) <= 1e-13 * pb.rho
        Wg = S.matrix()
        scale = np.abs(pb.W).max()
        assert np.abs(Wg - pb.W).max() <= 1e-12 * scale
        d = np.abs(np.diag(Wg) - np.diag(pb.W)) / np.abs(np.diag(pb.W))
        assert d.max() <= 1e-12
        S.factor()
        for g in (geom.g, np.array([0.2, -0.9, 0.4])):
            ref = pb.solve(g, rtol=1e-8)
            out = S.solve(g, rtol=1e-8)
            assert abs(out["iters"] - ref.iters) <= 1
            fx = S.solve(g, rtol=0.0, maxit=ref.iters, fixed=True)
            assert np.linalg.norm(fx["density"] - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
            assert _energy_rel(fx["density"], ref.x, pb.W) <= 1e-8
            assert np.abs(Z.T @ out["density"]).max() <= 1e-7 * np.linalg.norm(out["density"])
            mx = S.solve(g, rtol=1e-8, precision="mixed")
            L = pb.rhs(g)
            assert np.linalg.norm(L - pb.W @ mx["density"]) <= 1.05e-8 * np.linalg.norm(L)
            # the augmented solution solves the original singular system
            assert np.linalg.norm(L - pb.W0 @ out["density"]) <= 1e-7 * np.linalg.norm(L)


@pytest.mark.parametrize("geom,rows", [(WL.book(8, 2, jitter=True, seed=3), 64), (WL.cube_midplanes(6, 2), 128),
                                       (WL.panels(7, n=8, n_coarse=2), 192)], ids=lambda x: getattr(x, "name", x))
def test_panel_assembly(geom, rows):
    """V in row panels: W equals the one-piece assembly to rounding and the
    oracle to the parity bar; the solves agree."""
    pb = solver.Problem(geom)
    with M.Solver(geom) as S:
        S.assemble()
        W1 = S.matrix()
        S.assemble(panel_rows=rows)
        Wp = S.matrix()
        scale = np.abs(W1).max()
        # another summation order of the same double-float terms (each entry sums
        # ~100 terms with cancellation at 2^-48 per operation), and the panels
        # sum W[nu, nu'] and W[nu', nu] in different orders: both at rounding
        # level, ten times below the parity bar
        assert np.abs(Wp - W1).max() <= 1e-13 * scale
        assert np.abs(Wp - Wp.T).max() <= 1e-13 * scale
        assert np.abs(Wp - pb.W).max() <= 1e-12 * scale
        d = np.abs(np.diag(Wp) - np.diag(pb.W)) / np.abs(np.diag(pb.W))
        assert d.max() <= 1e-12
        S.factor()
        out = S.solve(geom.g, rtol=1e-8)
        pb.factor()
        ref = pb.solve(geom.g, rtol=1e-8)
        assert abs(out["iters"] - ref.iters) <= 1
        with pytest.raises(M.MsbemError) as e:
            S.assemble(panel_rows=100)
        assert e.value.status == -1
        with pytest.raises(M.MsbemError) as e:
            S.assemble(panel_rows=64, far_kernel=1)
        assert e.value.status == -1
