"""FP32 set-up of the preconditioner (msbem_precond_opts.precision = 1): the
face and wire-basket blocks inverted by Gauss-Jordan in FP32 (symmetrised),
the coarse block in double-float.  The mixed-precision solves read FP32
inverses in their inner PCG anyway, so their results must meet the same bars
as with the double-float set-up; the inverse itself is checked through a
one-patch geometry whose preconditioner is W^{-1}."""
import numpy as np
import pytest
import scipy.linalg as sla

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import build as B
from paper_2310_09204_gb300 import workloads as WL
from oracle import solver

pytestmark = pytest.mark.gpu

SMALL = [WL.book(8, 2, jitter=True, seed=3), WL.bowtie(6, 2), WL.cube_midplanes(6, 2), WL.panels(7, n=8, n_coarse=2)]


@pytest.fixture(scope="module", autouse=True)
def _build():
    B.build()
    M.lib()


def test_fp32_inverse_of_one_patch():
    geom = WL.book(8, 2, jitter=False)
    geom.patch = np.zeros(geom.nt, np.int32)
    with M.Solver(geom) as S:
        S.assemble().factor(use_coarse=0, precision="fp32")
        W = S.matrix()
        L = S.rhs(geom.g)
        x = S.solve(geom.g, rtol=0.0, maxit=1, fixed=True)["density"]   # one step: M L = A^{-1} L
        xs = sla.cho_solve(sla.cho_factor(W, lower=True), L)
        kappa = np.linalg.cond(W)
        err = np.linalg.norm(x - xs) / np.linalg.norm(xs)
        print("one-patch FP32 inverse: relative error", err, "kappa(W)", kappa)
        assert err <= 32 * kappa * 2.0 ** -24


@pytest.mark.parametrize("geom", SMALL, ids=lambda g: g.name)
def test_mixed_solves_with_fp32_setup(geom):
    pb = solver.Problem(geom)
    rng = np.random.default_rng(41)
    G = np.vstack([geom.g, rng.uniform(-1, 1, (2, 3))])
    with M.Solver(geom) as S:
        S.assemble().factor()
        ref = S.solve_batch(G, rtol=1e-8, precision="mixed-tc", density_tol=1e-9)
        S.factor(precision="fp32")
        for prec in ("mixed", "mixed-tc", "mixed-fp16"):
            out = S.solve_batch(G, rtol=1e-8, precision=prec, density_tol=1e-9)
            for c, g in enumerate(G):
                xs = pb.direct(g)
                L = pb.rhs(g)
                x = out["density"][c]
                assert np.linalg.norm(L - pb.W @ x) <= 1.05e-8 * np.linalg.norm(L), (prec, c)
                assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs), (prec, c)
            if prec == "mixed-tc":
                # the inner iterations barely change with an FP32 set-up
                assert out["iters"].max() <= ref["iters"].max() + 4
        # the double-float PCG still converges with the FP32 preconditioner
        df = S.solve(geom.g, rtol=1e-8)
        assert df["hist"][-1] <= 1e-8


def test_fp32_group_matches_one_by_one():
    geoms = [WL.panels(s, n=8, n_coarse=2) for s in (3, 4, 5)]
    first = M.Solver(geoms[0])
    group = [first] + [M.Solver(g, share=first) for g in geoms[1:]]
    try:
        G = np.array([[0.3, -0.2, 0.9]])
        for S in group:
            S.assemble()
        one = []
        for S in group:
            S.factor(precision="fp32")
            one.append(S.solve_batch(G, rtol=1e-8, precision="mixed")["density"].copy())
        M.msbem_factor_group(group, precision="fp32")
        for S, x in zip(group, one):
            y = S.solve_batch(G, rtol=1e-8, precision="mixed")["density"]
            assert np.array_equal(x, y)
    finally:
        for S in reversed(group):
            S.close()


def test_fp32_option_checked():
    geom = WL.flat_config()
    with M.Solver(geom) as S:
        S.assemble()
        o = M.PrecondOpts(0, 1, 2)
        assert M.lib().msbem_factor(S.geom, M.ctypes.byref(o)) == -1
