"""Precision modes of the solve (msbem_solve_opts.precision).

* "fp64", the plain FP64 comparator (FP64 copy of W, FP64 block inverses):
  the same parity bar as the default path -- iterations within +-1 and, at a
  fixed iteration count, densities within 1e-8 relative of the oracle.
* "mixed", FP32 inner PCG inside double-float iterative refinement: the
  refinement stops on the TRUE residual, so ||L - W Phi|| / ||L|| <= rtol
  must hold with the oracle's own W, and the W-energy error against the
  oracle's direct solution is then bounded by sqrt(kappa(W)) * rtol (the
  residual-to-error bound of an SPD system).
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import build as B
from paper_2310_09204_gb300 import workloads as WL
from oracle import solver

pytestmark = pytest.mark.gpu

SMALL = [WL.flat_config(), WL.book(8, 2, jitter=True, seed=3), WL.bowtie(6, 2)]
_PB = {}


@pytest.fixture(scope="module", autouse=True)
def _build():
    B.build()
    M.lib()


def problem(geom):
    if geom.name not in _PB:
        pb = solver.Problem(geom)
        pb.factor()
        _PB[geom.name] = pb
    return _PB[geom.name]


def _energy_rel(x, ref, W):
    e = x - ref
    return math.sqrt(max(e @ W @ e, 0.0)) / math.sqrt(ref @ W @ ref)


@pytest.mark.parametrize("geom", SMALL, ids=lambda g: g.name)
def test_plain_fp64_against_oracle(geom):
    pb = problem(geom)
    ref = pb.solve(rtol=1e-8)
    with M.Solver(geom) as S:
        S.assemble().factor()
        out = S.solve(geom.g, rtol=1e-8, precision="fp64")
        assert abs(out["iters"] - ref.iters) <= 1
        fx = S.solve(geom.g, rtol=0.0, maxit=ref.iters, fixed=True, precision="fp64")
        assert np.linalg.norm(fx["density"] - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
        assert _energy_rel(fx["density"], ref.x, pb.W) <= 1e-8


@pytest.mark.parametrize("geom", SMALL, ids=lambda g: g.name)
def test_mixed_reaches_true_residual(geom):
    pb = problem(geom)
    rng = np.random.default_rng(21)
    lam = sla.eigvalsh(pb.W)
    kappa = lam[-1] / lam[0]
    with M.Solver(geom) as S:
        S.assemble().factor()
        for g in (geom.g, rng.uniform(-1, 1, 3)):
            L = pb.rhs(g)
            xs = pb.direct(g)
            out = S.solve(g, rtol=1e-8, precision="mixed")
            x = out["density"]
            rel = np.linalg.norm(L - pb.W @ x) / np.linalg.norm(L)
            assert rel <= 1.05e-8, rel
            assert out["hist"][0] == 1.0 and out["hist"][-1] <= 1e-8
            assert len(out["hist"]) >= 2                       # at least one refinement step
            assert np.all(np.diff(out["hist"]) < 0)            # each step reduces the residual
            assert _energy_rel(x, xs, pb.W) <= 1.05 * math.sqrt(kappa) * 1e-8
            # stricter inner tolerance: fewer refinement steps, same answer
            tight = S.solve(g, rtol=1e-8, precision="mixed", inner_rtol=1e-6)
            assert len(tight["hist"]) <= len(out["hist"])
            assert _energy_rel(tight["density"], xs, pb.W) <= 1.05 * math.sqrt(kappa) * 1e-8


def test_mixed_batch_matches_single():
    geom = WL.book(8, 2, jitter=True, seed=3)
    pb = problem(geom)
    rng = np.random.default_rng(22)
    G = rng.uniform(-1, 1, (5, 3))
    G[3] = 0.0
    with M.Solver(geom) as S:
        S.assemble().factor()
        bt = S.solve_batch(G, rtol=1e-8, precision="mixed")
        for c in range(len(G)):
            if c == 3:
                assert bt["iters"][c] == 0 and np.all(bt["density"][c] == 0.0)
                continue
            L = pb.rhs(G[c])
            assert np.linalg.norm(L - pb.W @ bt["density"][c]) <= 1.05e-8 * np.linalg.norm(L)
            one = S.solve(G[c], rtol=1e-8, precision="mixed")
            assert np.linalg.norm(one["density"] - bt["density"][c]) <= 1e-7 * np.linalg.norm(one["density"])
        # a column alone and in the mix: bitwise the same
        alone = S.solve_batch(G[1:2], rtol=1e-8, precision="mixed")
        assert np.array_equal(alone["density"][0], bt["density"][1])
        # the plain comparator through the batch entry: one request at a time
        pl = S.solve_batch(G[:2], rtol=1e-8, precision="fp64")
        for c in range(2):
            one = S.solve(G[c], rtol=1e-8, precision="fp64")
            assert np.array_equal(pl["density"][c], one["density"])


def test_precision_option_errors():
    geom = WL.flat_config()
    with M.Solver(geom) as S:
        S.assemble().factor()
        with pytest.raises(M.MsbemError) as e:
            S.solve(geom.g, precision="mixed", fixed=True, maxit=3)
        assert e.value.status == -1
        with pytest.raises(M.MsbemError) as e:
            S.solve(geom.g, precision="mixed", inner_rtol=2.0)
        assert e.value.status == -1
        o = M.SolveOpts(1e-8, 100, 0, 1, 7, 0.0)
        out = np.empty(S.n)
        st = M.lib().msbem_solve(S.geom, M._ptr(np.asarray(geom.g, float)), M.ctypes.byref(o), M._ptr(out),
                                 None, None, 0, None)
        assert st == -1
        # the plain comparator follows a re-assembly (its FP64 copy is rebuilt)
        a = S.solve(geom.g, precision="fp64")["density"]
        S.assemble(ss_order=3).factor()
        b = S.solve(geom.g, precision="fp64")["density"]
        c = S.solve(geom.g)["density"]
        assert np.linalg.norm(b - c) <= 1e-8 * np.linalg.norm(c)
        assert not np.array_equal(a, b)


def test_book_config_full_size_mixed():
    geom = WL.book_config()
    with M.Solver(geom) as S:
        S.assemble().factor()
        ref = S.solve(geom.g, rtol=1e-10)
        mx = S.solve(geom.g, rtol=1e-8, precision="mixed")
        assert mx["hist"][-1] <= 1e-8
        assert np.linalg.norm(mx["density"] - ref["density"]) <= 1e-6 * np.linalg.norm(ref["density"])
        pl = S.solve(geom.g, rtol=1e-8, precision="fp64")
        df = S.solve(geom.g, rtol=1e-8)
        assert abs(pl["iters"] - df["iters"]) <= 1
        assert np.linalg.norm(pl["density"] - df["density"]) <= 1e-7 * np.linalg.norm(df["density"])


@pytest.mark.parametrize("geom", SMALL[:2], ids=lambda g: g.name)
def test_apply_matches_oracle_W(geom):
    """msbem_apply: Y = W X in the three product precisions against the
    oracle's W; a vector's product does not depend on the others beside it."""
    pb = problem(geom)
    rng = np.random.default_rng(23)
    X = rng.standard_normal((16, pb.ndof))
    Yo = X @ pb.W                                   # W is symmetric
    scale = np.abs(pb.W).max() * np.abs(X).sum(axis=1).max()
    with M.Solver(geom) as S:
        S.assemble()
        for prec, tol in (("df", 1e-12), ("fp64", 1e-12), ("fp32", 1e-6)):
            Y, ms = S.apply(X, precision=prec)
            assert np.abs(Y - Yo).max() <= tol * scale, (prec, np.abs(Y - Yo).max() / scale)
            assert ms > 0.0
        Y16, _ = S.apply(X)
        for c in (0, 5, 15):
            Y1, _ = S.apply(X[c:c + 1])
            assert np.array_equal(Y1[0], Y16[c])
        import torch
        Xd = torch.from_numpy(X[:3].copy()).cuda()
        Yd = torch.empty_like(Xd)
        S.apply(Xd, out=Yd)
        torch.cuda.synchronize()
        assert np.array_equal(Yd.cpu().numpy(), Y16[:3])
        with pytest.raises(M.MsbemError) as e:
            S.apply(np.zeros((17, pb.ndof)))
        assert e.value.status == -1
