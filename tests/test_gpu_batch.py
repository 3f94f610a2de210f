"""Batched solves (msbem_solve_batch): k Neumann data on one geometry, the
columns sharing each pass over W.  Every column runs the PCG recursion of
Sec. 2.1 on its own, so

* against the oracle: iteration counts within +-1 and, at a common fixed
  iteration count, densities within 1e-8 relative (l2 and W-energy);
* against itself: a column's result does not depend on the other columns of
  its batch, its position or the batch size -- bit for bit, since every
  per-column sum runs in the same order whatever the batch holds;
* against msbem_solve (another summation order of W p): iterations within +-1,
  densities within 1e-8 at a fixed count.
"""
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


def _rel(a, b, W=None):
    if W is None:
        return np.linalg.norm(a - b) / np.linalg.norm(b)
    e = a - b
    return math.sqrt(max(e @ W @ e, 0.0)) / math.sqrt(b @ W @ b)


def _data(geom, k, seed):
    rng = np.random.default_rng(seed)
    G = rng.uniform(-1.0, 1.0, (k, 3))
    G[0] = geom.g
    return G


@pytest.mark.parametrize("geom", [WL.flat_config(), WL.book(8, 2, jitter=True, seed=3), WL.bowtie(6, 2)],
                         ids=lambda g: g.name)
def test_batch_against_oracle(geom):
    pb = solver.Problem(geom)
    pb.factor()
    G = _data(geom, 5, 11)
    G[2] = 0.0                                            # no data: zero density, no iteration
    with M.Solver(geom) as S:
        S.assemble().factor()
        out = S.solve_batch(G, rtol=1e-8)
        for c in range(len(G)):
            if c == 2:
                assert out["iters"][c] == 0 and np.all(out["density"][c] == 0.0)
                continue
            ref = pb.solve(G[c], rtol=1e-8)
            assert abs(int(out["iters"][c]) - ref.iters) <= 1
            assert out["relres"][c] <= 1e-8
        K = pb.solve(G[0], rtol=1e-8).iters
        fx = S.solve_batch(G, rtol=0.0, maxit=K, fixed=True)
        for c in range(len(G)):
            if c == 2:
                continue
            ref = pb.solve(G[c], rtol=0.0, maxit=K, fixed=True)
            assert fx["iters"][c] == K
            assert _rel(fx["density"][c], ref.x) <= 1e-8
            assert _rel(fx["density"][c], ref.x, pb.W) <= 1e-8
            if K >= 3:
                assert abs(fx["kappa"][c] - ref.kappa) <= 1e-6 * ref.kappa


def test_column_independent_of_batch():
    geom = WL.book(8, 2, jitter=True, seed=3)
    G = _data(geom, 19, 12)                               # groups of 16 + 3
    with M.Solver(geom) as S:
        S.assemble().factor()
        full = S.solve_batch(G, rtol=1e-9)
        for c in (0, 7, 15, 16, 18):
            alone = S.solve_batch(G[c:c + 1], rtol=1e-9)
            assert alone["iters"][0] == full["iters"][c]
            assert np.array_equal(alone["density"][0], full["density"][c])
            assert alone["relres"][0] == full["relres"][c]
        # reversed order: the same columns, other positions
        rev = S.solve_batch(G[:16][::-1], rtol=1e-9)
        assert np.array_equal(rev["density"][::-1], full["density"][:16])


def test_batch_against_single_solves():
    geom = WL.book(8, 2, jitter=True, seed=3)
    G = _data(geom, 6, 13)
    with M.Solver(geom) as S:
        S.assemble().factor()
        bt = S.solve_batch(G, rtol=1e-8)
        for c in range(len(G)):
            one = S.solve(G[c], rtol=1e-8)
            assert abs(int(bt["iters"][c]) - one["iters"]) <= 1
        K = int(bt["iters"][0])
        fx = S.solve_batch(G, rtol=0.0, maxit=K, fixed=True)
        for c in range(len(G)):
            one = S.solve(G[c], rtol=0.0, maxit=K, fixed=True)
            assert _rel(fx["density"][c], one["density"]) <= 1e-8
        # unpreconditioned CG columns too
        pl = S.solve_batch(G[:2], precondition=False, rtol=1e-8)
        for c in range(2):
            one = S.solve(G[c], precondition=False, rtol=1e-8)
            assert abs(int(pl["iters"][c]) - one["iters"]) <= 1
            assert _rel(pl["density"][c], one["density"]) <= 1e-7


def test_batch_status_and_device_output():
    import torch
    geom = WL.flat_config()
    G = _data(geom, 3, 14)
    with M.Solver(geom) as S:
        S.assemble()
        with pytest.raises(M.MsbemError) as e:
            S.solve_batch(G)                               # factor missing
        assert e.value.status == -9
        S.factor()
        with pytest.raises(M.MsbemError) as e:
            S.solve_batch(np.zeros((0, 3)))
        assert e.value.status == -1
        out = S.solve_batch(G, maxit=1, raise_on_status=False)
        assert out["status"] == -5 and np.all(out["iters"] == 1)
        host = S.solve_batch(G)
        dev = torch.empty((3, S.n), dtype=torch.float64, device="cuda")
        S.solve_batch(G, out=dev)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), host["density"])


def test_book_config_full_size_batch():
    """Sixteen data on the full-size book (N = 12,033) in one batch, sampled
    columns against msbem_solve (itself held to the oracle at this size)."""
    geom = WL.book_config()
    G = _data(geom, 16, 15)
    with M.Solver(geom) as S:
        S.assemble().factor()
        bt = S.solve_batch(G, rtol=1e-8)
        assert np.all(bt["relres"] <= 1e-8)
        for c in (0, 9):
            one = S.solve(G[c], rtol=1e-8)
            assert abs(int(bt["iters"][c]) - one["iters"]) <= 1
            assert _rel(bt["density"][c], one["density"]) <= 1e-7
