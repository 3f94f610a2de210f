"""The field off the screen, U = DL Phi (Lemma lemrepDL, eq. formulaDL), on
the GPU (msbem_dl_potential) against the oracle's evaluation of the same
formula with the same rule, and Gauss's law on the cube's cells."""
import numpy as np
import pytest

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import build as B
from paper_2310_09204_gb300 import workloads as WL
from oracle import potential as P
from oracle import solver
from oracle.topology import Topology

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    B.build()
    M.lib()


def _targets(geom, m, seed, margin=0.15):
    """Random points of the bounding box inflated by 0.5, kept at least
    `margin` away from every vertex (so, for these meshes, away from Gamma)."""
    rng = np.random.default_rng(seed)
    lo, hi = geom.xyz.min(0) - 0.5, geom.xyz.max(0) + 0.5
    pts = []
    while len(pts) < m:
        x = rng.uniform(lo, hi)
        cen = geom.xyz[geom.tri].mean(axis=1)
        if np.min(np.linalg.norm(cen - x, axis=1)) > margin:
            pts.append(x)
    return np.array(pts)


@pytest.mark.parametrize("geom", [WL.panels(7, n=6), WL.book(8, 2, jitter=True, seed=3), WL.disk(8)],
                         ids=lambda g: g.name)
@pytest.mark.parametrize("refine", [0, 2])
def test_potential_against_oracle(geom, refine):
    top = Topology(geom.xyz, geom.tri)
    rng = np.random.default_rng(9)
    phi = rng.standard_normal(top.ndof)
    X = _targets(geom, 200, 10)
    Uo = P.dl_potential(top, phi, X, refine)
    with M.Solver(geom) as S:
        Ug, ms = S.potential(phi, X, refine)
        assert np.abs(Ug - Uo).max() <= 1e-12 * np.abs(Uo).max()
        assert ms > 0.0
        import torch
        Xd = torch.from_numpy(X).cuda()
        pd = torch.from_numpy(phi).cuda()
        Ud = torch.empty(X.shape[0], dtype=torch.float64, device="cuda")
        S.potential(pd, Xd, refine, out=Ud)
        torch.cuda.synchronize()
        assert np.array_equal(Ud.cpu().numpy(), Ug)


def test_gauss_law_on_gpu():
    g = WL.cube_midplanes(8, 2)
    centres = np.array([[0.25 + 0.5 * i, 0.25 + 0.5 * j, 0.25 + 0.5 * k]
                        for k in (0, 1) for j in (0, 1) for i in (0, 1)] + [[1.6, 0.4, 0.3]])
    with M.Solver(g) as S:
        Z, _ = S.cells()
        for c in range(8):
            U, _ = S.potential(Z[:, c], centres, refine=2)
            k = int(np.argmin(U[:8]))
            assert abs(U[k] + 1.0) <= 1e-9
            assert np.abs(np.delete(U, k)).max() <= 1e-9


def test_book_field_full_size():
    """The field of the full-size book's solution at 2,000 targets, sampled
    against the oracle at 64 of them."""
    geom = WL.book_config()
    X = _targets(geom, 2000, 11, margin=0.05)
    with M.Solver(geom) as S:
        S.assemble().factor()
        phi = S.solve(geom.g, rtol=1e-8)["density"]
        U, ms = S.potential(phi, X)
    top = Topology(geom.xyz, geom.tri)
    idx = np.arange(0, 2000, 32)
    Uo = P.dl_potential(top, phi, X[idx])
    assert np.abs(U[idx] - Uo).max() <= 1e-12 * np.abs(Uo).max()
