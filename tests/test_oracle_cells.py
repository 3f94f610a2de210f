"""Pins for screens that enclose cells (CPU only): the cube with its three
mid-planes encloses the eight octant cells, so W has the cells' indicators
in its kernel and the solve uses W + rho Z Z^T (the reading of the paper's
connectedness assumption).

* the regions found from the sectors are checked against a purely geometric
  classification: the octant of a point just off every triangle side;
* the surface curl of every cell indicator vanishes on every triangle, so
  S_k Z = 0 and W Z = 0 to rounding -- an identity of the discrete space, not
  of the quadrature;
* W has exactly as many rounding-level eigenvalues as there are cells;
* Z^T L = 0 for constant data, and the augmented PCG returns the solution
  of W Phi = L with Z^T Phi = 0.
"""
import numpy as np
import pytest

from oracle import solver
from oracle.topology import Topology
from paper_2310_09204_gb300 import workloads as WL


def _geometric_Z(top: Topology, cube_side: float = 1.0):
    """Z from geometry alone: a side (T, s) lies in the octant cell of the
    point centroid + 1e-6 n_(T,s) when that point is inside the cube."""
    cen = top.xyz[top.tri].mean(axis=1)
    cell_of = {}
    for T in range(top.nt):
        for s, sg in ((0, 1.0), (1, -1.0)):
            p = cen[T] + 1e-6 * sg * top.normal[T]
            inside = np.all(p > 0) and np.all(p < cube_side)
            c = int((p[0] > 0.5) + 2 * (p[1] > 0.5) + 4 * (p[2] > 0.5)) if inside else -1
            for a in range(3):
                key = (int(top.tri[T, a]), int(top.sector[T, s, a]))
                assert cell_of.setdefault(key, c) == c      # a sector lies in one region
    Z = np.zeros((top.ndof, 8))
    for v in range(top.nv):
        q = int(top.q[v])
        if q < 2:
            continue
        cnt = np.zeros(8)
        for j in range(q):
            c = cell_of[(v, j)]
            if c >= 0:
                cnt[c] += 1
        for j in range(q - 1):
            row = int(top.first_dof[v]) + j
            Z[row] = -cnt / q
            c = cell_of[(v, j)]
            if c >= 0:
                Z[row, c] += 1.0
    return Z


@pytest.mark.parametrize("n", [2, 4, 6])
def test_cells_match_geometry(n):
    g = WL.cube_midplanes(n, 2)
    top = Topology(g.xyz, g.tri)
    Z = top.cells()
    assert Z.shape[1] == 8
    Zg = _geometric_Z(top)
    # same columns up to order
    for c in range(8):
        d = [np.abs(Z[:, c] - Zg[:, k]).max() for k in range(8)]
        assert min(d) == 0.0


@pytest.mark.parametrize("geom", [WL.unit_square(4, 2), WL.book(4, 2), WL.bowtie(4, 2), WL.disk(3, fin=True),
                                  WL.panels(7, n=4)], ids=lambda g: g.name)
def test_open_screens_have_no_cells(geom):
    assert Topology(geom.xyz, geom.tri).cells().shape[1] == 0


def test_cell_indicators_are_in_the_kernel():
    g = WL.cube_midplanes(4, 2)
    pb = solver.Problem(g)
    Z = pb.Z
    for Sk in pb.top.S_matrices():
        assert np.abs(Sk @ Z).max() <= 1e-13
    W0 = pb.W0
    assert np.linalg.norm(W0 @ Z) <= 1e-14 * np.linalg.norm(W0) * np.linalg.norm(Z)
    ev = np.linalg.eigvalsh(W0)
    assert np.sum(np.abs(ev) <= 1e-12 * ev[-1]) == 8
    assert np.linalg.eigvalsh(pb.W)[0] > 1e-3 * ev[-1]          # augmented: SPD
    assert pb.rho == pytest.approx(np.mean(np.diag(W0)))


def test_augmented_solve():
    g = WL.cube_midplanes(4, 2)
    pb = solver.Problem(g)
    pb.factor()
    rng = np.random.default_rng(4)
    for _ in range(3):
        gv = rng.uniform(-1, 1, 3)
        L = pb.rhs(gv)
        assert np.abs(pb.Z.T @ L).max() <= 1e-14 * np.linalg.norm(L)
        r = pb.solve(gv, rtol=1e-10)
        assert np.abs(pb.Z.T @ r.x).max() <= 1e-8 * np.linalg.norm(r.x)
        assert np.linalg.norm(L - pb.W0 @ r.x) <= 1e-9 * np.linalg.norm(L)


def test_projector_augmentation():
    """W + rho Q Q^T with Q an orthonormal basis of span Z: Q^T Q = I, the
    kernel directions get the eigenvalue rho exactly (W Q = 0), and the
    preconditioned condition number stays small and bounded in h (the
    additive Schwarz bound of Thm. main with H fixed)."""
    kap = []
    for n in (4, 8):
        g = WL.cube_midplanes(n, 2)
        pb = solver.Problem(g)
        Q, Z = pb.Q, pb.Z
        assert np.abs(Q.T @ Q - np.eye(8)).max() <= 1e-13
        # span Q = span Z
        assert np.linalg.norm(Z - Q @ (Q.T @ Z)) <= 1e-12 * np.linalg.norm(Z)
        assert np.linalg.norm(pb.W @ Q - pb.rho * Q) <= 1e-13 * np.linalg.norm(pb.W) * 8
        pb.factor()
        r = pb.solve(g.g, rtol=1e-10)
        kap.append(r.kappa)
    assert max(kap) < 6.0
