"""Pins for the oracle's double-layer potential (CPU only).

* Gauss's law, an identity: the jump of a cell's indicator is 1 across the
  cell's boundary, so its double-layer potential is -1 inside that cell
  (orientation n . (y - x) of formulaDL) and 0 in every other cell and
  outside;
* the flat disk (g = (0, 0, 1)): the potential of the computed jump on the
  axis converges at first order in h to the potential of the exact jump
  (4/pi) sqrt(a^2 - r^2), an integral that reduces to one dimension on the
  axis (scipy quad);
* invariance under rigid motions and linearity in the density.
"""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle import potential as P
from oracle import solver
from oracle.topology import Topology
from paper_2310_09204_gb300 import workloads as WL


@pytest.mark.parametrize("refine,tol", [(0, 3e-6), (2, 1e-9)])
def test_gauss_law_on_cells(refine, tol):
    g = WL.cube_midplanes(8, 2)
    top = Topology(g.xyz, g.tri)
    Z = top.cells()
    centres = np.array([[0.25 + 0.5 * i, 0.25 + 0.5 * j, 0.25 + 0.5 * k]
                        for k in (0, 1) for j in (0, 1) for i in (0, 1)])
    outside = np.array([[1.6, 0.4, 0.3], [-0.7, 2.0, 0.5], [0.5, 0.5, 3.0]])
    seen = set()
    for c in range(8):
        U = P.dl_potential(top, Z[:, c], np.vstack([centres, outside]), refine)
        k = int(np.argmin(U[:8]))
        seen.add(k)
        assert abs(U[k] + 1.0) <= tol
        assert np.abs(np.delete(U, k)).max() <= tol
    assert seen == set(range(8))


def _disk_axis_exact(z, a=1.0, gn=1.0):
    mu = lambda r: (4.0 / np.pi) * gn * np.sqrt(max(a * a - r * r, 0.0))
    val = quad(lambda r: mu(r) * r / (r * r + z * z) ** 1.5, 0.0, a, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    return -(z / 2.0) * val


def test_disk_axis_converges():
    zs = np.array([0.3, 0.6, 1.0, 2.0])
    ex = np.array([_disk_axis_exact(z) for z in zs])
    errs = []
    for n in (4, 8, 16):
        g = WL.disk(n)
        pb = solver.Problem(g, with_coarse=False)
        x = pb.direct(g.g)
        U = P.dl_potential(pb.top, x, np.c_[np.zeros(4), np.zeros(4), zs], refine=1)
        errs.append(np.max(np.abs(U - ex) / np.abs(ex)))
    assert errs[-1] < 0.025
    assert 1.7 < errs[0] / errs[1] < 2.4 and 1.7 < errs[1] / errs[2] < 2.4


def test_rigid_motion_and_linearity():
    g = WL.panels(7, n=4)
    top = Topology(g.xyz, g.tri)
    rng = np.random.default_rng(8)
    phi = rng.standard_normal(top.ndof)
    psi = rng.standard_normal(top.ndof)
    X = rng.uniform(-1.0, 2.0, (20, 3))
    U = P.dl_potential(top, phi, X)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    shift = np.array([0.3, -1.2, 2.0])
    top_r = Topology(g.xyz @ R.T + shift, g.tri)
    U_r = P.dl_potential(top_r, phi, X @ R.T + shift)
    assert np.abs(U_r - U).max() <= 1e-12 * np.abs(U).max()
    U2 = P.dl_potential(top, 2.0 * phi - 3.0 * psi, X)
    assert np.abs(U2 - (2.0 * U - 3.0 * P.dl_potential(top, psi, X))).max() <= 1e-12 * np.abs(U2).max()
