"""Closed-form pins for the whole oracle pipeline (CPU only).

Flat disk of radius a in z = 0 with g = (0, 0, g_n): the exterior Neumann
problem (eq. PDE_intro) is solved by the potential of a disk moving
broadside; its jump is [U] = (4/pi) g_n sqrt(a^2 - r^2) and the energy
a(phi, phi) = l_g(phi) = (8/3) a^3 g_n^2 (energy identity, Lemma idDLDL).
Since psi = phi_{i,1} - phi_{i,2} has jump 2 phi_i, the coefficients tend to
(2/pi) g_n sqrt(a^2 - r^2).  The Galerkin energy approaches the exact one from
below (Cea / Galerkin orthogonality, Sec. 4.1) at rate O(h).

Disk plus a perpendicular fin along a diameter (a non-manifold multiscreen
with four sectors on the junction): by reflection symmetry the same field
solves it, so the jump on the fin is zero and the disk's jump is unchanged;
the discrete problem inherits the symmetry exactly.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import solver
from paper_2310_09204_gb300 import workloads as WL

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "invariants.json")))
E_EXACT = GOLDEN["disk_energy_over_a3_gn2"]["value"]


def _solve(geom):
    pb = solver.Problem(geom, with_coarse=False)
    x = pb.direct()
    return pb, x, float(pb.rhs() @ x)


@pytest.fixture(scope="module")
def disks():
    return {n: _solve(WL.disk(n)) for n in (4, 8, 12)}


def test_disk_energy_converges_from_below(disks):
    E = [disks[n][2] for n in (4, 8, 12)]
    assert E[0] < E[1] < E[2] < E_EXACT
    err = [E_EXACT - e for e in E]
    assert 1.6 < err[0] / err[1] < 2.6          # O(h)
    # Richardson extrapolation for an O(h) error lands on the closed form
    extrap = (12 * E[2] - 8 * E[1]) / 4
    assert abs(extrap - E_EXACT) < 5e-3 * E_EXACT


def test_disk_scaling_with_radius_and_data():
    a, gn = 0.5, -2.0
    pb, x, E = _solve(WL.disk(6, a=a, g=(0.0, 0.0, gn)))
    pb1, x1, E1 = _solve(WL.disk(6))
    assert abs(E - E1 * a ** 3 * gn ** 2) < 1e-12 * abs(E)


def test_disk_density_profile(disks):
    errs = []
    for n in (4, 8, 12):
        pb, x, _ = disks[n]
        r = np.linalg.norm(pb.top.xyz[pb.top.dof_vertex][:, :2], axis=1)
        ref = (2.0 / math.pi) * np.sqrt(1.0 - r ** 2)
        assert np.all(x > 0)
        errs.append(np.linalg.norm(x - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.02


def test_fin_leaves_the_disk_solution_unchanged():
    for n in (4, 6):
        pb, x, E = _solve(WL.disk(n))
        pf, xf, Ef = _solve(WL.disk(n, fin=True))
        assert abs(Ef - E) <= 1e-12 * E
        pos = pf.top.xyz[pf.top.dof_vertex]
        fin_only = (np.abs(pos[:, 1]) < 1e-12) & (np.abs(pos[:, 2]) > 1e-12)
        assert np.abs(xf[fin_only]).max() <= 1e-9 * np.abs(xf).max()
