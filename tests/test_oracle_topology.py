"""Pins for the oracle's topology (CPU only).

The sectors (generalized vertices, Sec. 4.2) are checked against a purely
geometric count: the connected components of a small sphere around each
vertex minus the arcs cut out by the incident triangles, found by a
flood fill over quasi-uniform sample points.  Dof counts are checked against
their closed-form values for the grid workloads.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components
from scipy.spatial import cKDTree

from oracle.topology import MeshError, Topology
from paper_2310_09204_gb300 import workloads as WL

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "invariants.json")))


def _fibonacci_sphere(n):
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = math.pi * (1 + 5 ** 0.5) * i
    return np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1)


def _arc_distance(pts, a, b):
    """Angular distance from unit vectors pts to the great-circle arc a->b."""
    n = np.cross(a, b)
    n /= np.linalg.norm(n)
    off = np.arcsin(np.clip(np.abs(pts @ n), 0, 1))
    proj = pts - np.outer(pts @ n, n)
    nrm = np.linalg.norm(proj, axis=1)
    proj = proj / np.maximum(nrm, 1e-300)[:, None]
    # inside the arc's angular range?
    inside = (np.cross(a, proj) @ n >= 0) & (np.cross(proj, b) @ n >= 0)
    da = np.arccos(np.clip(pts @ a, -1, 1))
    db = np.arccos(np.clip(pts @ b, -1, 1))
    return np.where(inside, off, np.minimum(da, db))


def sphere_sectors(top: Topology, v: int, npts=20000):
    """Partition of the oriented triangles at vertex v by the components of
    (small sphere about x_v) minus (the triangles' arcs)."""
    pts = _fibonacci_sphere(npts)
    p = top.xyz[v]
    inc = [(T, a) for T in range(top.nt) for a in range(3) if top.tri[T, a] == v]
    blocked = np.zeros(npts, bool)
    delta = 0.05
    for T, a in inc:
        e1 = top.xyz[top.tri[T, (a + 1) % 3]] - p
        e2 = top.xyz[top.tri[T, (a + 2) % 3]] - p
        e1 /= np.linalg.norm(e1)
        e2 /= np.linalg.norm(e2)
        blocked |= _arc_distance(pts, e1, e2) < delta
    free = np.nonzero(~blocked)[0]
    tree = cKDTree(pts[free])
    pairs = tree.query_pairs(0.04, output_type="ndarray")
    G = sp.coo_matrix((np.ones(len(pairs)), (pairs[:, 0], pairs[:, 1])), shape=(len(free), len(free)))
    ncomp, lab = connected_components(G, directed=False)
    label_of = {}
    for T, a in inc:
        e1 = top.xyz[top.tri[T, (a + 1) % 3]] - p
        e2 = top.xyz[top.tri[T, (a + 2) % 3]] - p
        bis = e1 / np.linalg.norm(e1) + e2 / np.linalg.norm(e2)
        bis /= np.linalg.norm(bis)
        for s, sign in ((0, 1.0), (1, -1.0)):
            d = bis + sign * 0.35 * top.normal[T]
            d /= np.linalg.norm(d)
            _, k = tree.query(d)
            label_of[(T, s)] = int(lab[k])
    return label_of


def _same_partition(lab_a, lab_b):
    keys = sorted(lab_a)
    m_ab, m_ba = {}, {}
    for k in keys:
        x, y = lab_a[k], lab_b[k]
        if m_ab.setdefault(x, y) != y or m_ba.setdefault(y, x) != x:
            return False
    return True


@pytest.mark.parametrize("geom", [WL.book(4, 2, jitter=False), WL.disk(3, fin=True), WL.bowtie(4, 2),
                                  WL.unit_square(4, 2), WL.panels(7, n=2, angle_range=(60.0, 180.0)),
                                  WL.panels(5, n=2, angle_range=(60.0, 180.0))], ids=lambda g: g.name)
def test_sectors_match_sphere_flood_fill(geom):
    # (the probe directions of the geometric count need wedges of some width:
    # the panel screens here keep >= 60 degrees between squares on a hinge)
    top = Topology(geom.xyz, geom.tri)
    for v in range(top.nv):
        geo = sphere_sectors(top, v)
        alg = {(T, s): int(top.sector[T, s, a]) for (T, s) in geo
               for a in range(3) if top.tri[T, a] == v}
        assert len(set(geo.values())) == top.q[v], (v, top.q[v], len(set(geo.values())))
        assert _same_partition(geo, alg), v


def test_flat_screen_reduces_to_manifold_case():
    """Remark 'Case where Gamma is a manifold': two sectors at interior
    vertices, one on the boundary, one dof per interior vertex."""
    g = WL.unit_square(16, 2)
    top = Topology(g.xyz, g.tri)
    x = g.xyz
    boundary = (np.abs(x[:, 0]) < 1e-12) | (np.abs(x[:, 0] - 1) < 1e-12) | \
               (np.abs(x[:, 1]) < 1e-12) | (np.abs(x[:, 1] - 1) < 1e-12)
    assert np.all(top.q[boundary] == 1)
    assert np.all(top.q[~boundary] == 2)
    assert top.ndof == GOLDEN["flat_square_h1_16_ndof"]["value"]


def test_book_dof_count_and_junction_sectors():
    g = WL.book_config()
    top = Topology(g.xyz, g.tri)
    assert top.ndof == GOLDEN["book3_h1_64_ndof"]["value"]
    spine = (np.abs(g.xyz[:, 0]) < 1e-12) & (np.abs(g.xyz[:, 1]) < 1e-12)
    z = g.xyz[:, 2]
    inner_spine = spine & (z > 1e-12) & (z < 1 - 1e-12)
    assert np.all(top.q[inner_spine] == 3)
    assert int(inner_spine.sum()) == 63


def test_fin_junction_has_four_sectors():
    g = WL.disk(4, fin=True)
    top = Topology(g.xyz, g.tri)
    x = g.xyz
    line = (np.abs(x[:, 1]) < 1e-12) & (np.abs(x[:, 2]) < 1e-12) & (np.abs(x[:, 0]) < 1 - 1e-12)
    assert np.all(top.q[line] == 4)
    assert int(line.sum()) == 2 * 4 - 1


def test_dof_numbering_is_canonical():
    """Dofs run over vertices in id order, then sectors in the order of their
    smallest oriented-triangle key 2T + side."""
    g = WL.book(4, 2, jitter=False)
    top = Topology(g.xyz, g.tri)
    assert np.all(np.diff(top.dof_vertex) >= 0)
    for v in range(top.nv):
        keys = {}
        for T in range(top.nt):
            for a in range(3):
                if top.tri[T, a] == v:
                    for s in (0, 1):
                        j = int(top.sector[T, s, a])
                        keys[j] = min(keys.get(j, 10 ** 9), 2 * T + s)
        if keys:
            assert [keys[j] for j in sorted(keys)] == sorted(keys.values())


def test_rejects_point_contact_and_duplicates():
    # two triangles touching at a single vertex
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0.5], [0, -1, 0.5]], float)
    with pytest.raises(MeshError):
        Topology(xyz, np.array([[0, 1, 2], [0, 3, 4]]))
    with pytest.raises(MeshError):
        Topology(xyz, np.array([[0, 1, 2], [1, 2, 0]]))
    with pytest.raises(MeshError):
        Topology(np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0]], float), np.array([[0, 1, 2]]))


@pytest.mark.parametrize("seed", range(16))
def test_panels_dof_count(seed):
    """Squares hinged at arbitrary dihedral angles: every interior vertex of a
    square has 2 sectors (1 dof), a vertex inside a hinge shared by m squares
    has m sectors (m - 1 dofs), square corners have 1; so
    N = sum over squares (n-1)^2 + sum over hinges (m-1)(n-1)."""
    n = 4
    g = WL.panels(seed, n=n)
    top = Topology(g.xyz, g.tri)
    expected = g.meta["panels"] * (n - 1) ** 2 + sum((m - 1) * (n - 1) for m in g.meta["hinges"])
    assert top.ndof == expected
    assert int(np.max(top.q)) == max(g.meta["hinges"])
