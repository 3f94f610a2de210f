"""Seeded synthetic multiscreen geometries (inputs only).

This module builds triangle meshes, nested coarse meshes and patch partitions
for the workloads the solver is measured and tested on.  It holds none of the
method's arithmetic: no sectors, no quadrature, no matrices.  Both the CUDA
path (through the C ABI) and the CPU oracle consume its output, and nothing
else is shared between them.

Every generator returns a ``Geometry`` with

* ``xyz``  float64 [nv, 3]  fine-mesh vertices,
* ``tri``  int32   [nt, 3]  fine triangles (vertex ids),
* ``coarse_xyz`` / ``coarse_tri``: the nested coarse mesh (mesh size H),
* ``parent``  int32 [nt]: coarse triangle containing each fine triangle,
* ``patch``   int32 [nt]: non-overlapping patch (substructure) of each fine
  triangle, the face spaces of the two-level splitting (Sec. 5, eq. jumpSplit),
* ``g``       float64 [3]: the constant Neumann datum of the workload.

Geometries follow the shapes used in the paper's experiments (Sec. 2.2: the
bow-tie multiscreen of Experiment 3) and the synthetic workloads the project is
measured on (flat unit square, three-page book, disk with a perpendicular fin).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Geometry:
    name: str
    xyz: np.ndarray
    tri: np.ndarray
    coarse_xyz: np.ndarray
    coarse_tri: np.ndarray
    parent: np.ndarray
    patch: np.ndarray
    g: np.ndarray
    h: float
    H: float
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def nt(self) -> int:
        return int(self.tri.shape[0])


# --------------------------------------------------------------------------
# small mesh-building helpers (pure bookkeeping)
# --------------------------------------------------------------------------

class _MeshBuilder:
    """Collects triangles given by vertex coordinates and merges coincident
    vertices by rounded position, so that separately generated panels become
    one conforming mesh."""

    def __init__(self, decimals: int = 10):
        self.decimals = decimals
        self.scale = 10.0 ** decimals
        self.key_to_id: dict = {}
        self.pts: list = []
        self.tris: list = []

    def vid(self, p) -> int:
        # key: the coordinates rounded to `decimals` places, as integers
        # (rint(x * 10^decimals), ties to even)
        x, y, z = float(p[0]), float(p[1]), float(p[2])
        s = self.scale
        key = (round(x * s), round(y * s), round(z * s))
        i = self.key_to_id.get(key)
        if i is None:
            i = len(self.pts)
            self.key_to_id[key] = i
            self.pts.append((x, y, z))
        return i

    def add(self, a, b, c) -> int:
        self.tris.append((self.vid(a), self.vid(b), self.vid(c)))
        return len(self.tris) - 1

    def add_ids(self, a: int, b: int, c: int) -> int:
        self.tris.append((a, b, c))
        return len(self.tris) - 1

    def arrays(self):
        return (np.array(self.pts, dtype=np.float64).reshape(-1, 3),
                np.array(self.tris, dtype=np.int32).reshape(-1, 3))


def _grid_panel(mb: _MeshBuilder, origin, eu, ev, nu: int, nv: int, tags=None, tag_fn=None):
    """Uniform grid on the parallelogram origin + [0,1]eu + [0,1]ev with nu x nv
    cells, each split along the diagonal from (i, j) to (i+1, j+1)."""
    origin = np.asarray(origin, float)
    eu = np.asarray(eu, float)
    ev = np.asarray(ev, float)

    I, J = np.meshgrid(np.arange(nu + 1) / nu, np.arange(nv + 1) / nv, indexing="ij")
    pts = (origin[None, None, :] + I[:, :, None] * eu[None, None, :] + J[:, :, None] * ev[None, None, :]).tolist()
    ids: dict = {}

    def V(i, j):   # vertex id of grid point (i, j), in order of first use
        k = ids.get((i, j))
        if k is None:
            k = ids[(i, j)] = mb.vid(pts[i][j])
        return k

    for j in range(nv):
        for i in range(nu):
            v00 = V(i, j)
            v10 = V(i + 1, j)
            v11 = V(i + 1, j + 1)
            mb.add_ids(v00, v10, v11)
            v01 = V(i, j + 1)
            mb.add_ids(v00, v11, v01)
            if tags is not None:
                tags.append(tag_fn(i, j, 0))
                tags.append(tag_fn(i, j, 1))


def _subdivided_triangle(mb: _MeshBuilder, A, B, C, n: int):
    """Uniform subdivision of triangle ABC into n^2 similar triangles; keeps
    the orientation of ABC."""
    A, B, C = (np.asarray(x, float) for x in (A, B, C))

    def P(i, j):
        return A + (i / n) * (B - A) + (j / n) * (C - A)

    out = []
    for j in range(n):
        for i in range(n - j):
            out.append(mb.add(P(i, j), P(i + 1, j), P(i, j + 1)))
            if i + j + 1 < n:
                out.append(mb.add(P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)))
    return out


def _locate_parents(xyz, tri, cxyz, ctri) -> np.ndarray:
    """Coarse triangle containing each fine triangle (by its centroid)."""
    cen = xyz[tri].mean(axis=1)                      # [nt, 3]
    A = cxyz[ctri[:, 0]]
    B = cxyz[ctri[:, 1]]
    C = cxyz[ctri[:, 2]]
    e1 = B - A
    e2 = C - A
    nrm = np.cross(e1, e2)
    area2 = np.linalg.norm(nrm, axis=1)
    nhat = nrm / area2[:, None]
    parent = np.full(tri.shape[0], -1, dtype=np.int32)
    chunk = 4096
    for s in range(0, cen.shape[0], chunk):
        c = cen[s:s + chunk]                          # [m, 3]
        d = c[:, None, :] - A[None, :, :]             # [m, nc, 3]
        off = np.abs(np.einsum('mkj,kj->mk', d, nhat))
        # barycentric coordinates in each coarse triangle's plane
        d11 = np.einsum('kj,kj->k', e1, e1)
        d12 = np.einsum('kj,kj->k', e1, e2)
        d22 = np.einsum('kj,kj->k', e2, e2)
        p1 = np.einsum('mkj,kj->mk', d, e1)
        p2 = np.einsum('mkj,kj->mk', d, e2)
        den = d11 * d22 - d12 * d12
        l1 = (d22 * p1 - d12 * p2) / den
        l2 = (d11 * p2 - d12 * p1) / den
        l0 = 1.0 - l1 - l2
        ok = (off < 1e-9) & (l0 > -1e-9) & (l1 > -1e-9) & (l2 > -1e-9)
        cnt = ok.sum(axis=1)
        if np.any(cnt != 1):
            raise ValueError("fine mesh does not nest in the coarse mesh")
        parent[s:s + chunk] = np.argmax(ok, axis=1)
    return parent


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def unit_square(n: int = 16, n_coarse: int = 2, patch_mode: str = "square",
                g=(0.0, 0.0, 1.0)) -> Geometry:
    """Flat screen [0,1]^2 in the plane z = 0 with h = 1/n, H = 1/n_coarse.

    ``patch_mode``: 'square' -> one patch per coarse square (two coarse
    triangles); 'coarse_tri' -> one patch per coarse triangle (the face spaces
    of Sec. 5 taken literally)."""
    if n % n_coarse:
        raise ValueError("n must be a multiple of n_coarse")
    r = n // n_coarse
    mb = _MeshBuilder()
    _grid_panel(mb, (0, 0, 0), (1, 0, 0), (0, 1, 0), n, n)
    xyz, tri = mb.arrays()
    cb = _MeshBuilder()
    _grid_panel(cb, (0, 0, 0), (1, 0, 0), (0, 1, 0), n_coarse, n_coarse)
    cxyz, ctri = cb.arrays()
    parent = _locate_parents(xyz, tri, cxyz, ctri)
    if patch_mode == "coarse_tri":
        patch = parent.copy()
    elif patch_mode == "square":
        cen = xyz[tri].mean(axis=1)
        I = np.minimum((cen[:, 0] * n_coarse).astype(int), n_coarse - 1)
        J = np.minimum((cen[:, 1] * n_coarse).astype(int), n_coarse - 1)
        patch = (J * n_coarse + I).astype(np.int32)
    else:
        raise ValueError(patch_mode)
    return Geometry(f"unit_square_h1/{n}_H1/{n_coarse}", xyz, tri, cxyz, ctri, parent,
                    patch, np.asarray(g, float), 1.0 / n, 1.0 / n_coarse,
                    {"family": "square", "n": n, "n_coarse": n_coarse, "r": r})


def _jittered_cuts(n: int, n_coarse: int, rng, jitter: bool):
    r = n // n_coarse
    cuts = []
    for k in range(1, n_coarse):
        c = k * r
        if jitter:
            c += int(rng.integers(-1, 2))
        cuts.append(c)
    return cuts


def book(n: int = 64, n_coarse: int = 4, jitter: bool = True, seed: int = 0,
         pages: int = 3, g=(1.0, 0.5, 0.25)) -> Geometry:
    """'Three-page book': ``pages`` unit squares sharing the edge
    {x = 0, y = 0, z in [0,1]}, at angles 2*pi*k/pages about the z-axis.

    Each page carries an n x n grid (h = 1/n) and the nested coarse grid
    n_coarse x n_coarse (H = 1/n_coarse).  Patches: n_coarse x n_coarse per
    page, whose cut lines are shifted by a seeded random -1/0/+1 fine rows
    (independently for every cut line of every page) so patch sizes are uneven.
    """
    rng = np.random.default_rng(seed)
    mb = _MeshBuilder()
    tags = []
    cb = _MeshBuilder()
    for k in range(pages):
        th = 2.0 * math.pi * k / pages
        er = (math.cos(th), math.sin(th), 0.0)
        ez = (0.0, 0.0, 1.0)
        cr = _jittered_cuts(n, n_coarse, rng, jitter)
        cz = _jittered_cuts(n, n_coarse, rng, jitter)

        def tag(i, j, t, k=k, cr=cr, cz=cz):
            bi = sum(1 for c in cr if i >= c)
            bj = sum(1 for c in cz if j >= c)
            return (k * n_coarse + bj) * n_coarse + bi

        _grid_panel(mb, (0, 0, 0), er, ez, n, n, tags, tag)
        _grid_panel(cb, (0, 0, 0), er, ez, n_coarse, n_coarse)
    xyz, tri = mb.arrays()
    cxyz, ctri = cb.arrays()
    parent = _locate_parents(xyz, tri, cxyz, ctri)
    patch = np.array(tags, dtype=np.int32)
    return Geometry(f"book{pages}_h1/{n}_H1/{n_coarse}" + ("_jit" if jitter else ""), xyz, tri,
                    cxyz, ctri, parent, patch, np.asarray(g, float), 1.0 / n, 1.0 / n_coarse,
                    {"family": "book", "n": n, "n_coarse": n_coarse, "pages": pages,
                     "seed": seed, "jitter": jitter})


def _hex_disk(mb: _MeshBuilder, n: int, a: float):
    """Disk of radius a in z = 0: ring k (k = 1..n) holds 6k vertices at radius
    a*k/n and equal angles; rings are joined sector by sector as in a
    hexagonal grid, so the diameter on the x-axis is a union of mesh edges."""
    def P(k, m):
        if k == 0:
            return (0.0, 0.0, 0.0)
        m %= 6 * k
        th = 2.0 * math.pi * m / (6 * k)
        return (a * k / n * math.cos(th), a * k / n * math.sin(th), 0.0)

    ids = []
    for k in range(1, n + 1):
        for s in range(6):
            for t in range(k):
                o0 = P(k, s * k + t)
                o1 = P(k, s * k + t + 1)
                i0 = P(k - 1, s * (k - 1) + t)
                ids.append(mb.add(i0, o0, o1))
                if t < k - 1:
                    i1 = P(k - 1, s * (k - 1) + t + 1)
                    ids.append(mb.add(i0, o1, i1))
    return ids


def disk(n: int = 8, a: float = 1.0, fin: bool = False, fin_half_height: float | None = None,
         g=(0.0, 0.0, 1.0)) -> Geometry:
    """Flat disk of radius a (n rings, h ~ a/n) in z = 0, optionally crossed by
    a perpendicular rectangular fin {y = 0, |x| <= a, |z| <= b} along the
    x-axis diameter.  For g = (0, 0, g_n) the exact jump is
    (4/pi) g_n sqrt(a^2 - r^2) on the disk and 0 on the fin.

    The coarse mesh is the single-level mesh itself (no coarse space is needed
    for the closed-form tests); every triangle is its own patch parent."""
    mb = _MeshBuilder()
    _hex_disk(mb, n, a)
    if fin:
        b = a if fin_half_height is None else fin_half_height
        mz = max(1, int(round(b / (a / n))))
        _grid_panel(mb, (-a, 0.0, -b), (2 * a, 0.0, 0.0), (0.0, 0.0, 2 * b), 2 * n, 2 * mz)
    xyz, tri = mb.arrays()
    # enforce a consistent upward/forward orientation for readability
    P0, P1, P2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    nrm = np.cross(P1 - P0, P2 - P0)
    flip = (nrm[:, 2] < -1e-14) | ((np.abs(nrm[:, 2]) <= 1e-14) & (nrm[:, 1] < 0))
    tri[flip] = tri[flip][:, [0, 2, 1]]
    parent = np.arange(tri.shape[0], dtype=np.int32)
    return Geometry(("diskfin" if fin else "disk") + f"_n{n}", xyz, tri, xyz.copy(), tri.copy(),
                    parent, np.zeros(tri.shape[0], np.int32), np.asarray(g, float), a / n, a,
                    {"family": "disk", "n": n, "a": a, "fin": fin})


def bowtie(n: int = 8, n_coarse: int = 2, g=(1.0, 0.5, 0.25)) -> Geometry:
    """The bow-tie of Experiment 3 (Sec. 2.2): two unit equilateral triangles in
    perpendicular planes sharing a median.  Each is pre-split along that
    median so the junction is a mesh line; the four halves are subdivided
    uniformly (coarse level n_coarse, fine level n, nested).  Patches are the
    coarse triangles (the face spaces of Sec. 5)."""
    if n % n_coarse:
        raise ValueError("n must be a multiple of n_coarse")
    top = (0.0, 0.0, math.sqrt(3.0) / 2.0)
    mid = (0.0, 0.0, 0.0)
    halves = [((-0.5, 0.0, 0.0), mid, top), (mid, (0.5, 0.0, 0.0), top),
              ((0.0, -0.5, 0.0), mid, top), (mid, (0.0, 0.5, 0.0), top)]
    mb = _MeshBuilder()
    cb = _MeshBuilder()
    for (A, B, C) in halves:
        _subdivided_triangle(mb, A, B, C, n)
        _subdivided_triangle(cb, A, B, C, n_coarse)
    xyz, tri = mb.arrays()
    cxyz, ctri = cb.arrays()
    parent = _locate_parents(xyz, tri, cxyz, ctri)
    return Geometry(f"bowtie_n{n}_nc{n_coarse}", xyz, tri, cxyz, ctri, parent, parent.copy(),
                    np.asarray(g, float), 1.0 / n, 1.0 / n_coarse,
                    {"family": "bowtie", "n": n, "n_coarse": n_coarse})


def _square_points(origin, eu, ev, m: int = 13) -> np.ndarray:
    t = np.linspace(0.0, 1.0, m)
    U, V = np.meshgrid(t, t, indexing="ij")
    return (np.asarray(origin)[None, :] + U.reshape(-1, 1) * np.asarray(eu)[None, :]
            + V.reshape(-1, 1) * np.asarray(ev)[None, :])


def _min_dist(a: np.ndarray, b: np.ndarray) -> float:
    d = a[:, None, :] - b[None, :, :]
    return float(np.sqrt(np.min(np.einsum("ijk,ijk->ij", d, d))))


def panels(seed: int, n: int | None = None, n_panels: int | None = None, g=None,
           max_tries: int = 200, angle_range=(30.0, 180.0), n_coarse: int | None = None) -> Geometry:
    """Multiscreen of 2-6 unit squares joined at shared edges with seeded
    random dihedral angles (the 'batched + mixed precision' workload family).

    The first square is [0,1]^2 in z = 0; every further square hinges on a
    random edge of a square already placed, at a dihedral angle drawn from
    U[30, 180] degrees (180: coplanar continuation; ``angle_range`` changes
    the interval), folded to a random side.
    A draw is rejected when two squares that share no hinge come closer than h
    (points of each square kept 3h away from the points they share), or two
    squares on the same hinge make an angle below 30 degrees; so the screen has
    no closed cells and no point contacts.  h = 1/n with n drawn from
    {24, 32, 48} unless given, H chosen so (H/h - 1)^2 lies in [150, 600]
    (n = 24: H = 1; 32, 48: H = 1/2; ``n_coarse`` overrides).  Patches: the
    coarse squares of every panel.  g: uniform in [-1, 1]^3 unless given."""
    rng = np.random.default_rng(seed)
    if n is None:
        n = int(rng.choice([24, 32, 48]))
    if n_coarse is None:
        n_coarse = {24: 1, 32: 2, 48: 2}.get(n, max(1, n // 24))
    if n % n_coarse:
        raise ValueError("n must be a multiple of n_coarse")
    if n_panels is None:
        n_panels = int(rng.integers(2, 7))
    h = 1.0 / n
    sq = [(np.zeros(3), np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]))]
    hinge_dirs: dict = {}   # hinge (sorted end points) -> directions of the squares on it
    tries = 0
    while len(sq) < n_panels:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("panels: no admissible placement found")
        k = int(rng.integers(len(sq)))
        o, eu, ev = sq[k]
        corners = [o, o + eu, o + eu + ev, o + ev]
        e = int(rng.integers(4))
        a, b = corners[e], corners[(e + 1) % 4]
        w = o + 0.5 * (eu + ev) - 0.5 * (a + b)
        w /= np.linalg.norm(w)                  # in square k's plane, into it
        nrm = np.cross(eu, ev)
        nrm /= np.linalg.norm(nrm)
        th = math.radians(float(rng.uniform(*angle_range)))
        side = 1.0 if rng.random() < 0.5 else -1.0
        d = math.cos(th) * w + side * math.sin(th) * nrm
        d /= np.linalg.norm(d)
        new = (a.copy(), b - a, d)
        hkey = tuple(sorted((tuple(np.round(a, 9)), tuple(np.round(b, 9)))))
        dirs = hinge_dirs.get(hkey, [w])
        ok = all(math.degrees(math.acos(float(np.clip(np.dot(dj, d), -1.0, 1.0)))) >= angle_range[0]
                 for dj in dirs)
        if ok:
            pn = _square_points(*new)
            for j, (oj, euj, evj) in enumerate(sq):
                if j == k:
                    continue
                pj = _square_points(oj, euj, evj)
                # points both squares share (hinges, corners) and their neighbourhood
                shared = [p for p in pn if np.min(np.linalg.norm(pj - p, axis=1)) < 1e-9]
                A, Bp = pn, pj
                if shared:
                    S = np.array(shared)
                    A = pn[np.min(np.linalg.norm(pn[:, None, :] - S[None], axis=2), axis=1) > 3 * h]
                    Bp = pj[np.min(np.linalg.norm(pj[:, None, :] - S[None], axis=2), axis=1) > 3 * h]
                if A.size and Bp.size and _min_dist(A, Bp) < h:
                    ok = False
                    break
        if not ok:
            continue
        sq.append(new)
        hinge_dirs[hkey] = dirs + [d]
    mb = _MeshBuilder()
    cb = _MeshBuilder()
    tags = []
    for k, (o, eu, ev) in enumerate(sq):
        def tag(i, j, t, k=k):
            return (k * n_coarse + (j * n_coarse) // n) * n_coarse + (i * n_coarse) // n
        _grid_panel(mb, o, eu, ev, n, n, tags, tag)
        _grid_panel(cb, o, eu, ev, n_coarse, n_coarse)
    xyz, tri = mb.arrays()
    cxyz, ctri = cb.arrays()
    parent = _locate_parents(xyz, tri, cxyz, ctri)
    if g is None:
        g = rng.uniform(-1.0, 1.0, 3)
    return Geometry(f"panels{len(sq)}_s{seed}_h1/{n}", xyz, tri, cxyz, ctri, parent,
                    np.array(tags, dtype=np.int32), np.asarray(g, float), h, 1.0 / n_coarse,
                    {"family": "panels", "seed": seed, "n": n, "n_coarse": n_coarse, "panels": len(sq),
                     "hinges": sorted(len(v) for v in hinge_dirs.values())})


def panels_config(instances: int = 16) -> list:
    """Sixteen seeded panel multiscreens (instance seeds 0..15)."""
    return [panels(seed) for seed in range(instances)]


def cube_midplanes(n: int = 24, n_coarse: int = 6, g=None, seed: int = 0) -> Geometry:
    """Surface of the unit cube [0,1]^3 with its three interior mid-planes
    x = 1/2, y = 1/2, z = 1/2 (nine unit squares; non-manifold junction lines
    where a mid-plane meets a face or another mid-plane, and a junction point
    at the centre).  The screen encloses the eight octant cells, so the
    hypersingular operator has an eight-dimensional kernel (the cells'
    indicators).

    h = 1/n (n even), H = 1/n_coarse (n_coarse even, dividing n); every square
    carries the nested "/"-split grids; patches are the coarse grid squares of
    every face and mid-plane quarter.  g: uniform in [-1, 1]^3 (seeded) unless
    given."""
    if n % 2 or n_coarse % 2 or n % n_coarse:
        raise ValueError("n and n_coarse must be even, n a multiple of n_coarse")
    mb = _MeshBuilder()
    cb = _MeshBuilder()
    tags = []
    sheets = []
    e = np.eye(3)
    for ax in range(3):
        u, v = e[(ax + 1) % 3], e[(ax + 2) % 3]
        for off in (0.0, 0.5, 1.0):            # two faces and the mid-plane
            sheets.append((off * e[ax], u, v))
    for k, (o, u, v) in enumerate(sheets):
        def tag(i, j, t, k=k):
            return (k * n_coarse + (j * n_coarse) // n) * n_coarse + (i * n_coarse) // n
        _grid_panel(mb, o, u, v, n, n, tags, tag)
        _grid_panel(cb, o, u, v, n_coarse, n_coarse)
    xyz, tri = mb.arrays()
    cxyz, ctri = cb.arrays()
    parent = _locate_parents(xyz, tri, cxyz, ctri)
    if g is None:
        g = np.random.default_rng(seed).uniform(-1.0, 1.0, 3)
    return Geometry(f"cube_midplanes_h1/{n}_H1/{n_coarse}", xyz, tri, cxyz, ctri, parent,
                    np.array(tags, dtype=np.int32), np.asarray(g, float), 1.0 / n, 1.0 / n_coarse,
                    {"family": "cube", "n": n, "n_coarse": n_coarse, "cells": 8})


def cube_config() -> Geometry:
    """Cube with mid-planes at h = 1/96 (83,817 dofs, 165,888 triangles), the
    coarse squares of H = 1/6 as patches (324 of them), g seeded (seed 0)."""
    return cube_midplanes(96, 6, seed=0)


def flat_config() -> Geometry:
    """Plain FP64 flat-screen workload: unit square h = 1/16 (225 interior
    dofs), 2 x 2 substructuring (H = 1/2) plus the coarse space, g = (0,0,1)."""
    return unit_square(16, 2, "square", g=(0.0, 0.0, 1.0))


def book_config() -> Geometry:
    """Three-page book, h = 1/64 (12,033 dofs), 48 jittered patches (4 x 4 per
    page, seed 0), coarse H = 1/4, g = (1, 0.5, 0.25)."""
    return book(64, 4, jitter=True, seed=0, g=(1.0, 0.5, 0.25))


def rotate(geom: Geometry, R: np.ndarray, shift=(0.0, 0.0, 0.0)) -> Geometry:
    """Rigidly moved copy of a geometry (vertices and g rotated by R)."""
    R = np.asarray(R, float)
    s = np.asarray(shift, float)
    return dataclasses.replace(geom, name=geom.name + "_rot", xyz=geom.xyz @ R.T + s,
                               coarse_xyz=geom.coarse_xyz @ R.T + s, g=R @ geom.g)
