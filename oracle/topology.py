"""Multiscreen topology from the surface mesh alone (test infrastructure only).

Follows Sec. 4.2-4.3 of the paper:

* every triangle T of the mesh has two sides, the oriented triangles
  (T,+) and (T,-) of the inflated mesh (Def. Mstar); (T,+) is the side the
  normal n_T = (x1-x0) x (x2-x0) points into, so n_(T,+) = n_T, n_(T,-) = -n_T;
* the sectors (connected components Delta_{i,j} of the star graph
  G(x_i), Sec. 4.2) of a vertex x_i are found without a volume mesh: around
  every edge the incident triangles are ordered by angle, and the two faces
  bounding each wedge between angular neighbours belong to the same sector
  at both ends of the edge; an edge with one triangle joins (T,+) and (T,-)
  (the surface sets alpha_{k,l} of eq. defAlphaij);
* q_i = number of sectors of x_i; the dofs are the pairs (i,j) with q_i > 1
  and j < q_i (eq. defCurlyHtildeGamma), with psi_{i,j} = phi_{i,j} -
  phi_{i,q_i} (eq. defYij).  Sectors are numbered by the smallest key
  2T + (0 for +, 1 for -) of their oriented triangles, so the last one is q_i;
* on the oriented triangle t = (T, sigma) the trace of psi_{(a,j)} is
  c_t lambda_a with c_t = [sector_t(a) = j] - [sector_t(a) = q_a]; its surface
  curl is c_t n_t x grad lambda_a.  Summing the two sides, the curl of the
  jump on T is s_{T,nu} = (c_+ - c_-) (x_{a+1} - x_{a+2}) / (2|T|)
  (eq. eval_a_phiij, defvarphikij).

Point contacts (footnote of Sec. 4.3) are rejected.
"""
from __future__ import annotations

import math

import numpy as np


class MeshError(ValueError):
    pass


class _DSU:
    def __init__(self, n):
        self.p = list(range(n))

    def find(self, a):
        p = self.p
        while p[a] != a:
            p[a] = p[p[a]]
            a = p[a]
        return a

    def union(self, a, b):
        ra, rb = self.find(a), self.find(b)
        if ra != rb:
            if ra < rb:
                self.p[rb] = ra
            else:
                self.p[ra] = rb


class Topology:
    """Sectors, dofs and curl lists of a triangle mesh."""

    def __init__(self, xyz, tri):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.tri = np.asarray(tri, dtype=np.int64)
        nv, nt = self.xyz.shape[0], self.tri.shape[0]
        self.nv, self.nt = nv, nt
        P0, P1, P2 = (self.xyz[self.tri[:, k]] for k in range(3))
        cr = np.cross(P1 - P0, P2 - P0)
        self.area = 0.5 * np.linalg.norm(cr, axis=1)
        if np.any(self.area <= 1e-14 * (np.linalg.norm(P1 - P0, axis=1) ** 2 + 1e-300)):
            raise MeshError("degenerate triangle")
        self.normal = cr / (2.0 * self.area[:, None])
        self._check_duplicates()
        self._sectors()
        self._dofs()

    # ------------------------------------------------------------------
    def _check_duplicates(self):
        key = np.sort(self.tri, axis=1)
        u = np.unique(key, axis=0)
        if u.shape[0] != key.shape[0]:
            raise MeshError("duplicate triangle")
        if np.any(key[:, 0] == key[:, 1]) or np.any(key[:, 1] == key[:, 2]):
            raise MeshError("repeated vertex in a triangle")

    def _local(self, T, v):
        t = self.tri[T]
        for a in range(3):
            if t[a] == v:
                return a
        raise KeyError

    def _sectors(self):
        tri, xyz = self.tri, self.xyz
        nt = self.nt
        # corner node of oriented triangle (T, s) at its local vertex a
        node = lambda T, s, a: (2 * T + s) * 3 + a  # noqa: E731
        dsu = _DSU(6 * nt)
        # triangle adjacency around each vertex (point-contact check)
        fan = _DSU(3 * nt)
        edges = {}
        for T in range(nt):
            for a in range(3):
                i, k = int(tri[T, a]), int(tri[T, (a + 1) % 3])
                edges.setdefault((min(i, k), max(i, k)), []).append(T)
        self.edges = edges
        for (i, k), Ts in edges.items():
            if len(Ts) == 1:
                T = Ts[0]
                for v in (i, k):
                    a = self._local(T, v)
                    dsu.union(node(T, 0, a), node(T, 1, a))
                continue
            u = xyz[k] - xyz[i]
            u = u / np.linalg.norm(u)
            info = []
            for T in Ts:
                r = [int(x) for x in tri[T] if x != i and x != k][0]
                d = xyz[r] - xyz[i]
                d = d - np.dot(d, u) * u
                d = d / np.linalg.norm(d)
                info.append((T, d))
            e1 = info[0][1]
            e2 = np.cross(u, e1)
            ang = []
            for T, d in info:
                th = math.atan2(float(np.dot(d, e2)), float(np.dot(d, e1)))
                if th < 0:
                    th += 2 * math.pi
                # side of T facing increasing angle: + if n_T . (u x d) > 0
                plus_faces_up = float(np.dot(self.normal[T], np.cross(u, d))) > 0
                ang.append((th, T, 0 if plus_faces_up else 1))
            ang.sort()
            for m in range(len(ang)):
                th_a = ang[m][0]
                th_b = ang[(m + 1) % len(ang)][0] + (2 * math.pi if m + 1 == len(ang) else 0.0)
                if th_b - th_a < 1e-10:
                    raise MeshError("overlapping triangles at an edge")
            for m in range(len(ang)):
                _, Ta, sa_up = ang[m]
                _, Tb, sb_up = ang[(m + 1) % len(ang)]
                sb_down = 1 - sb_up
                for v in (i, k):
                    dsu.union(node(Ta, sa_up, self._local(Ta, v)), node(Tb, sb_down, self._local(Tb, v)))
            for v in (i, k):
                for T in Ts[1:]:
                    fan.union(3 * Ts[0] + self._local(Ts[0], v), 3 * T + self._local(T, v))
        # gather corners per vertex
        corners = [[] for _ in range(self.nv)]
        for T in range(nt):
            for a in range(3):
                corners[int(tri[T, a])].append((T, a))
        q = np.zeros(self.nv, dtype=np.int64)
        sector = np.full((nt, 2, 3), -1, dtype=np.int64)
        for v in range(self.nv):
            cs = corners[v]
            if not cs:
                continue
            roots_fan = {fan.find(3 * T + a) for (T, a) in cs}
            if len(roots_fan) > 1:
                raise MeshError(f"point contact at vertex {v}")
            comp_min = {}
            for (T, a) in cs:
                for s in (0, 1):
                    r = dsu.find(node(T, s, a))
                    key = 2 * T + s
                    if r not in comp_min or key < comp_min[r]:
                        comp_min[r] = key
            order = sorted(comp_min, key=lambda r: comp_min[r])
            idx = {r: j for j, r in enumerate(order)}
            q[v] = len(order)
            for (T, a) in cs:
                for s in (0, 1):
                    sector[T, s, a] = idx[dsu.find(node(T, s, a))]
        self.q = q
        self.sector = sector  # sector[T, s, a]: sector index at vertex tri[T, a]

    def _dofs(self):
        q = self.q
        first = np.zeros(self.nv + 1, dtype=np.int64)
        first[1:] = np.cumsum(np.maximum(q - 1, 0))
        self.first_dof = first
        self.ndof = int(first[-1])
        self.dof_vertex = np.repeat(np.arange(self.nv), np.maximum(q - 1, 0))
        self.dof_sector = np.concatenate([np.arange(max(int(x) - 1, 0)) for x in q]) \
            if self.ndof else np.zeros(0, np.int64)
        # curl lists: per dof, entries (T, a, coef)
        entries = []
        for T in range(self.nt):
            for a in range(3):
                v = int(self.tri[T, a])
                qv = int(q[v])
                if qv < 2:
                    continue
                sp, sm = int(self.sector[T, 0, a]), int(self.sector[T, 1, a])
                for j in range(qv - 1):
                    cp = (1 if sp == j else 0) - (1 if sp == qv - 1 else 0)
                    cm = (1 if sm == j else 0) - (1 if sm == qv - 1 else 0)
                    coef = cp - cm
                    if coef != 0:
                        entries.append((int(first[v]) + j, T, a, coef))
        entries.sort()
        self.s_dof = np.array([e[0] for e in entries], dtype=np.int64)
        self.s_tri = np.array([e[1] for e in entries], dtype=np.int64)
        self.s_loc = np.array([e[2] for e in entries], dtype=np.int64)
        self.s_coef = np.array([e[3] for e in entries], dtype=np.float64)

    # ------------------------------------------------------------------
    def cells(self) -> np.ndarray:
        """Closed cells of the screen and the psi-coordinates of their
        indicators, Z (ndof x ncells).

        The oriented triangles (T, s) that share a sector at some vertex lie
        in the same connected region of R^3 minus the screen; the regions are
        the components of that relation.  A region is bounded exactly when
        the flux of x through its sides, sum |T| (x_T . n_(T,s)) / 3 with
        n_(T,s) pointing into the region, is minus its volume (negative); the
        unbounded one has zero or positive flux (divergence theorem).  For a
        cell K, the function that is 1 in K and 0 outside has, at vertex i,
        the value [sector j in K] on sector j; modulo the continuous
        functions its coordinate on psi_(i,j) is [sector j in K] - (number of
        sectors of i in K) / q_i (the coefficients minus their mean, Sec. 4.2).
        """
        nt = self.nt
        dsu = _DSU(2 * nt)
        first_node = {}
        for T in range(nt):
            for a in range(3):
                v = int(self.tri[T, a])
                for s in (0, 1):
                    key = (v, int(self.sector[T, s, a]))
                    node = 2 * T + s
                    if key in first_node:
                        dsu.union(first_node[key], node)
                    else:
                        first_node[key] = node
        roots = np.array([dsu.find(k) for k in range(2 * nt)])
        cen = self.xyz[self.tri].mean(axis=1)
        flux_T = self.area * np.einsum("ij,ij->i", cen, self.normal) / 3.0   # side +; side - has the opposite
        flux = {}
        for k in range(2 * nt):
            T, s = divmod(k, 2)
            flux[roots[k]] = flux.get(roots[k], 0.0) + (flux_T[T] if s == 0 else -flux_T[T])
        scale = float(self.area.sum() * np.abs(self.xyz).max() + 1e-300)
        cell_roots = sorted(r for r, f in flux.items() if f < -1e-9 * scale)
        cid = {r: c for c, r in enumerate(cell_roots)}
        Z = np.zeros((self.ndof, len(cell_roots)))
        # sectors of each vertex -> cell (every side in a sector is in one region)
        sec_cell = {}
        for T in range(nt):
            for a in range(3):
                v = int(self.tri[T, a])
                for s in (0, 1):
                    r = roots[2 * T + s]
                    sec_cell[(v, int(self.sector[T, s, a]))] = cid.get(r, -1)
        for v in range(self.nv):
            q = int(self.q[v])
            if q < 2:
                continue
            cnt = np.zeros(len(cell_roots))
            for j in range(q):
                c = sec_cell[(v, j)]
                if c >= 0:
                    cnt[c] += 1
            for j in range(q - 1):
                row = int(self.first_dof[v]) + j
                c = sec_cell[(v, j)]
                Z[row] = -cnt / q
                if c >= 0:
                    Z[row, c] += 1.0
        return Z

    def curl_vectors(self) -> np.ndarray:
        """s_{T,nu} for every curl-list entry: coef (x_{a+1} - x_{a+2}) / (2|T|)."""
        T, a = self.s_tri, self.s_loc
        xa1 = self.xyz[self.tri[T, (a + 1) % 3]]
        xa2 = self.xyz[self.tri[T, (a + 2) % 3]]
        return (self.s_coef / (2.0 * self.area[T]))[:, None] * (xa1 - xa2)

    def S_matrices(self):
        """Sparse S_k (nt x ndof), k = x, y, z: S_k[T, nu] = (s_{T,nu})_k."""
        import scipy.sparse as sp
        s = self.curl_vectors()
        return [sp.csr_matrix((s[:, k], (self.s_tri, self.s_dof)), shape=(self.nt, self.ndof))
                for k in range(3)]

    def jump_coefficients(self):
        """Sparse C (nt x ndof), C[T, nu] = c_+ - c_- (the jump of psi_nu across
        T at the vertex of nu, in units of lambda_a) with the local vertex a."""
        return self.s_tri, self.s_loc, self.s_dof, self.s_coef


def classify_dofs(top: Topology, patch) -> np.ndarray:
    """Face/wire-basket classes (Sec. 5, eq. jumpSplit): a dof (i,j) belongs to
    the face space of patch p when every triangle incident to x_i lies in
    patch p; otherwise to the wire basket (class -1)."""
    patch = np.asarray(patch)
    cls_v = np.full(top.nv, -2, dtype=np.int64)
    for T in range(top.nt):
        p = int(patch[T])
        for v in top.tri[T]:
            v = int(v)
            if cls_v[v] == -2:
                cls_v[v] = p
            elif cls_v[v] != p:
                cls_v[v] = -1
    return cls_v[top.dof_vertex]


def prolongation(fine: Topology, coarse: Topology, parent):
    """Coarse space V~_H([Gamma]) inside V~_h([Gamma]) (Sec. 5, eq. jumpSplit).

    Column mu = (I,J) holds the fine psi-coefficients of the coarse basis
    function psi^H_{I,J}: the coarse split function is evaluated at every fine
    generalized vertex x_{a,j} (its value is lambda_I(x_a) times
    [K = J] - [K = q_I] where K is the coarse sector containing the fine sector),
    and the sector mean at each fine vertex is removed (the l2-orthogonal
    complement Psi_h of the continuous functions, eq. orthogonalityVhYh)."""
    import scipy.sparse as sp
    parent = np.asarray(parent, dtype=np.int64)
    rows, cols, vals = [], [], []
    # members of each fine sector
    members = {}
    for T in range(fine.nt):
        for a in range(3):
            v = int(fine.tri[T, a])
            if fine.q[v] < 2:
                continue
            for s in (0, 1):
                members.setdefault((v, int(fine.sector[T, s, a])), []).append((T, s))
    for v in range(fine.nv):
        qv = int(fine.q[v])
        if qv < 2:
            continue
        x = fine.xyz[v]
        U = {}  # (mu) -> array over fine sectors
        for j in range(qv):
            seen = None
            for (T, s) in members[(v, j)]:
                Tc = int(parent[T])
                ct = coarse.tri[Tc]
                A, B, C = coarse.xyz[ct[0]], coarse.xyz[ct[1]], coarse.xyz[ct[2]]
                # barycentric coordinates of x in the coarse triangle
                M = np.stack([B - A, C - A], axis=1)
                l12, *_ = np.linalg.lstsq(M, x - A, rcond=None)
                lam = np.array([1.0 - l12.sum(), l12[0], l12[1]])
                same = float(np.dot(fine.normal[T], coarse.normal[Tc])) > 0
                sc = s if same else 1 - s
                vals_here = {}
                for c in range(3):
                    if lam[c] <= 1e-12:
                        continue
                    I = int(ct[c])
                    qI = int(coarse.q[I])
                    K = int(coarse.sector[Tc, sc, c])
                    for J in range(qI - 1):
                        cval = (1.0 if K == J else 0.0) - (1.0 if K == qI - 1 else 0.0)
                        mu = int(coarse.first_dof[I]) + J
                        vals_here[mu] = vals_here.get(mu, 0.0) + lam[c] * cval
                if seen is None:
                    seen = vals_here
                else:
                    keys = set(seen) | set(vals_here)
                    for kk in keys:
                        if abs(seen.get(kk, 0.0) - vals_here.get(kk, 0.0)) > 1e-9:
                            raise MeshError("fine sector straddles two coarse sectors")
            for mu, val in seen.items():
                U.setdefault(mu, np.zeros(qv))[j] += val
        for mu, arr in U.items():
            arr = arr - arr.mean()
            for j in range(qv - 1):
                if abs(arr[j]) > 1e-15:
                    rows.append(int(fine.first_dof[v]) + j)
                    cols.append(mu)
                    vals.append(arr[j])
    return sp.csr_matrix((vals, (rows, cols)), shape=(fine.ndof, coarse.ndof))
