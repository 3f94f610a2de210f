// Host topology of a polygonal multiscreen (Sec. 4.2-4.3 of the paper).
//
// The sets alpha_{k,l} of oriented triangles in each sector (eq. defAlphaij)
// are computed from the surface mesh alone: around every edge, the incident
// triangles are ordered by the angle of their third vertex about the edge
// axis; the two faces that bound a wedge between angular neighbours lie in the
// same connected component of the complement of Gamma near the edge, hence in
// the same sector at both edge end points.  An edge with a single triangle
// joins the two sides of that triangle.  Sectors of a vertex are the connected
// components of its oriented corners under these joins.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "msbem_internal.h"

namespace msbem {
namespace {

// Union-find whose root is the smallest index of its set: unite links the
// larger root under the smaller and path halving only moves links down, so
// p[i] <= i always, and one pass in index order (flatten) then points every
// node at its root.  Indices fit in 32 bits (at most 6 * 2^28 nodes).
struct Dsu {
  std::vector<int32_t> p;
  explicit Dsu(int64_t n) : p(n) { std::iota(p.begin(), p.end(), 0); }
  int32_t find(int64_t a) {
    while (p[a] != a) {
      p[a] = p[p[a]];
      a = p[a];
    }
    return (int32_t)a;
  }
  void unite(int64_t a, int64_t b) {
    const int32_t ra = find(a), rb = find(b);
    if (ra == rb) return;
    if (ra < rb) p[rb] = ra; else p[ra] = rb;
  }
  void flatten() {
    for (size_t i = 0; i < p.size(); ++i) p[i] = p[p[i]];
  }
};

inline void sub3(const double* a, const double* b, double* o) {
  o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
inline void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
inline double norm3(const double* a) { return std::sqrt(dot3(a, a)); }

inline int local_index(const int32_t* t, int32_t v) {
  return t[0] == v ? 0 : (t[1] == v ? 1 : (t[2] == v ? 2 : -1));
}

}  // namespace

int build_topology(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, Topo& o,
                   std::string& err) {
  if (nv <= 0 || nt <= 0 || !xyz || !tri) { err = "empty mesh"; return MSBEM_INVALID_ARG; }
  if (nt > (int64_t)1 << 28) { err = "too many triangles"; return MSBEM_INVALID_ARG; }
  o = Topo();
  o.nv = nv;
  o.nt = nt;
  o.xyz.assign(xyz, xyz + 3 * nv);
  o.tri.assign(tri, tri + 3 * nt);
  o.area.resize(nt);
  o.normal.resize(3 * nt);
  for (int64_t T = 0; T < nt; ++T) {
    const int32_t* t = &o.tri[3 * T];
    for (int a = 0; a < 3; ++a)
      if (t[a] < 0 || t[a] >= nv) { err = "vertex id out of range"; return MSBEM_INVALID_ARG; }
    if (t[0] == t[1] || t[1] == t[2] || t[0] == t[2]) {
      err = "triangle with a repeated vertex";
      return MSBEM_NONCONFORMING;
    }
    double e1[3], e2[3], c[3];
    sub3(&o.xyz[3 * t[1]], &o.xyz[3 * t[0]], e1);
    sub3(&o.xyz[3 * t[2]], &o.xyz[3 * t[0]], e2);
    cross3(e1, e2, c);
    double nc = norm3(c);
    double scale = std::max(dot3(e1, e1), dot3(e2, e2));
    if (!(nc > 1e-12 * scale)) { err = "degenerate triangle"; return MSBEM_NONCONFORMING; }
    o.area[T] = 0.5 * nc;
    for (int k = 0; k < 3; ++k) o.normal[3 * T + k] = c[k] / nc;
  }
  // duplicate triangles: the sorted vertex triples, bucketed by their
  // smallest vertex (counting sort); two equal triples share a bucket
  {
    std::vector<std::array<int32_t, 3>> keys(nt);
    std::vector<int64_t> start(nv + 1, 0);
    for (int64_t T = 0; T < nt; ++T) {
      std::array<int32_t, 3> k = {o.tri[3 * T], o.tri[3 * T + 1], o.tri[3 * T + 2]};
      if (k[0] > k[1]) std::swap(k[0], k[1]);
      if (k[1] > k[2]) std::swap(k[1], k[2]);
      if (k[0] > k[1]) std::swap(k[0], k[1]);
      keys[T] = k;
      start[k[0] + 1]++;
    }
    for (int64_t v = 0; v < nv; ++v) start[v + 1] += start[v];
    std::vector<std::array<int32_t, 3>> byv(nt);
    std::vector<int64_t> put(start.begin(), start.end() - 1);
    for (int64_t T = 0; T < nt; ++T) byv[put[keys[T][0]]++] = keys[T];
    for (int64_t v = 0; v < nv; ++v) {
      std::sort(byv.begin() + start[v], byv.begin() + start[v + 1]);
      for (int64_t x = start[v] + 1; x < start[v + 1]; ++x)
        if (byv[x] == byv[x - 1]) { err = "duplicate triangle"; return MSBEM_NONCONFORMING; }
    }
  }
  // edges: (lo, hi, T) sorted -- a counting sort on lo, then the few edges
  // of each lo (a vertex's degree) by insertion on (hi, T)
  struct E { int32_t lo, hi, T; };
  std::vector<E> edges(3 * nt);
  {
    std::vector<int64_t> start(nv + 1, 0);
    for (int64_t T = 0; T < nt; ++T)
      for (int a = 0; a < 3; ++a)
        start[std::min(o.tri[3 * T + a], o.tri[3 * T + (a + 1) % 3]) + 1]++;
    for (int64_t v = 0; v < nv; ++v) start[v + 1] += start[v];
    std::vector<int64_t> put(start.begin(), start.end() - 1);
    for (int64_t T = 0; T < nt; ++T)
      for (int a = 0; a < 3; ++a) {
        int32_t i = o.tri[3 * T + a], k = o.tri[3 * T + (a + 1) % 3];
        edges[put[std::min(i, k)]++] = {std::min(i, k), std::max(i, k), (int32_t)T};
      }
    for (int64_t v = 0; v < nv; ++v)
      for (int64_t x = start[v] + 1; x < start[v + 1]; ++x) {
        const E e = edges[x];
        int64_t y = x;
        while (y > start[v] && (edges[y - 1].hi > e.hi || (edges[y - 1].hi == e.hi && edges[y - 1].T > e.T))) {
          edges[y] = edges[y - 1];
          --y;
        }
        edges[y] = e;
      }
  }
  Dsu side(6 * nt);   // node (2T+s)*3 + a
  Dsu fan(3 * nt);    // node 3T + a
  auto node = [](int64_t T, int s, int a) { return (2 * T + s) * 3 + a; };
  std::vector<std::pair<double, int>> ang;
  std::vector<int> up;
  for (size_t e0 = 0; e0 < edges.size();) {
    size_t e1 = e0;
    while (e1 < edges.size() && edges[e1].lo == edges[e0].lo && edges[e1].hi == edges[e0].hi) ++e1;
    const int32_t vi = edges[e0].lo, vk = edges[e0].hi;
    const int m = (int)(e1 - e0);
    if (m == 1) {
      int32_t T = edges[e0].T;
      for (int32_t v : {vi, vk}) {
        int a = local_index(&o.tri[3 * T], v);
        side.unite(node(T, 0, a), node(T, 1, a));
      }
    } else if (m == 2) {
      // two triangles: the cyclic order is (0, 1) whatever their angle, so the
      // wedges are (0 up, 1 down) and (1 up, 0 down).  The angle of the second
      // about the edge, from the first, only decides whether they overlap
      // (within 1e-10 of 0 or 2 pi).  It can be that close only when its
      // sine is tiny and its cosine positive; a test on the unnormalised
      // directions (a bound 1e3 looser) picks those rare edges, and only for
      // them are the unit directions and the angle formed, as for m > 2.
      const double* xi = &o.xyz[3 * vi];
      double e[3];
      sub3(&o.xyz[3 * vk], xi, e);
      const double ee = dot3(e, e);
      double w[2][3];   // third vertex minus its projection on the edge line
      int up2[2];
      for (int j = 0; j < 2; ++j) {
        const int32_t T = edges[e0 + j].T;
        const int32_t* t = &o.tri[3 * T];
        const int32_t r = (t[0] != vi && t[0] != vk) ? t[0] : ((t[1] != vi && t[1] != vk) ? t[1] : t[2]);
        double d[3];
        sub3(&o.xyz[3 * r], xi, d);
        const double de = dot3(d, e) / ee;
        for (int k = 0; k < 3; ++k) w[j][k] = d[k] - de * e[k];
        double ew[3];
        cross3(e, w[j], ew);
        // the side facing increasing angle (u x d is a positive multiple of e x w)
        up2[j] = dot3(&o.normal[3 * T], ew) > 0 ? 0 : 1;
      }
      double ew0[3];
      cross3(e, w[0], ew0);
      const double c0 = dot3(w[1], w[0]), s0 = dot3(w[1], ew0);
      if (c0 > 0.0 && s0 * s0 < 1e-12 * ee * dot3(w[0], w[0]) * dot3(w[1], w[1])) {
        double u[3];
        const double nu = norm3(e);
        for (int k = 0; k < 3; ++k) u[k] = e[k] / nu;
        double d[2][3];
        for (int j = 0; j < 2; ++j) {
          const int32_t* t = &o.tri[3 * edges[e0 + j].T];
          const int32_t r = (t[0] != vi && t[0] != vk) ? t[0] : ((t[1] != vi && t[1] != vk) ? t[1] : t[2]);
          sub3(&o.xyz[3 * r], xi, d[j]);
          const double du = dot3(d[j], u);
          for (int k = 0; k < 3; ++k) d[j][k] -= du * u[k];
          const double nd = norm3(d[j]);
          for (int k = 0; k < 3; ++k) d[j][k] /= nd;
        }
        double ref2[3];
        cross3(u, d[0], ref2);
        const double cs = dot3(d[1], d[0]), sn = dot3(d[1], ref2);
        if (cs > 0.0 && std::fabs(sn) < 1e-9) {
          double th = std::atan2(sn, cs);
          if (th < 0) th += 2.0 * M_PI;
          if (th < 1e-10 || 2.0 * M_PI - th < 1e-10) { err = "overlapping triangles at an edge"; return MSBEM_NONCONFORMING; }
        }
      }
      const int32_t T0 = edges[e0].T, T1 = edges[e0 + 1].T;
      for (int32_t v : {vi, vk}) {
        const int a0 = local_index(&o.tri[3 * T0], v), a1 = local_index(&o.tri[3 * T1], v);
        side.unite(node(T0, up2[0], a0), node(T1, 1 - up2[1], a1));
        side.unite(node(T1, up2[1], a1), node(T0, 1 - up2[0], a0));
        fan.unite(3 * (int64_t)T0 + a0, 3 * (int64_t)T1 + a1);
      }
    } else {
      double u[3];
      sub3(&o.xyz[3 * vk], &o.xyz[3 * vi], u);
      double nu = norm3(u);
      for (int k = 0; k < 3; ++k) u[k] /= nu;
      double ref1[3] = {0, 0, 0}, ref2[3];
      ang.clear();
      up.assign(m, 0);
      for (int j = 0; j < m; ++j) {
        int32_t T = edges[e0 + j].T;
        const int32_t* t = &o.tri[3 * T];
        int32_t r = (t[0] != vi && t[0] != vk) ? t[0] : ((t[1] != vi && t[1] != vk) ? t[1] : t[2]);
        double d[3];
        sub3(&o.xyz[3 * r], &o.xyz[3 * vi], d);
        double du = dot3(d, u);
        for (int k = 0; k < 3; ++k) d[k] -= du * u[k];
        double nd = norm3(d);
        for (int k = 0; k < 3; ++k) d[k] /= nd;
        if (j == 0) {
          std::memcpy(ref1, d, sizeof ref1);
          cross3(u, ref1, ref2);
        }
        double th = std::atan2(dot3(d, ref2), dot3(d, ref1));
        if (th < 0) th += 2.0 * M_PI;
        double ud[3];
        cross3(u, d, ud);
        up[j] = dot3(&o.normal[3 * T], ud) > 0 ? 0 : 1;   // side facing increasing angle
        ang.push_back({th, j});
      }
      std::sort(ang.begin(), ang.end());
      for (int j = 0; j < m; ++j) {
        double a0 = ang[j].first;
        double a1 = (j + 1 < m) ? ang[j + 1].first : ang[0].first + 2.0 * M_PI;
        if (a1 - a0 < 1e-10) { err = "overlapping triangles at an edge"; return MSBEM_NONCONFORMING; }
      }
      for (int j = 0; j < m; ++j) {
        int ja = ang[j].second, jb = ang[(j + 1) % m].second;
        int32_t Ta = edges[e0 + ja].T, Tb = edges[e0 + jb].T;
        int sa = up[ja], sb = 1 - up[jb];
        for (int32_t v : {vi, vk})
          side.unite(node(Ta, sa, local_index(&o.tri[3 * Ta], v)),
                     node(Tb, sb, local_index(&o.tri[3 * Tb], v)));
      }
      for (int32_t v : {vi, vk}) {
        int32_t T0 = edges[e0].T;
        for (int j = 1; j < m; ++j) {
          int32_t T = edges[e0 + j].T;
          fan.unite(3 * (int64_t)T0 + local_index(&o.tri[3 * T0], v),
                    3 * (int64_t)T + local_index(&o.tri[3 * T], v));
        }
      }
    }
    e0 = e1;
  }
  side.flatten();   // from here on p[x] is the root of x
  fan.flatten();
  // corners per vertex (counting sort)
  std::vector<int64_t> cptr(nv + 1, 0);
  for (int64_t i = 0; i < 3 * nt; ++i) cptr[o.tri[i] + 1]++;
  for (int64_t v = 0; v < nv; ++v) cptr[v + 1] += cptr[v];
  std::vector<int64_t> corner(3 * nt), fill(cptr.begin(), cptr.end() - 1);
  for (int64_t i = 0; i < 3 * nt; ++i) corner[fill[o.tri[i]]++] = i;  // i = 3T + a
  o.q.assign(nv, 0);
  o.sector.assign(6 * nt, -1);
  std::vector<std::pair<int64_t, int64_t>> roots;  // (min key, root)
  for (int64_t v = 0; v < nv; ++v) {
    if (cptr[v] == cptr[v + 1]) continue;
    const int32_t r0 = fan.p[corner[cptr[v]]];
    for (int64_t c = cptr[v]; c < cptr[v + 1]; ++c)
      if (fan.p[corner[c]] != r0) {
        err = "point contact at vertex " + std::to_string(v);
        return MSBEM_POINT_CONTACT;
      }
    roots.clear();
    for (int64_t c = cptr[v]; c < cptr[v + 1]; ++c) {
      int64_t T = corner[c] / 3;
      int a = (int)(corner[c] % 3);
      for (int s = 0; s < 2; ++s) {
        const int64_t r = side.p[node(T, s, a)];
        int64_t key = 2 * T + s;
        bool found = false;
        for (auto& pr : roots)
          if (pr.second == r) { pr.first = std::min(pr.first, key); found = true; break; }
        if (!found) roots.push_back({key, r});
      }
    }
    std::sort(roots.begin(), roots.end());
    o.q[v] = (int32_t)roots.size();
    for (int64_t c = cptr[v]; c < cptr[v + 1]; ++c) {
      int64_t T = corner[c] / 3;
      int a = (int)(corner[c] % 3);
      for (int s = 0; s < 2; ++s) {
        const int64_t r = side.p[node(T, s, a)];
        for (size_t j = 0; j < roots.size(); ++j)
          if (roots[j].second == r) { o.sector[(2 * T + s) * 3 + a] = (int32_t)j; break; }
      }
    }
  }
  // dofs (i, j), j < q_i - 1 (0-based), vertex-major
  o.first_dof.assign(nv + 1, 0);
  for (int64_t v = 0; v < nv; ++v) o.first_dof[v + 1] = o.first_dof[v] + std::max(0, o.q[v] - 1);
  o.ndof = o.first_dof[nv];
  o.dof_vertex.resize(o.ndof);
  o.dof_sector.resize(o.ndof);
  for (int64_t v = 0; v < nv; ++v)
    for (int j = 0; j + 1 < o.q[v]; ++j) {
      o.dof_vertex[o.first_dof[v] + j] = (int32_t)v;
      o.dof_sector[o.first_dof[v] + j] = j;
    }
  // jump coefficients c_+ - c_- per (dof, triangle, local vertex)
  o.jptr.assign(o.ndof + 1, 0);
  auto coef_of = [&](int64_t T, int a, int j, int qv) {
    int sp = o.sector[(2 * T + 0) * 3 + a], sm = o.sector[(2 * T + 1) * 3 + a];
    int cp = (sp == j) - (sp == qv - 1);
    int cm = (sm == j) - (sm == qv - 1);
    return cp - cm;
  };
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<int64_t> pos;
    if (pass == 1) {
      for (int64_t d = 0; d < o.ndof; ++d) o.jptr[d + 1] += o.jptr[d];
      o.jtri.resize(o.jptr[o.ndof]);
      o.jloc.resize(o.jptr[o.ndof]);
      o.jcoef.resize(o.jptr[o.ndof]);
      pos.assign(o.jptr.begin(), o.jptr.end() - 1);
    }
    for (int64_t T = 0; T < nt; ++T)
      for (int a = 0; a < 3; ++a) {
        int32_t v = o.tri[3 * T + a];
        int qv = o.q[v];
        for (int j = 0; j + 1 < qv; ++j) {
          int c = coef_of(T, a, j, qv);
          if (!c) continue;
          int64_t d = o.first_dof[v] + j;
          if (pass == 0) {
            o.jptr[d + 1]++;
          } else {
            int64_t k = pos[d]++;
            o.jtri[k] = (int32_t)T;
            o.jloc[k] = a;
            o.jcoef[k] = (double)c;
          }
        }
      }
  }
  return MSBEM_OK;
}

// Regions of R^3 minus the screen: oriented triangles (T, s) that share a
// sector at a vertex lie in the same region (components of that relation).
// A region is bounded when the flux of x through its sides (normals into the
// region), sum |T| (c_T . n_(T,s)) / 3, is negative: minus its volume by the
// divergence theorem; the unbounded region's flux is zero or positive.  The
// indicator of a bounded cell K takes the value [sector j in K] on sector j of
// vertex i; modulo continuous functions its coordinate on psi_(i,j) is that
// value minus its mean over the q_i sectors.
void build_cells(Topo& t) {
  const int64_t nt = t.nt, nv = t.nv;
  std::vector<int64_t> sbase(nv + 1, 0);
  for (int64_t v = 0; v < nv; ++v) sbase[v + 1] = sbase[v] + t.q[v];
  std::vector<int64_t> rep(sbase[nv], -1);
  Dsu dsu(2 * nt);
  for (int64_t T = 0; T < nt; ++T)
    for (int a = 0; a < 3; ++a) {
      const int32_t v = t.tri[3 * T + a];
      for (int s = 0; s < 2; ++s) {
        const int64_t key = sbase[v] + t.sector[(2 * T + s) * 3 + a];
        const int64_t node = 2 * T + s;
        if (rep[key] < 0) rep[key] = node; else dsu.unite(rep[key], node);
      }
    }
  std::vector<double> flux(2 * nt, 0.0);
  double area_sum = 0.0, xmax = 0.0;
  for (int64_t i = 0; i < 3 * nv; ++i) xmax = std::max(xmax, std::fabs(t.xyz[i]));
  for (int64_t T = 0; T < nt; ++T) {
    double c[3];
    for (int k = 0; k < 3; ++k)
      c[k] = (t.xyz[3 * t.tri[3 * T] + k] + t.xyz[3 * t.tri[3 * T + 1] + k] + t.xyz[3 * t.tri[3 * T + 2] + k]) / 3.0;
    const double f = t.area[T] * (c[0] * t.normal[3 * T] + c[1] * t.normal[3 * T + 1] + c[2] * t.normal[3 * T + 2]) / 3.0;
    flux[dsu.find(2 * T)] += f;
    flux[dsu.find(2 * T + 1)] -= f;
    area_sum += t.area[T];
  }
  const double tol = 1e-9 * (area_sum * xmax + 1e-300);
  std::vector<int> cell_of_root(2 * nt, -1);
  int nc = 0;
  for (int64_t r = 0; r < 2 * nt; ++r)
    if (dsu.find(r) == r && flux[r] < -tol) cell_of_root[r] = nc++;
  t.ncells = nc;
  t.cellZ.assign((size_t)t.ndof * nc, 0.0);
  if (!nc) return;
  std::vector<int> sec_cell(sbase[nv], -1);
  for (int64_t T = 0; T < nt; ++T)
    for (int a = 0; a < 3; ++a) {
      const int32_t v = t.tri[3 * T + a];
      for (int s = 0; s < 2; ++s)
        sec_cell[sbase[v] + t.sector[(2 * T + s) * 3 + a]] = cell_of_root[dsu.find(2 * T + s)];
    }
  std::vector<double> cnt(nc);
  for (int64_t v = 0; v < nv; ++v) {
    const int q = t.q[v];
    if (q < 2) continue;
    std::fill(cnt.begin(), cnt.end(), 0.0);
    for (int j = 0; j < q; ++j)
      if (sec_cell[sbase[v] + j] >= 0) cnt[sec_cell[sbase[v] + j]] += 1.0;
    for (int j = 0; j + 1 < q; ++j) {
      double* z = &t.cellZ[(size_t)(t.first_dof[v] + j) * nc];
      for (int c = 0; c < nc; ++c) z[c] = -cnt[c] / q;
      const int c = sec_cell[sbase[v] + j];
      if (c >= 0) z[c] += 1.0;
    }
  }
  // orthonormal basis Q = Z L^-T of the kernel (Z^T Z = L L^T, Cholesky)
  std::vector<double> G((size_t)nc * nc, 0.0), Lc((size_t)nc * nc, 0.0);
  for (int64_t r = 0; r < t.ndof; ++r) {
    const double* z = &t.cellZ[(size_t)r * nc];
    for (int a = 0; a < nc; ++a)
      for (int b = 0; b < nc; ++b) G[(size_t)a * nc + b] += z[a] * z[b];
  }
  for (int a = 0; a < nc; ++a) {
    for (int b = 0; b <= a; ++b) {
      double sum = G[(size_t)a * nc + b];
      for (int k = 0; k < b; ++k) sum -= Lc[(size_t)a * nc + k] * Lc[(size_t)b * nc + k];
      Lc[(size_t)a * nc + b] = (a == b) ? std::sqrt(sum) : sum / Lc[(size_t)b * nc + b];
    }
  }
  t.cellQ.assign(t.cellZ.size(), 0.0);
  for (int64_t r = 0; r < t.ndof; ++r) {
    const double* z = &t.cellZ[(size_t)r * nc];
    double* qv = &t.cellQ[(size_t)r * nc];
    for (int a = 0; a < nc; ++a) {   // L q = z (forward substitution)
      double sum = z[a];
      for (int k = 0; k < a; ++k) sum -= Lc[(size_t)a * nc + k] * qv[k];
      qv[a] = sum / Lc[(size_t)a * nc + a];
    }
  }
}

void build_near_pairs(const Topo& t, std::vector<NearPair>& out) {
  out.clear();
  const int64_t nt = t.nt, nv = t.nv;
  std::vector<int64_t> cptr(nv + 1, 0);
  for (int64_t i = 0; i < 3 * nt; ++i) cptr[t.tri[i] + 1]++;
  for (int64_t v = 0; v < nv; ++v) cptr[v + 1] += cptr[v];
  std::vector<int32_t> inc(3 * nt);
  std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
  for (int64_t i = 0; i < 3 * nt; ++i) inc[fill[t.tri[i]]++] = (int32_t)(i / 3);
  // candidates S >= T sharing a vertex with T, deduplicated with a stamp array;
  // kept in increasing S so the list order is deterministic
  std::vector<int32_t> stamp(nt, -1);
  std::vector<int32_t> nb;
  nb.reserve(64);
  out.reserve((size_t)nt * 8);
  for (int64_t T = 0; T < nt; ++T) {
    nb.clear();
    for (int a = 0; a < 3; ++a) {
      int32_t v = t.tri[3 * T + a];
      for (int64_t c = cptr[v]; c < cptr[v + 1]; ++c) {
        const int32_t S = inc[c];
        if (S >= T && stamp[S] != (int32_t)T) {
          stamp[S] = (int32_t)T;
          nb.push_back(S);
        }
      }
    }
    std::sort(nb.begin(), nb.end());
    const int32_t* a = &t.tri[3 * T];
    for (int32_t S : nb) {
      const int32_t* b = &t.tri[3 * S];
      NearPair p;
      p.T = (int32_t)T;
      p.S = S;
      if (S == T) {
        p.cls = 3;
        for (int k = 0; k < 3; ++k) { p.v[k] = a[k]; p.v[3 + k] = a[k]; }
        out.push_back(p);
        continue;
      }
      int ia[3], ib[3], ns = 0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          if (a[i] == b[j]) { ia[ns] = i; ib[ns] = j; ++ns; }
      if (ns == 1) {
        p.cls = 1;
        for (int k = 0; k < 3; ++k) {
          p.v[k] = a[(ia[0] + k) % 3];
          p.v[3 + k] = b[(ib[0] + k) % 3];
        }
      } else {
        p.cls = 2;
        int iA = ia[0], iB = ia[1], jA = ib[0], jB = ib[1];
        if (a[iA] > a[iB]) { std::swap(iA, iB); std::swap(jA, jB); }
        p.v[0] = a[iA]; p.v[1] = a[iB]; p.v[2] = a[3 - iA - iB];
        p.v[3] = b[jA]; p.v[4] = b[jB]; p.v[5] = b[3 - jA - jB];
      }
      out.push_back(p);
    }
  }
}

// ---------------------------------------------------------------------------
// Face / wire-basket split and coarse prolongation (Sec. 5, eq. jumpSplit).
// The coarse space is the jump space of P1 on the coarse mesh; its basis
// function psi^H_{I,J} is written in the fine basis by evaluating the coarse
// split function at every fine generalized vertex and removing the sector
// mean at each fine vertex (the l2-orthogonal complement Psi_h of the
// continuous functions, eq. orthogonalityVhYh).
// ---------------------------------------------------------------------------
int build_split(const Topo& f, const Topo& c, const int32_t* parent, const int32_t* patch, Split& o,
                std::string& err) {
  o = Split();
  const int64_t nt = f.nt, nv = f.nv;
  for (int64_t T = 0; T < nt; ++T) {
    if (parent[T] < 0 || parent[T] >= c.nt) { err = "parent id out of range"; return MSBEM_INVALID_ARG; }
    if (patch[T] < 0) { err = "negative patch id"; return MSBEM_INVALID_ARG; }
  }
  // nesting check: fine vertices inside the parent's plane and triangle
  // (the coarse triangles' edge vectors and Gram entries computed once each)
  struct CoarseFrame { double e1[3], e2[3], d11, d12, d22, den, hs; };
  std::vector<CoarseFrame> frame(c.nt);
  for (int64_t Tc = 0; Tc < c.nt; ++Tc) {
    const int32_t* ct = &c.tri[3 * Tc];
    CoarseFrame& F = frame[Tc];
    sub3(&c.xyz[3 * ct[1]], &c.xyz[3 * ct[0]], F.e1);
    sub3(&c.xyz[3 * ct[2]], &c.xyz[3 * ct[0]], F.e2);
    F.d11 = dot3(F.e1, F.e1);
    F.d12 = dot3(F.e1, F.e2);
    F.d22 = dot3(F.e2, F.e2);
    F.den = F.d11 * F.d22 - F.d12 * F.d12;
    F.hs = std::sqrt(c.area[Tc]);
  }
  auto bary = [&](int64_t Tc, const double* x, double lam[3]) {
    const CoarseFrame& F = frame[Tc];
    double d[3];
    sub3(x, &c.xyz[3 * c.tri[3 * Tc]], d);
    double p1 = dot3(d, F.e1), p2 = dot3(d, F.e2);
    double l1 = (F.d22 * p1 - F.d12 * p2) / F.den, l2 = (F.d11 * p2 - F.d12 * p1) / F.den;
    lam[0] = 1.0 - l1 - l2;
    lam[1] = l1;
    lam[2] = l2;
    double off = std::fabs(dot3(d, &c.normal[3 * Tc]));
    return off;
  };
  for (int64_t T = 0; T < nt; ++T)
    for (int a = 0; a < 3; ++a) {
      double lam[3];
      double off = bary(parent[T], &f.xyz[3 * f.tri[3 * T + a]], lam);
      double hs = frame[parent[T]].hs;
      if (off > 1e-9 * hs || lam[0] < -1e-9 || lam[1] < -1e-9 || lam[2] < -1e-9) {
        err = "fine mesh not nested in the coarse mesh";
        return MSBEM_NONCONFORMING;
      }
    }
  // vertex classes
  std::vector<int64_t> cls(nv, -2);
  for (int64_t T = 0; T < nt; ++T)
    for (int a = 0; a < 3; ++a) {
      int32_t v = f.tri[3 * T + a];
      if (cls[v] == -2) cls[v] = patch[T];
      else if (cls[v] != patch[T]) cls[v] = -1;
    }
  int64_t maxp = 0;
  for (int64_t T = 0; T < nt; ++T) maxp = std::max<int64_t>(maxp, patch[T] + 1);
  std::vector<int64_t> cnt(maxp + 1, 0);   // last slot: wire basket
  for (int64_t d = 0; d < f.ndof; ++d) {
    int64_t k = cls[f.dof_vertex[d]];
    cnt[k < 0 ? maxp : k]++;
  }
  // blocks: non-empty faces in patch order, then the wire basket
  std::vector<int64_t> block_of(maxp + 1, -1);
  o.block_ptr.push_back(0);
  for (int64_t p = 0; p < maxp; ++p)
    if (cnt[p] > 0) {
      block_of[p] = (int64_t)o.block_ptr.size() - 1;
      o.block_ptr.push_back(o.block_ptr.back() + cnt[p]);
      o.max_face = std::max(o.max_face, cnt[p]);
    }
  o.n_faces = (int64_t)o.block_ptr.size() - 1;
  o.n_wb = cnt[maxp];
  if (o.n_wb > 0) {
    block_of[maxp] = (int64_t)o.block_ptr.size() - 1;
    o.block_ptr.push_back(o.block_ptr.back() + o.n_wb);
  }
  o.block_dofs.resize(f.ndof);
  {
    std::vector<int64_t> pos(o.block_ptr.begin(), o.block_ptr.end() - 1);
    for (int64_t d = 0; d < f.ndof; ++d) {
      int64_t k = cls[f.dof_vertex[d]];
      int64_t b = block_of[k < 0 ? maxp : k];
      o.block_dofs[pos[b]++] = (int32_t)d;
    }
  }
  // coarse prolongation
  o.n_coarse = c.ndof;
  o.p_ptr.assign(f.ndof + 1, 0);
  if (c.ndof == 0) return MSBEM_OK;
  // representative oriented triangle of every fine sector
  std::vector<int64_t> sec_first(nv + 1, 0);
  for (int64_t v = 0; v < nv; ++v) sec_first[v + 1] = sec_first[v] + f.q[v];
  std::vector<int64_t> sec_rep(sec_first[nv], -1);  // (2T+s)*3+a
  for (int64_t T = 0; T < nt; ++T)
    for (int s = 0; s < 2; ++s)
      for (int a = 0; a < 3; ++a) {
        int32_t v = f.tri[3 * T + a];
        int64_t slot = sec_first[v] + f.sector[(2 * T + s) * 3 + a];
        if (sec_rep[slot] < 0) sec_rep[slot] = (2 * T + s) * 3 + a;
      }
  // rows of P in dof order: the dofs of a vertex are consecutive and the
  // vertices are visited in increasing order, so each row is appended to the
  // CSR arrays as soon as it is formed (entries sorted by coarse dof)
  std::vector<double> U;
  std::vector<int32_t> mus;
  std::vector<std::pair<int32_t, double>> row;
  int64_t done_dof = 0;   // rows of P written so far
  for (int64_t v = 0; v < nv; ++v) {
    const int qv = f.q[v];
    if (qv < 2) continue;
    mus.clear();
    U.clear();
    for (int j = 0; j < qv; ++j) {
      int64_t id = sec_rep[sec_first[v] + j];
      int64_t T = id / 6, s = (id / 3) % 2;
      int64_t Tc = parent[T];
      double lam[3];
      bary(Tc, &f.xyz[3 * v], lam);
      bool same = dot3(&f.normal[3 * T], &c.normal[3 * Tc]) > 0;
      int sc = same ? (int)s : 1 - (int)s;
      for (int cc = 0; cc < 3; ++cc) {
        if (lam[cc] <= 1e-12) continue;
        int32_t I = c.tri[3 * Tc + cc];
        int qI = c.q[I];
        int K = c.sector[(2 * Tc + sc) * 3 + cc];
        for (int J = 0; J + 1 < qI; ++J) {
          double cv = (double)((K == J) - (K == qI - 1));
          if (cv == 0.0) continue;
          int32_t mu = (int32_t)(c.first_dof[I] + J);
          size_t m = 0;
          while (m < mus.size() && mus[m] != mu) ++m;
          if (m == mus.size()) {
            mus.push_back(mu);
            U.resize(U.size() + qv, 0.0);
          }
          U[m * qv + j] += lam[cc] * cv;
        }
      }
    }
    std::vector<double> mean(mus.size(), 0.0);
    for (size_t m = 0; m < mus.size(); ++m) {
      for (int j = 0; j < qv; ++j) mean[m] += U[m * qv + j];
      mean[m] /= qv;
    }
    for (int j = 0; j + 1 < qv; ++j) {
      const int64_t d = f.first_dof[v] + j;
      for (; done_dof < d; ++done_dof) o.p_ptr[done_dof + 1] = o.p_ptr[done_dof];
      row.clear();
      for (size_t m = 0; m < mus.size(); ++m) {
        double val = U[m * qv + j] - mean[m];
        if (std::fabs(val) > 1e-15) row.push_back({mus[m], val});
      }
      std::sort(row.begin(), row.end());
      for (auto& pr : row) {
        o.p_col.push_back(pr.first);
        o.p_val.push_back(pr.second);
      }
      o.p_ptr[d + 1] = o.p_ptr[d] + (int64_t)row.size();
      done_dof = d + 1;
    }
  }
  for (; done_dof < f.ndof; ++done_dof) o.p_ptr[done_dof + 1] = o.p_ptr[done_dof];
  return MSBEM_OK;
}

// ---------------------------------------------------------------------------
// Quadrature constants (host).
// ---------------------------------------------------------------------------
void gauss_legendre01(int n, double* x, double* w) {
  // Golub-Welsch would need an eigensolver; Newton on P_n from the classical
  // cosine initial guess converges quadratically for every root.
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 200; ++it) {
      double pkm1 = 1.0, pk = t;
      for (int k = 2; k <= n; ++k) {
        double pk1 = ((2.0 * k - 1.0) * t * pk - (k - 1.0) * pkm1) / k;
        pkm1 = pk;
        pk = pk1;
      }
      if (n == 1) { pk = t; pkm1 = 1.0; }
      dp = n * (pkm1 - t * pk) / (1.0 - t * t);
      double step = pk / dp;
      t -= step;
      if (std::fabs(step) <= 1e-17) break;
    }
    double pkm1 = 1.0, pk = t;
    for (int k = 2; k <= n; ++k) {
      double pk1 = ((2.0 * k - 1.0) * t * pk - (k - 1.0) * pkm1) / k;
      pkm1 = pk;
      pk = pk1;
    }
    if (n == 1) { pk = t; pkm1 = 1.0; }
    dp = n * (pkm1 - t * pk) / (1.0 - t * t);
    x[n - 1 - i] = 0.5 * (1.0 + t);          // ascending on [0, 1]
    w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);
  }
}

void six_point_rule(double bary[6][3], double w[6]) {
  // symmetric degree-4 rule: orbits (a,a,1-2a) and (b,b,1-2b)
  const double r10 = std::sqrt(10.0);
  const double s = std::sqrt(38.0 - 44.0 * std::sqrt(2.0 / 5.0));
  const double a = (8.0 - r10 + s) / 18.0, b = (8.0 - r10 - s) / 18.0;
  const double t = std::sqrt(213125.0 - 53320.0 * r10);
  const double wa = (620.0 + t) / 3720.0, wb = (620.0 - t) / 3720.0;
  const double orb[2] = {a, b};
  for (int o = 0; o < 2; ++o)
    for (int k = 0; k < 3; ++k) {
      for (int m = 0; m < 3; ++m) bary[3 * o + k][m] = (m == k) ? 1.0 - 2.0 * orb[o] : orb[o];
      w[3 * o + k] = o == 0 ? wa : wb;
    }
}

}  // namespace msbem
