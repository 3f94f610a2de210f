/*
 * CPU FP64 oracle: quadrature core.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or run this file.  It
 * shares no code with the CUDA library and includes none of its headers.
 *
 * What it computes (plain definitions, slow on purpose):
 *
 *   V[T,T'] = int_T int_T' 1 / (4 pi |x - y|) dy dx
 *
 * for every pair of flat triangles of a surface mesh.  By Cor. corW and
 * eq. (eval_a_phiij) of the paper (Sec. 3.4, Sec. 4.3), the surface curls of
 * the piecewise-linear shape functions are constant on each triangle, so the
 * hypersingular Galerkin matrix is W = sum_k S_k^T V S_k; the Python side of
 * the oracle forms S_k and that product.
 *
 * Quadrature (the paper fixes none; these readings are the workload's):
 *   - pairs sharing no vertex: the symmetric 6-point degree-4 triangle rule
 *     (Strang-Fix/Dunavant) on each triangle, 36 kernel evaluations;
 *   - identical, edge-adjacent and vertex-adjacent pairs: Sauter-Schwab-type
 *     regularising maps onto [0,1]^4 (6, 4 and 2 regions), Gauss-Legendre
 *     of order n in each of the four coordinates.
 *
 * The regularising maps are written out in the comments of each routine.
 * Reference triangle:  That = { 0 <= s2 <= s1 <= 1 },
 *   chi(s) = P0 + s1 (P1 - P0) + s2 (P2 - P1),   dx = 2|T| ds.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define ORC_PI 3.14159265358979323846

/* ----------------------------------------------------------------------- */
/* 1-D Gauss-Legendre on [0,1]: Newton iteration on the Legendre recurrence */
/* ----------------------------------------------------------------------- */
int orc_gauss_legendre01(int n, double* x, double* w) {
  if (n < 1 || n > 64) return -1;
  for (int i = 0; i < n; ++i) {
    /* root i of P_n on [-1,1] (descending), Newton from a cosine guess */
    double t = cos(ORC_PI * (i + 0.75) / (n + 0.5));
    double pn = 0.0, pm = 0.0, dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      /* (k+1) P_{k+1} = (2k+1) t P_k - k P_{k-1} */
      double p0 = 1.0, p1 = t;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
        p0 = p1; p1 = p2;
      }
      pn = p1; pm = (n == 1) ? 1.0 : p0;
      dp = n * (t * pn - pm) / (t * t - 1.0);      /* P_n'(t) */
      double dt = pn / dp;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    double p0 = 1.0, p1 = t;
    for (int k = 1; k < n; ++k) {
      double p2 = ((2.0 * k + 1.0) * t * p1 - k * p0) / (k + 1.0);
      p0 = p1; p1 = p2;
    }
    pm = (n == 1) ? 1.0 : p0;
    dp = n * (t * p1 - pm) / (t * t - 1.0);
    x[i] = 0.5 * (1.0 - t);                          /* ascending on [0,1] */
    w[i] = 1.0 / ((1.0 - t * t) * dp * dp);          /* (2/((1-t^2)P'^2)) / 2 */
  }
  return 0;
}

/* ----------------------------------------------------------------------- */
/* 6-point degree-4 symmetric triangle rule (Strang-Fix / Dunavant 1985).   */
/* Orbits (a,a,1-2a) with weight wa and (b,b,1-2b) with weight wb, weights   */
/* normalised to sum 1.  Closed forms of the published constants:            */
/*   a  = (8 - sqrt10 + sqrt(38 - 44 sqrt(2/5))) / 18                        */
/*   b  = (8 - sqrt10 - sqrt(38 - 44 sqrt(2/5))) / 18                        */
/*   wa = (620 + sqrt(213125 - 53320 sqrt10)) / 3720,  wb = 1/3 - wa         */
/* ----------------------------------------------------------------------- */
void orc_dunavant6(double* bary /*[6*3]*/, double* w /*[6]*/) {
  double s10 = sqrt(10.0);
  double r = sqrt(38.0 - 44.0 * sqrt(0.4));
  double a = (8.0 - s10 + r) / 18.0;
  double b = (8.0 - s10 - r) / 18.0;
  double wa = (620.0 + sqrt(213125.0 - 53320.0 * s10)) / 3720.0;
  double wb = (620.0 - sqrt(213125.0 - 53320.0 * s10)) / 3720.0;
  double pts[6][3] = {{a, a, 1 - 2 * a}, {a, 1 - 2 * a, a}, {1 - 2 * a, a, a},
                      {b, b, 1 - 2 * b}, {b, 1 - 2 * b, b}, {1 - 2 * b, b, b}};
  for (int i = 0; i < 6; ++i) {
    for (int k = 0; k < 3; ++k) bary[3 * i + k] = pts[i][k];
    w[i] = (i < 3) ? wa : wb;
  }
}

/* ----------------------------------------------------------------------- */
/* kernels: id 0 is the Laplace single-layer kernel; the others are smooth  */
/* test integrands used to pin the regularising maps.                       */
/* x, y absolute points; d = x - y formed from local coordinates.           */
/* ----------------------------------------------------------------------- */
static double kern(int id, const double* x, const double* y, const double* d) {
  switch (id) {
    case 0: return 1.0 / (4.0 * ORC_PI * sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
    case 1: return 1.0;
    case 2: return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    case 3: return x[0] * y[1] + 2.0 * x[2] - y[0] * y[0] + x[1] * x[1] * y[2];
    case 4: { double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2]; return r2 * r2 + x[0]; }
    default: return 0.0;
  }
}

static double tri_area(const double* P) {
  double e1[3], e2[3], c[3];
  for (int k = 0; k < 3; ++k) { e1[k] = P[3 + k] - P[k]; e2[k] = P[6 + k] - P[k]; }
  c[0] = e1[1] * e2[2] - e1[2] * e2[1];
  c[1] = e1[2] * e2[0] - e1[0] * e2[2];
  c[2] = e1[0] * e2[1] - e1[1] * e2[0];
  return 0.5 * sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
}

/* ----------------------------------------------------------------------- */
/* Separated pairs.  far_order 0: the 6-point rule on each triangle.         */
/* far_order n > 0: collapsed (Duffy) Gauss product rule with n^2 points per */
/* triangle (only for convergence studies).                                  */
/* ----------------------------------------------------------------------- */
static int triangle_rule(int far_order, double* bary, double* w) {
  if (far_order == 0) { orc_dunavant6(bary, w); return 6; }
  double gx[64], gw[64];
  orc_gauss_legendre01(far_order, gx, gw);
  int m = 0;
  for (int i = 0; i < far_order; ++i)
    for (int j = 0; j < far_order; ++j) {
      /* s1 = u, s2 = u v on That; barycentric of chi(s) = (1-s1, s1-s2, s2) */
      double u = gx[i], v = gx[j];
      double s1 = u, s2 = u * v;
      bary[3 * m + 0] = 1.0 - s1;
      bary[3 * m + 1] = s1 - s2;
      bary[3 * m + 2] = s2;
      w[m] = gw[i] * gw[j] * u * 2.0;   /* reference area 1/2 -> weights sum 1 */
      ++m;
    }
  return m;
}

double orc_rule_far(const double* P, const double* Q, int kernel_id, int far_order) {
  double bp6[18], wp6[6];
  double* bp = bp6;
  double* wp = wp6;
  if (far_order > 0) {
    bp = (double*)malloc(sizeof(double) * 3 * far_order * far_order);
    wp = (double*)malloc(sizeof(double) * far_order * far_order);
  }
  int m = triangle_rule(far_order, bp, wp);
  double sum = 0.0;
  for (int p = 0; p < m; ++p) {
    double x[3];
    for (int k = 0; k < 3; ++k) x[k] = bp[3 * p] * P[k] + bp[3 * p + 1] * P[3 + k] + bp[3 * p + 2] * P[6 + k];
    double inner = 0.0;
    for (int q = 0; q < m; ++q) {
      double y[3], d[3];
      for (int k = 0; k < 3; ++k) {
        y[k] = bp[3 * q] * Q[k] + bp[3 * q + 1] * Q[3 + k] + bp[3 * q + 2] * Q[6 + k];
        d[k] = x[k] - y[k];
      }
      inner += wp[q] * kern(kernel_id, x, y, d);
    }
    sum += wp[p] * inner;
  }
  if (far_order > 0) { free(bp); free(wp); }
  return tri_area(P) * tri_area(Q) * sum;
}

/* ----------------------------------------------------------------------- */
/* Identical pair T = T' = (P0,P1,P2).                                       */
/* Relative coordinates z = t - s (s, t in That).  For fixed z the admissible */
/* s form the triangle { u_k >= m_k } in the coordinates u = (s2, 1-s1,      */
/* s1-s2), with m = (max(0,-z2), max(0,z1), max(0,z2-z1)): a copy of That    */
/* scaled by 1 - sum m and shifted by (m1+m3, m1).  The difference body is   */
/* the hexagon with vertices (1,0),(1,1),(0,1),(-1,0),(-1,-1),(0,-1); on each */
/* of its 6 triangles (origin, H_i, H_{i+1}) sum m is linear and equals 1 on  */
/* the outer edge.  Map per region:                                          */
/*   z = xi ((1-eta) H_i + eta H_{i+1}),  dz = xi d(xi) d(eta)               */
/*   s = (m1+m3, m1) + (1-xi) (e2, e2 e3),  ds = (1-xi)^2 e2 d(e2) d(e3)     */
/* so the integrand carries xi (1-xi)^2 e2 and 1/|x-y| = O(1/xi) cancels.    */
/* ----------------------------------------------------------------------- */
double orc_rule_identical(const double* P, int n, int kernel_id) {
  static const double H[6][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 0}, {-1, -1}, {0, -1}};
  double gx[64], gw[64];
  orc_gauss_legendre01(n, gx, gw);
  double e1[3], e2[3];
  for (int k = 0; k < 3; ++k) { e1[k] = P[3 + k] - P[k]; e2[k] = P[6 + k] - P[3 + k]; }
  double area = tri_area(P);
  double sum = 0.0;
  for (int reg = 0; reg < 6; ++reg) {
    const double* a = H[reg];
    const double* b = H[(reg + 1) % 6];
    for (int i0 = 0; i0 < n; ++i0)
      for (int i1 = 0; i1 < n; ++i1)
        for (int i2 = 0; i2 < n; ++i2)
          for (int i3 = 0; i3 < n; ++i3) {
            double xi = gx[i0], eta = gx[i1], e2v = gx[i2], e3v = gx[i3];
            double wq = gw[i0] * gw[i1] * gw[i2] * gw[i3];
            double z1 = xi * ((1 - eta) * a[0] + eta * b[0]);
            double z2 = xi * ((1 - eta) * a[1] + eta * b[1]);
            double m1 = fmax(0.0, -z2), m2 = fmax(0.0, z1), m3 = fmax(0.0, z2 - z1);
            double sc = 1.0 - (m1 + m2 + m3);
            double s1 = m1 + m3 + sc * e2v;
            double s2 = m1 + sc * e2v * e3v;
            double t1 = s1 + z1, t2 = s2 + z2;
            double x[3], y[3], d[3];
            for (int k = 0; k < 3; ++k) {
              x[k] = P[k] + s1 * e1[k] + s2 * e2[k];
              y[k] = P[k] + t1 * e1[k] + t2 * e2[k];
              d[k] = (s1 - t1) * e1[k] + (s2 - t2) * e2[k];
            }
            double jac = xi * sc * sc * e2v;
            sum += wq * jac * kern(kernel_id, x, y, d);
          }
  }
  return 4.0 * area * area * sum;
}

/* ----------------------------------------------------------------------- */
/* Edge-adjacent pair T = (A,B,C), T' = (A,B,D), common edge AB.             */
/*   x = A + s1 (B-A) + s2 (C-B),  y = A + t1 (B-A) + t2 (D-B).              */
/* Variables (u,v,w) = (t1 - s1, s2, t2) and s1.  The admissible s1 form the */
/* interval [max(v, w-u), 1 - max(0,u)] of length 1 - l(u,v,w) with          */
/* l = max(0,u) + max(v, w-u), homogeneous of degree 1.  The (u,v,w) domain   */
/* { v,w >= 0, l <= 1 } splits into 4 cones where l is linear:               */
/*   A: u>=0, v>=w-u (l=u+v)  face (sg, 1-sg, ta)             J=1  lo = v     */
/*   B: u>=0, v<=w-u (l=w)    face (s, t, 1)  s+t<=1          J=sg lo = w-u   */
/*   C: u<=0, v>=w-u (l=v)    face (-s, 1, t) s+t<=1          J=sg lo = v     */
/*   D: u<=0, v<=w-u (l=w-u)  face (-sg, ta, 1-sg)            J=1  lo = w-u   */
/* with (s,t) = (sg(1-ta), sg ta) on the triangular faces.  Map per cone:     */
/*   (u,v,w) = xi f(sg,ta),  s1 = lo + (1-xi) e4,                            */
/*   Jacobian xi^2 J(sg) (1-xi); 1/|x-y| = O(1/xi).                          */
/* ----------------------------------------------------------------------- */
double orc_rule_edge(const double* P, const double* Q, int n, int kernel_id) {
  double gx[64], gw[64];
  orc_gauss_legendre01(n, gx, gw);
  double e[3], c[3], dd[3];
  for (int k = 0; k < 3; ++k) {
    e[k] = P[3 + k] - P[k];        /* B - A */
    c[k] = P[6 + k] - P[3 + k];    /* C - B */
    dd[k] = Q[6 + k] - Q[3 + k];   /* D - B */
  }
  double aT = tri_area(P), aS = tri_area(Q);
  double sum = 0.0;
  for (int reg = 0; reg < 4; ++reg)
    for (int i0 = 0; i0 < n; ++i0)
      for (int i1 = 0; i1 < n; ++i1)
        for (int i2 = 0; i2 < n; ++i2)
          for (int i3 = 0; i3 < n; ++i3) {
            double xi = gx[i0], sg = gx[i1], ta = gx[i2], e4 = gx[i3];
            double wq = gw[i0] * gw[i1] * gw[i2] * gw[i3];
            double fu, fv, fw, J;
            int lo_is_v;
            if (reg == 0) { fu = sg; fv = 1 - sg; fw = ta; J = 1; lo_is_v = 1; }
            else if (reg == 1) { fu = sg * (1 - ta); fv = sg * ta; fw = 1; J = sg; lo_is_v = 0; }
            else if (reg == 2) { fu = -sg * (1 - ta); fv = 1; fw = sg * ta; J = sg; lo_is_v = 1; }
            else { fu = -sg; fv = ta; fw = 1 - sg; J = 1; lo_is_v = 0; }
            double u = xi * fu, v = xi * fv, w = xi * fw;
            double lo = lo_is_v ? v : (w - u);
            double s1 = lo + (1 - xi) * e4, s2 = v;
            double t1 = s1 + u, t2 = w;
            double x[3], y[3], d[3];
            for (int k = 0; k < 3; ++k) {
              x[k] = P[k] + s1 * e[k] + s2 * c[k];
              y[k] = P[k] + t1 * e[k] + t2 * dd[k];
              d[k] = (s1 - t1) * e[k] + s2 * c[k] - t2 * dd[k];
            }
            double jac = xi * xi * J * (1 - xi);
            sum += wq * jac * kern(kernel_id, x, y, d);
          }
  return 4.0 * aT * aS * sum;
}

/* ----------------------------------------------------------------------- */
/* Vertex-adjacent pair T = (O,P1,P2), T' = (O,Q1,Q2), common vertex O.      */
/*   x = O + s1 (P1-O) + s2 (P2-P1),  y = O + t1 (Q1-O) + t2 (Q2-Q1).        */
/* Two regions: s1 >= t1:  s = xi (1, e1),  t = xi e2 (1, e3);               */
/*              t1 >= s1:  t = xi (1, e1),  s = xi e2 (1, e3);               */
/* Jacobian xi^3 e2; 1/|x-y| = O(1/xi).                                      */
/* ----------------------------------------------------------------------- */
double orc_rule_vertex(const double* P, const double* Q, int n, int kernel_id) {
  double gx[64], gw[64];
  orc_gauss_legendre01(n, gx, gw);
  double p1[3], p2[3], q1[3], q2[3];
  for (int k = 0; k < 3; ++k) {
    p1[k] = P[3 + k] - P[k];
    p2[k] = P[6 + k] - P[3 + k];
    q1[k] = Q[3 + k] - Q[k];
    q2[k] = Q[6 + k] - Q[3 + k];
  }
  double aT = tri_area(P), aS = tri_area(Q);
  double sum = 0.0;
  for (int reg = 0; reg < 2; ++reg)
    for (int i0 = 0; i0 < n; ++i0)
      for (int i1 = 0; i1 < n; ++i1)
        for (int i2 = 0; i2 < n; ++i2)
          for (int i3 = 0; i3 < n; ++i3) {
            double xi = gx[i0], a1 = gx[i1], a2 = gx[i2], a3 = gx[i3];
            double wq = gw[i0] * gw[i1] * gw[i2] * gw[i3];
            double s1, s2, t1, t2;
            if (reg == 0) { s1 = xi; s2 = xi * a1; t1 = xi * a2; t2 = xi * a2 * a3; }
            else { t1 = xi; t2 = xi * a1; s1 = xi * a2; s2 = xi * a2 * a3; }
            double x[3], y[3], d[3];
            for (int k = 0; k < 3; ++k) {
              double xr = s1 * p1[k] + s2 * p2[k];
              double yr = t1 * q1[k] + t2 * q2[k];
              x[k] = P[k] + xr;
              y[k] = Q[k] + yr;
              d[k] = xr - yr;
            }
            double jac = xi * xi * xi * a2;
            sum += wq * jac * kern(kernel_id, x, y, d);
          }
  return 4.0 * aT * aS * sum;
}

/* ----------------------------------------------------------------------- */
/* Pair dispatch with the canonical local orderings (the singular rules are  */
/* not symmetric under relabelling, so both codes fix the same labels):     */
/*   the triangle with the smaller index is T; V[T',T] := V[T,T'];           */
/*   identical:  (v0,v1,v2) as stored;                                       */
/*   edge:       A = smaller shared vertex id, B = larger, C/D the others;  */
/*   vertex:     O shared, then the cyclic successors of O in each triangle. */
/* Returns the class in *cls: 0 separated, 1 vertex, 2 edge, 3 identical.   */
/* ----------------------------------------------------------------------- */
static void load_tri(const double* xyz, const int32_t* t, int a, int b, int c, double* P) {
  int id[3] = {t[a], t[b], t[c]};
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) P[3 * i + k] = xyz[3 * (int64_t)id[i] + k];
}

double orc_pair(const double* xyz, const int32_t* tri, int64_t T, int64_t S, int far_order,
                int ss_order, int kernel_id, int* cls) {
  if (S < T) { int64_t tmp = T; T = S; S = tmp; }
  const int32_t* a = tri + 3 * T;
  const int32_t* b = tri + 3 * S;
  double P[9], Q[9];
  int shared = 0, ia[3], ib[3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (a[i] == b[j]) { ia[shared] = i; ib[shared] = j; ++shared; }
  if (cls) *cls = shared;
  if (T == S) {
    load_tri(xyz, a, 0, 1, 2, P);
    return orc_rule_identical(P, ss_order, kernel_id);
  }
  if (shared == 0) {
    load_tri(xyz, a, 0, 1, 2, P);
    load_tri(xyz, b, 0, 1, 2, Q);
    return orc_rule_far(P, Q, kernel_id, far_order);
  }
  if (shared == 1) {
    load_tri(xyz, a, ia[0], (ia[0] + 1) % 3, (ia[0] + 2) % 3, P);
    load_tri(xyz, b, ib[0], (ib[0] + 1) % 3, (ib[0] + 2) % 3, Q);
    return orc_rule_vertex(P, Q, ss_order, kernel_id);
  }
  if (shared == 2) {
    int iA = ia[0], iB = ia[1], jA = ib[0], jB = ib[1];
    if (a[iA] > a[iB]) { int t = iA; iA = iB; iB = t; t = jA; jA = jB; jB = t; }
    int iC = 3 - iA - iB, jD = 3 - jA - jB;
    load_tri(xyz, a, iA, iB, iC, P);
    load_tri(xyz, b, jA, jB, jD, Q);
    return orc_rule_edge(P, Q, ss_order, kernel_id);
  }
  /* two distinct triangles with the same three vertices: not a mesh */
  if (cls) *cls = -1;
  return NAN;
}

/* Dense V (row-major nt x nt).  OpenMP over rows only. */
void orc_assemble_V(int64_t nt, const double* xyz, const int32_t* tri, int far_order, int ss_order,
                    double* V) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t T = 0; T < nt; ++T) {
    for (int64_t S = T; S < nt; ++S) {
      double v = orc_pair(xyz, tri, T, S, far_order, ss_order, 0, NULL);
      V[T * nt + S] = v;
      V[S * nt + T] = v;
    }
  }
}

/* Selected entries of V (for sampled parity at sizes where V is too big). */
void orc_V_entries(int64_t m, const int64_t* rows, const int64_t* cols, const double* xyz,
                   const int32_t* tri, int far_order, int ss_order, double* out) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < m; ++i)
    out[i] = orc_pair(xyz, tri, rows[i], cols[i], far_order, ss_order, 0, NULL);
}

/* Kernel-selectable single pair, for the tests that pin the rules. */
double orc_pair_kernel(const double* xyz, const int32_t* tri, int64_t T, int64_t S, int far_order,
                       int ss_order, int kernel_id) {
  int cls;
  return orc_pair(xyz, tri, T, S, far_order, ss_order, kernel_id, &cls);
}

int orc_version(void) { return 1; }
