"""Closed-form integrals of 1/|x - y| over flat triangles and segments.

Derived for the tests from Euler's identity for homogeneous functions (they
pin the oracle's quadrature and share nothing with it):

* potential of a uniform triangle T = ABC at its vertex A: polar coordinates
  about A give  u(A) = h_A [asinh(s_C/h_A) - asinh(s_B/h_A)],  with h_A the
  distance from A to line BC and s_B, s_C the positions of B, C along BC
  measured from the foot of the perpendicular;
* E(O; P, Q) = int_{OP} int_{OQ} 1/|x-y|: the integral is homogeneous of degree
  1 in the two lengths, so E = |OP| int_{OQ} dt/|P - y| + |OQ| int_{OP} ds/|x - Q|,
  each a closed-form asinh difference;
* G(T, BC) = int_{BC} int_T 1/|x-y|: scaling about B (degree 2) gives
  2 G = |BC| u(C) + h_B E(C; B, A);
* F(T) = int_T int_T 1/|x-y|: scaling about A (degree 3) gives
  3 F = 2 h_A G(T, BC).

Edge- and vertex-adjacent coplanar pairs follow by subtraction: splitting ABC
at a point M of BC gives V(ABM, AMC) = (F(ABC) - F(ABM) - F(AMC)) / 2, and a
three-triangle fan gives the vertex-adjacent pair.
"""
import math

import numpy as np


def _dist_to_line(P, A, B):
    t = (B - A) / np.linalg.norm(B - A)
    d = P - A
    return float(np.linalg.norm(d - np.dot(d, t) * t))


def potential_at_vertex(A, B, C) -> float:
    BC = C - B
    t = BC / np.linalg.norm(BC)
    F = B + np.dot(A - B, t) * t
    h = float(np.linalg.norm(A - F))
    sB = float(np.dot(B - F, t))
    sC = float(np.dot(C - F, t))
    return h * (math.asinh(sC / h) - math.asinh(sB / h))


def segments_sharing_vertex(O, P, Q) -> float:
    l1 = float(np.linalg.norm(P - O))
    l2 = float(np.linalg.norm(Q - O))
    cb = float(np.dot(P - O, Q - O)) / (l1 * l2)
    sb = math.sqrt(max(0.0, 1.0 - cb * cb))
    phi1 = math.asinh((l2 - l1 * cb) / (l1 * sb)) - math.asinh(-cb / sb)
    phi2 = math.asinh((l1 - l2 * cb) / (l2 * sb)) - math.asinh(-cb / sb)
    return l1 * phi1 + l2 * phi2


def self_integral(A, B, C) -> float:
    """int_T int_T 1/|x - y| dx dy for the triangle ABC."""
    A, B, C = (np.asarray(x, float) for x in (A, B, C))
    G = 0.5 * (float(np.linalg.norm(C - B)) * potential_at_vertex(C, A, B)
               + _dist_to_line(B, C, A) * segments_sharing_vertex(C, B, A))
    return (2.0 / 3.0) * _dist_to_line(A, B, C) * G


def V_identical(P) -> float:
    return self_integral(*P) / (4.0 * math.pi)


def V_edge_split(A, B, C, t=0.5):
    """(T1, T2, V) with T1 = (A, M, B), T2 = (A, M, C), M = B + t (C - B)."""
    A, B, C = (np.asarray(x, float) for x in (A, B, C))
    M = B + t * (C - B)
    v = (self_integral(A, B, C) - self_integral(A, B, M) - self_integral(A, M, C)) / 2.0
    return np.array([A, M, B]), np.array([A, M, C]), v / (4.0 * math.pi)


def V_vertex_fan(A, B, C, t1=0.3, t2=0.7):
    """(T1, T3, V): fan of ABC from A through M1, M2 on BC; T1 = (A, B, M1) and
    T3 = (A, M2, C) share only the vertex A."""
    A, B, C = (np.asarray(x, float) for x in (A, B, C))
    M1 = B + t1 * (C - B)
    M2 = B + t2 * (C - B)
    F = self_integral
    v12 = (F(A, B, M2) - F(A, B, M1) - F(A, M1, M2)) / 2.0
    v23 = (F(A, M1, C) - F(A, M1, M2) - F(A, M2, C)) / 2.0
    v13 = (F(A, B, C) - F(A, B, M1) - F(A, M1, M2) - F(A, M2, C)) / 2.0 - v12 - v23
    return np.array([A, B, M1]), np.array([A, M2, C]), v13 / (4.0 * math.pi)


def triangle_potential(T, r) -> float:
    """u(r) = int_T dS'/|r - r'| for a flat triangle T (3 x 3 vertices) and any
    point r outside T or at one of its vertices: the edge-by-edge closed form of Wilton et al. (IEEE Trans.
    Antennas Propag. 32, 1984), restated.  With n the unit normal, d the height
    of r over the plane and rho its foot, each edge (a, b) with unit tangent t
    and in-plane outward normal m contributes
        P0 ln((R+ + l+) / (R- + l-)) - |d| [atan(P0 l+ / (R0^2 + |d| R+))
                                          - atan(P0 l- / (R0^2 + |d| R-))],
    P0 = (a - rho).m, l-/+ = (a/b - rho).t, R0^2 = P0^2 + d^2, R-/+ = |r - a/b|."""
    T = np.asarray(T, float)
    r = np.asarray(r, float)
    n = np.cross(T[1] - T[0], T[2] - T[0])
    n /= np.linalg.norm(n)
    d = float(np.dot(r - T[0], n))
    rho = r - d * n
    c = T.mean(axis=0)
    ad = abs(d)
    u = 0.0
    for i in range(3):
        a, b = T[i], T[(i + 1) % 3]
        t = (b - a) / np.linalg.norm(b - a)
        m = np.cross(t, n)
        if np.dot(c - a, m) > 0:          # outward from the triangle
            m = -m
        P0 = float(np.dot(a - rho, m))
        lm, lp = float(np.dot(a - rho, t)), float(np.dot(b - rho, t))
        R0s = P0 * P0 + d * d
        Rm, Rp = float(np.linalg.norm(r - a)), float(np.linalg.norm(r - b))
        if abs(P0) > 1e-14 * (Rm + Rp):   # r on the edge's line: no log term
            u += P0 * math.log((Rp + lp) / (Rm + lm))
        u -= ad * (math.atan2(P0 * lp, R0s + ad * Rp) - math.atan2(P0 * lm, R0s + ad * Rm))
    return u


def collapsed_gauss(T, f, n: int = 24) -> float:
    """int_T f dS by the n x n Gauss-Legendre rule on the square collapsed onto
    T (x = A + s (B - A) + t (1 - s) (C - A), Jacobian 2|T| (1 - s)); for
    smooth f."""
    T = np.asarray(T, float)
    x, w = np.polynomial.legendre.leggauss(n)
    x, w = 0.5 * (x + 1.0), 0.5 * w
    area2 = float(np.linalg.norm(np.cross(T[1] - T[0], T[2] - T[0])))
    tot = 0.0
    for i in range(n):
        for j in range(n):
            p = T[0] + x[i] * (T[1] - T[0]) + x[j] * (1.0 - x[i]) * (T[2] - T[0])
            tot += w[i] * w[j] * (1.0 - x[i]) * f(p)
    return area2 * tot


def V_separated(P, Q, n: int = 24) -> float:
    """V_PQ = int_P int_Q 1/(4 pi |x - y|) for triangles that share no point:
    the closed-form inner potential over P, integrated over Q."""
    return collapsed_gauss(Q, lambda y: triangle_potential(P, y), n) / (4.0 * math.pi)
