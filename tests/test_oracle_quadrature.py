"""Pins for the oracle's quadrature (CPU only).

What fixes the expected values here is not the oracle:
* numpy's Gauss-Legendre routine and exact monomial integrals;
* closed forms of int int 1/|x-y| derived in tests/closed_forms.py;
* exactness of a product rule for polynomial integrands;
* an independent hierarchical-subdivision evaluation of singular pairs.
"""
import math

import numpy as np
import pytest

from oracle import core
from tests import closed_forms as cf


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 20])
def test_gauss_legendre_matches_numpy(n):
    x, w = core.gauss_legendre01(n)
    t, wt = np.polynomial.legendre.leggauss(n)
    order = np.argsort(0.5 * (1 - t))
    np.testing.assert_allclose(x, 0.5 * (1 - t)[order], rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, 0.5 * wt[order], rtol=0, atol=2e-15)
    for k in range(2 * n):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 5e-15


def _monomial_exact(a, b, c, area):
    # int_T l1^a l2^b l3^c = 2 |T| a! b! c! / (a+b+c+2)!
    return 2 * area * math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 2)


def test_six_point_rule_degree_four():
    bary, w = core.dunavant6()
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.all(bary > 0) and np.allclose(bary.sum(axis=1), 1.0, atol=1e-15)
    for deg in range(0, 7):
        worst = 0.0
        for a in range(deg + 1):
            for b in range(deg + 1 - a):
                c = deg - a - b
                approx = float(np.dot(w, bary[:, 0] ** a * bary[:, 1] ** b * bary[:, 2] ** c))
                worst = max(worst, abs(approx - _monomial_exact(a, b, c, 0.5) / 0.5))
        if deg <= 4:
            assert worst < 1e-15, (deg, worst)
        else:
            assert worst > 1e-6, (deg, worst)   # the rule is degree 4, not more


def _random_pair(rng, kind):
    O = rng.normal(size=3)
    if kind == "identical":
        return rng.normal(size=(3, 3)) * 0.7 + O, None
    if kind == "edge":
        A, B = O, O + rng.normal(size=3)
        C = A + rng.normal(size=3)
        D = A + rng.normal(size=3)
        return np.array([A, B, C]), np.array([A, B, D])
    P1, P2, Q1, Q2 = (O + rng.normal(size=3) for _ in range(4))
    return np.array([O, P1, P2]), np.array([O, Q1, Q2])


@pytest.mark.parametrize("kind", ["identical", "edge", "vertex"])
@pytest.mark.parametrize("kernel", [1, 2, 3, 4])
def test_singular_maps_exact_for_polynomials(kind, kernel):
    """The regularising maps must integrate polynomial kernels exactly: compare
    with the 6x6 product rule, exact for degree <= 4 in each point."""
    rng = np.random.default_rng(7 + kernel)
    for _ in range(3):
        P, Q = _random_pair(rng, kind)
        if kind == "identical":
            got = core.rule_identical(P, 5, kernel)
            ref = core.rule_far(P, P, kernel, 0)
        elif kind == "edge":
            got = core.rule_edge(P, Q, 5, kernel)
            ref = core.rule_far(P, Q, kernel, 0)
        else:
            got = core.rule_vertex(P, Q, 5, kernel)
            ref = core.rule_far(P, Q, kernel, 0)
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (got, ref)


MESH_TRIANGLES = [
    np.array([[0, 0, 0], [1 / 16, 0, 0], [1 / 16, 1 / 16, 0]], float),        # right isosceles (grid)
    np.array([[0, 0, 0], [1, 0, 0], [0.5, math.sqrt(3) / 2, 0]], float),       # equilateral
    np.array([[0.2, 0.1, 0.3], [0.9, 0.2, 0.1], [0.4, 0.8, 0.6]], float),       # general, tilted
]


@pytest.mark.parametrize("P", MESH_TRIANGLES)
def test_identical_rule_converges_to_closed_form(P):
    exact = cf.V_identical(P)
    errs = [abs(core.rule_identical(P, n) - exact) / exact for n in (5, 8, 12, 16)]
    assert errs[-1] < 1e-12
    assert errs[0] < 2e-3                      # the default order-5 rule
    assert errs[2] <= errs[0]


@pytest.mark.parametrize("t", [0.5, 0.3])
def test_edge_rule_converges_to_closed_form(t):
    A, B, C = np.array([0., 0, 0]), np.array([1.0, 0.1, 0]), np.array([0.3, 0.9, 0])
    T1, T2, exact = cf.V_edge_split(A, B, C, t)
    errs = [abs(core.rule_edge(T1, T2, n) - exact) / exact for n in (5, 8, 16, 24)]
    assert errs[0] < 1e-4 and errs[1] < 1e-6 and errs[2] < 1e-10 and errs[3] < 1e-12


def test_vertex_rule_converges_to_closed_form():
    A, B, C = np.array([0., 0, 0]), np.array([1.0, 0.1, 0]), np.array([0.3, 0.9, 0])
    T1, T3, exact = cf.V_vertex_fan(A, B, C)
    errs = [abs(core.rule_vertex(T1, T3, n) - exact) / exact for n in (5, 8, 16)]
    assert errs[0] < 1e-4 and errs[1] < 1e-7 and errs[2] < 1e-12


def _subdivide(P):
    A, B, C = P
    ab, bc, ca = (A + B) / 2, (B + C) / 2, (C + A) / 2
    return [np.array(x) for x in ([A, ab, ca], [ab, B, bc], [ca, bc, C], [ab, bc, ca])]


def _shared_vertices(P, Q):
    return sum(1 for p in P for q in Q if np.linalg.norm(p - q) < 1e-14)


def _brute(P, Q, depth, n_ss=10, n_far=8):
    """Hierarchical subdivision: children pairs that touch recurse, separated
    children use a high-order product rule."""
    total = 0.0
    for a in _subdivide(P):
        for b in _subdivide(Q):
            k = _shared_vertices(a, b)
            if k == 0:
                total += core.rule_far(a, b, 0, n_far)
            elif depth > 1:
                total += _brute(a, b, depth - 1, n_ss, n_far)
            else:
                if k == 3:
                    total += core.rule_identical(a, n_ss)
                elif k == 2:
                    sh = [p for p in a if any(np.linalg.norm(p - q) < 1e-14 for q in b)]
                    ra = [p for p in a if all(np.linalg.norm(p - s) > 1e-14 for s in sh)][0]
                    rb = [q for q in b if all(np.linalg.norm(q - s) > 1e-14 for s in sh)][0]
                    total += core.rule_edge(np.array([sh[0], sh[1], ra]), np.array([sh[0], sh[1], rb]), n_ss)
                else:
                    o = [p for p in a if any(np.linalg.norm(p - q) < 1e-14 for q in b)][0]
                    ra = [p for p in a if np.linalg.norm(p - o) > 1e-14]
                    rb = [q for q in b if np.linalg.norm(q - o) > 1e-14]
                    total += core.rule_vertex(np.array([o, ra[0], ra[1]]), np.array([o, rb[0], rb[1]]), n_ss)
    return total


@pytest.mark.parametrize("angle_deg", [90.0, 120.0, 45.0])
def test_nonplanar_edge_pair_against_subdivision(angle_deg):
    """Junction pairs (two panels meeting at an edge at a dihedral angle):
    the order-20 rule and a two-level subdivision agree."""
    th = math.radians(angle_deg)
    A, B = np.array([0., 0, 0]), np.array([0., 0, 1])
    C = np.array([0.8, 0.0, 0.4])
    D = np.array([0.8 * math.cos(th), 0.8 * math.sin(th), 0.6])
    P, Q = np.array([A, B, C]), np.array([A, B, D])
    hi = core.rule_edge(P, Q, 20)
    assert abs(core.rule_edge(P, Q, 24) - hi) < 1e-12 * hi
    ref = _brute(P, Q, 2)
    assert abs(hi - ref) < 2e-7 * hi, (hi, ref)
    assert abs(core.rule_edge(P, Q, 5) - hi) < 2e-4 * hi


def test_nonplanar_vertex_pair_against_subdivision():
    O = np.array([0., 0, 0])
    P = np.array([O, [1.0, 0, 0], [0.5, 0.8, 0]])
    Q = np.array([O, [0.0, -0.3, 0.9], [-0.6, 0.2, 0.7]])
    hi = core.rule_vertex(P, Q, 20)
    ref = _brute(P, Q, 2)
    assert abs(hi - ref) < 2e-7 * hi, (hi, ref)


def test_far_rule_symmetric_and_consistent():
    rng = np.random.default_rng(3)
    P = rng.normal(size=(3, 3))
    Q = P + np.array([8.0, 3.0, -5.0])
    a = core.rule_far(P, Q)
    b = core.rule_far(Q, P)
    assert abs(a - b) < 1e-15 * a
    # well separated: the 6-point product rule matches a high-order rule closely
    assert abs(a - core.rule_far(P, Q, 0, 12)) < 1e-6 * a


# --- separated pairs against the closed-form potential of a flat triangle ---

P_GEN = np.array([[0.2, 0.1, 0.3], [0.9, 0.2, 0.1], [0.4, 0.8, 0.6]])
Q_GEN = np.array([[0.0, 0.0, 0.0], [0.7, 0.3, 0.2], [0.1, 0.6, -0.4]])


def test_triangle_potential_two_derivations_agree():
    # at a vertex, in the plane: the edge formula against the polar one
    A, B, C = np.array([0., 0, 0]), np.array([1.0, 0.1, 0]), np.array([0.3, 0.9, 0])
    T = np.array([A, B, C])
    for v, (a, b, c) in ((A, (A, B, C)), (B, (B, C, A)), (C, (C, A, B))):
        assert abs(cf.triangle_potential(T, v) - cf.potential_at_vertex(a, b, c)) < 1e-14
    # off the plane, against a high-order rule of the smooth integrand
    for r in ([0.4, 0.3, 0.5], [2.4, -0.3, -0.2], [-0.5, 1.2, 0.3], [0.5, 0.4, -2.0]):
        r = np.array(r)
        ref = cf.collapsed_gauss(T, lambda x: 1.0 / np.linalg.norm(r - x), 60)
        assert abs(cf.triangle_potential(T, r) - ref) < 1e-13 * ref
    # far away it is the monopole area / distance
    r = np.array([300.0, 200.0, 400.0])
    area = 0.5 * np.linalg.norm(np.cross(B - A, C - A))
    mono = area / np.linalg.norm(r - T.mean(axis=0))
    assert abs(cf.triangle_potential(T, r) - mono) < 1e-5 * mono


def test_far_rule_against_exact_entries():
    """V for separated pairs: the oracle's high-order far rule equals the exact
    value, and its 6-point product rule (degree 4 on each triangle) errs like
    (diameter / distance)^6."""
    e6 = []
    for dist in (1.5, 3.0, 6.0, 12.0):
        Q = Q_GEN + np.array([dist, 0.3 * dist, -0.2 * dist])
        exact = cf.V_separated(P_GEN, Q)
        assert abs(core.rule_far(P_GEN, Q, 0, 12) - exact) < 1e-12 * exact
        e6.append(abs(core.rule_far(P_GEN, Q) - exact) / exact)
    assert e6[0] < 3e-5
    for a, b in zip(e6, e6[1:]):
        assert a / b > 32.0, e6


def test_oracle_entry_of_a_mesh_pair_is_the_exact_integral():
    # two triangles of the flat h = 1/16 screen, far apart: the oracle's pair
    # entry (classification, vertex order, areas) against the exact integral
    from paper_2310_09204_gb300 import workloads as WL
    geom = WL.flat_config()
    xyz, tri = geom.xyz, geom.tri
    cen = xyz[tri].mean(axis=1)
    T = 0
    S = int(np.argmax(np.linalg.norm(cen - cen[T], axis=1)))
    exact = cf.V_separated(xyz[tri[T]], xyz[tri[S]])
    assert abs(core.pair(xyz, tri, T, S, far_order=12) - exact) < 1e-12 * exact
    assert abs(core.pair(xyz, tri, T, S) - exact) < 1e-9 * exact
