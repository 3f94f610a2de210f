"""Pins for the oracle's Galerkin system, preconditioner and PCG (CPU only).

Fixed by mathematics, not by the oracle:
* W symmetric positive definite (Thm. lemequivInner, Sec. 3.3);
* invariance under rigid motions of the mesh together with g;
* Galerkin energy L^T Phi symmetric under the book's 120-degree rotation;
* PCG reproduces a dense Cholesky solve; its Lanczos estimate equals the
  dense generalized eigenvalues; its error obeys the bound of the Remark on
  PCG iterations (Sec. 2.1); the preconditioned condition number grows no
  faster than (1 + log H/h)^2 (Thm. main) while the plain one grows like 1/h;
* the coarse space is the jump space of the coarse mesh: P^T W_h P equals the
  coarse Galerkin matrix up to quadrature error.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import solver
from oracle.topology import classify_dofs
from paper_2310_09204_gb300 import workloads as WL

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "invariants.json")))


@pytest.fixture(scope="module")
def flat():
    pb = solver.Problem(WL.flat_config())
    pb.factor()
    return pb


@pytest.fixture(scope="module")
def book8():
    pb = solver.Problem(WL.book(8, 2, jitter=True, seed=1))
    pb.factor()
    return pb


def test_W_symmetric_positive_definite(flat, book8):
    for pb in (flat, book8):
        W = pb.W
        assert np.abs(W - W.T).max() <= 1e-15 * np.abs(W).max()
        assert np.linalg.eigvalsh(W).min() > 0


def test_flat_classes(flat):
    cls = flat.M.cls
    gold = GOLDEN["flat_square_h1_16_classes"]["value"]
    assert int((cls == -1).sum()) == gold["wire_basket"]
    for p in range(4):
        assert int((cls == p).sum()) == gold["face_per_patch"]
    assert flat.coarse.ndof == gold["coarse"]


def test_rigid_motion_invariance(book8):
    th = 0.7
    R = np.array([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]])
    R = R @ np.array([[1, 0, 0], [0, math.cos(0.3), -math.sin(0.3)], [0, math.sin(0.3), math.cos(0.3)]])
    g2 = WL.rotate(book8.geom, R, shift=(0.3, -2.0, 1.1))
    pb2 = solver.Problem(g2)
    assert np.abs(pb2.W - book8.W).max() <= 1e-12 * np.abs(book8.W).max()
    assert np.abs(pb2.rhs() - book8.rhs()).max() <= 1e-13 * np.abs(book8.rhs()).max()


def test_book_symmetries(book8):
    # g along the spine: g . n = 0 on every page
    assert np.abs(book8.rhs(np.array([0.0, 0.0, 1.0]))).max() < 1e-15
    # energy is invariant under a 120-degree rotation of g about the spine
    c, s = math.cos(2 * math.pi / 3), math.sin(2 * math.pi / 3)
    R = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
    g = np.array([1.0, 0.5, 0.25])
    Wf = sla.cho_factor(book8.W)
    e = [float(book8.rhs(v) @ sla.cho_solve(Wf, book8.rhs(v))) for v in (g, R @ g, R @ R @ g)]
    assert max(e) - min(e) < 1e-12 * max(e)


def test_pcg_matches_direct_solve(flat, book8):
    for pb in (flat, book8):
        x = pb.direct()
        r = pb.solve(rtol=1e-12)
        assert r.converged
        assert np.linalg.norm(r.x - x) <= 1e-10 * np.linalg.norm(x)
        # final recursive residual is the true residual
        res = np.linalg.norm(pb.rhs() - pb.W @ r.x) / np.linalg.norm(pb.rhs())
        assert abs(res - r.hist[-1]) < 1e-12


def _dense_kappa(pb):
    n = pb.ndof
    M = np.stack([pb.M.apply(e) for e in np.eye(n)], axis=1)
    ev = sla.eigh(pb.W, np.linalg.inv(M), eigvals_only=True)
    return float(ev.max() / ev.min()), ev


def test_lanczos_estimate_equals_dense_spectrum(flat):
    # a generic right-hand side (the flat workload's own is symmetric and
    # leaves part of the spectrum outside its Krylov space)
    kd, _ = _dense_kappa(flat)
    L = np.random.default_rng(0).normal(size=flat.ndof)
    r = solver.pcg(flat.W, L, flat.M.apply, rtol=1e-14, maxit=500)
    assert abs(r.kappa - kd) <= 1e-3 * kd


def test_pcg_error_bound(flat):
    """a(e_n,e_n)^(1/2) <= 2 rho^n a(e_0,e_0)^(1/2), rho = (sqrt k - 1)/(sqrt k + 1)."""
    kd, _ = _dense_kappa(flat)
    rho = (math.sqrt(kd) - 1) / (math.sqrt(kd) + 1)
    x = flat.direct()
    W, L = flat.W, flat.rhs()
    e0 = math.sqrt(x @ W @ x)
    for n in range(1, 9):
        r = solver.pcg(W, L, flat.M.apply, rtol=0.0, maxit=n, fixed=True)
        e = r.x - x
        assert math.sqrt(e @ W @ e) <= 2 * rho ** n * e0 * (1 + 1e-9)


@pytest.mark.slow
def test_condition_number_growth_thm_main():
    """Face spaces = coarse triangles (Sec. 5), H = 1/2, h = H/4 ... H/16."""
    kp, kw = [], []
    for n in (8, 16, 32):
        pb = solver.Problem(WL.unit_square(n, 2, "coarse_tri"))
        pb.factor()
        kp.append(_dense_kappa(pb)[0])
        ev = np.linalg.eigvalsh(pb.W)
        kw.append(ev.max() / ev.min())
    ratio = [k / (1 + math.log(n / 2)) ** 2 for k, n in zip(kp, (8, 16, 32))]
    assert ratio[0] >= ratio[1] >= ratio[2]
    assert kp[0] < kp[1] < kp[2] < 6.0
    for a, b in zip(kw, kw[1:]):
        assert 1.7 < b / a < 2.3          # O(1/h) without preconditioner


@pytest.mark.parametrize("geom", [WL.unit_square(4, 2), WL.bowtie(4, 2), WL.book(4, 2, jitter=False)],
                         ids=lambda g: g.name)
def test_coarse_space_is_coarse_jump_space(geom):
    """P^T W_h P is the coarse Galerkin matrix: both approximate the same
    a(psi^H, psi^H); with accurate quadrature they agree to its error."""
    fine = solver.Problem(geom, far_order=10, ss_order=10)
    pb = solver.build_preconditioner(fine.top, fine.W, fine.coarse, geom.parent, geom.patch)
    AH = pb.P.T @ (fine.W @ pb.P.toarray())
    from paper_2310_09204_gb300.workloads import Geometry
    cg = Geometry("coarse", geom.coarse_xyz, geom.coarse_tri, geom.coarse_xyz, geom.coarse_tri,
                  np.arange(geom.coarse_tri.shape[0], dtype=np.int32),
                  np.zeros(geom.coarse_tri.shape[0], np.int32), geom.g, geom.H, geom.H)
    coarse = solver.Problem(cg, far_order=10, ss_order=10, with_coarse=False)
    assert coarse.ndof == AH.shape[0] > 0
    assert np.abs(AH - coarse.W).max() <= 2e-5 * np.abs(coarse.W).max()


def test_wire_basket_contains_junctions(book8):
    cls = classify_dofs(book8.top, book8.geom.patch)
    spine = (np.abs(book8.geom.xyz[:, 0]) < 1e-12) & (np.abs(book8.geom.xyz[:, 1]) < 1e-12)
    assert np.all(cls[spine[book8.top.dof_vertex]] == -1)
