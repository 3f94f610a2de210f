"""Oracle solver: Galerkin system, preconditioner and PCG (test infrastructure only).

Plain dense FP64 linear algebra (numpy / scipy), following the paper:

* W[nu,nu'] = a(psi~_nu, psi~_nu') = sum_{T,T'} V[T,T'] s_{T,nu} . s_{T',nu'},
  i.e. W = sum_k S_k^T V S_k (Cor. corW with eq. eval_a_phiij, Sec. 3.4/4.3);
* L_nu = l_g(psi~_nu) = sum_t int_t g . n_t psi^t_nu = sum_T (c_+ - c_-) (g . n_T) |T| / 3
  for a constant g (Sec. 4.3, last display);
* M(H;h) r = sum_F R_F^T A_F^{-1} R_F r + R_W^T A_W^{-1} R_W r + P A_H^{-1} P^T r,
  the additive Schwarz operator of the splitting (eq. jumpSplit), every subspace
  solve exact (Remark "Bound on the number of PCG iterations", Sec. 2.1);
* preconditioned conjugate gradients from a zero initial guess; the stopping
  test is ||L - W Phi_k||_2 / ||L||_2 <= rtol on the recursively updated
  residual; the Lanczos tridiagonal of the PCG coefficients gives the
  condition number estimate of M W.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from . import core
from .topology import Topology, classify_dofs, prolongation


def assemble_W(top: Topology, V: np.ndarray) -> np.ndarray:
    """W = sum_k S_k^T V S_k with the dense pair matrix V."""
    W = np.zeros((top.ndof, top.ndof))
    for Sk in top.S_matrices():
        SkT = Sk.T.tocsr()
        Y = np.asarray(SkT @ V)          # S_k^T V            (ndof x nt)
        W += np.asarray(SkT @ Y.T).T     # (S_k^T (S_k^T V)^T)^T = S_k^T V S_k  (V symmetric)
    return W


def W_entries(top: Topology, rows, cols, far_order=0, ss_order=5) -> np.ndarray:
    """Selected entries of W computed one by one from their defining double
    sum over triangle pairs (for sampled parity on large meshes)."""
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    s = top.curl_vectors()
    starts = np.searchsorted(top.s_dof, np.arange(top.ndof + 1))
    pr, pc, coef = [], [], []
    owner = []
    for m, (i, j) in enumerate(zip(rows, cols)):
        for a in range(starts[i], starts[i + 1]):
            for b in range(starts[j], starts[j + 1]):
                pr.append(top.s_tri[a])
                pc.append(top.s_tri[b])
                coef.append(float(np.dot(s[a], s[b])))
                owner.append(m)
    v = core.V_entries(top.xyz, top.tri.astype(np.int32), np.array(pr), np.array(pc), far_order,
                       ss_order)
    out = np.zeros(rows.shape[0])
    np.add.at(out, np.array(owner, np.int64), v * np.array(coef))
    return out


def rhs(top: Topology, g) -> np.ndarray:
    """L_nu = sum_T (c_+ - c_-) (g . n_T) |T| / 3 for constant Neumann data g."""
    g = np.asarray(g, float)
    gn = top.normal @ g
    L = np.zeros(top.ndof)
    np.add.at(L, top.s_dof, top.s_coef * gn[top.s_tri] * top.area[top.s_tri] / 3.0)
    return L


@dataclasses.dataclass
class Preconditioner:
    blocks: list           # list of (dof index array, cho_factor)
    P: object              # sparse N x N_H prolongation
    AH: object             # cho_factor of P^T W P (or None)
    cls: np.ndarray        # class per dof: patch id or -1 (wire basket)

    def apply(self, r: np.ndarray) -> np.ndarray:
        z = np.zeros_like(r)
        for idx, fac in self.blocks:
            z[idx] += sla.cho_solve(fac, r[idx])
        if self.AH is not None:
            z += self.P @ sla.cho_solve(self.AH, self.P.T @ r)
        return z


def build_preconditioner(top: Topology, W: np.ndarray, coarse: Topology | None, parent, patch,
                         wire_basket: str = "exact") -> Preconditioner:
    cls = classify_dofs(top, patch)
    blocks = []
    for p in sorted(set(int(c) for c in cls)):
        idx = np.nonzero(cls == p)[0]
        A = W[np.ix_(idx, idx)]
        if p == -1 and wire_basket == "diagonal":
            # approximate wire-basket solver: pointwise scalar product scaled by diag(W)
            blocks.append((idx, (np.diag(np.sqrt(np.diag(A))), False)))
            continue
        blocks.append((idx, sla.cho_factor(A, lower=True)))
    P, AH = None, None
    if coarse is not None and coarse.ndof > 0:
        P = prolongation(top, coarse, parent)
        A_H = P.T @ (W @ P.toarray())
        AH = sla.cho_factor(np.asarray(A_H), lower=True)
    return Preconditioner(blocks, P, AH, cls)


@dataclasses.dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    hist: list
    alphas: list
    betas: list
    converged: bool

    @property
    def kappa(self) -> float:
        return lanczos_kappa(self.alphas, self.betas)


def pcg(W: np.ndarray, L: np.ndarray, M=None, rtol: float = 1e-8, maxit: int = 1000,
        fixed: bool = False) -> PCGResult:
    """Preconditioned CG from Phi_0 = 0 (fixed=True runs exactly maxit steps)."""
    n = L.shape[0]
    x = np.zeros(n)
    r = L.copy()
    nL = float(np.linalg.norm(L))
    if nL == 0.0:
        return PCGResult(x, 0, [0.0], [], [], True)
    z = M(r) if M is not None else r.copy()
    p = z.copy()
    rz = float(r @ z)
    hist = [1.0]
    alphas, betas = [], []
    it = 0
    conv = False
    for k in range(maxit):
        q = W @ p
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        rel = float(np.linalg.norm(r)) / nL
        hist.append(rel)
        alphas.append(alpha)
        it = k + 1
        if rel <= rtol:
            conv = True
            if not fixed:
                break
        if it == maxit:
            break
        z = M(r) if M is not None else r.copy()
        rz_new = float(r @ z)
        beta = rz_new / rz
        betas.append(beta)
        rz = rz_new
        p = z + beta * p
    return PCGResult(x, it, hist, alphas, betas, conv)


def lanczos_kappa(alphas, betas) -> float:
    """Condition number of the Lanczos tridiagonal built from PCG coefficients:
    diagonal 1/alpha_0, 1/alpha_j + beta_{j-1}/alpha_{j-1}; off-diagonal
    sqrt(beta_j)/alpha_j."""
    m = len(alphas)
    if m == 0:
        return float("nan")
    d = np.zeros(m)
    e = np.zeros(max(m - 1, 0))
    for j in range(m):
        d[j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j < m - 1:
            e[j] = np.sqrt(betas[j]) / alphas[j]
    ev = sla.eigvalsh_tridiagonal(d, e) if m > 1 else d
    return float(ev.max() / ev.min())


def augment_cells(top: Topology, W: np.ndarray):
    """A screen enclosing cells has the cells' indicators in the kernel of W
    (their jumps are constant on every triangle, so their surface curls
    vanish).  Reading of the paper's connectedness assumption: solve with
    W + rho Q Q^T, rho the mean of diag(W) and Q = Z L^-T (Z^T Z = L L^T) an
    orthonormal basis of the span of the indicators' psi-coordinates Z
    (Topology.cells): rho times the orthogonal projector onto the kernel, so
    the kernel directions take the eigenvalue rho, inside the spectrum of W.
    For constant g, Z^T L = 0, and the solution is the one with Z^T Phi = 0.
    Returns (W, Z, rho, Q); W unchanged."""
    Z = top.cells()
    rho = float(np.mean(np.diag(W))) if W.size else 0.0
    Q = Z
    if Z.shape[1]:
        Lc = np.linalg.cholesky(Z.T @ Z)
        Q = sla.solve_triangular(Lc, Z.T, lower=True).T
    return W, Z, rho, Q


class Problem:
    """Everything the oracle knows about one geometry."""

    def __init__(self, geom, far_order: int = 0, ss_order: int = 5, with_coarse: bool = True,
                 assemble: bool = True):
        self.geom = geom
        self.top = Topology(geom.xyz, geom.tri)
        self.coarse = Topology(geom.coarse_xyz, geom.coarse_tri) if with_coarse else None
        self.far_order, self.ss_order = far_order, ss_order
        self.V = None
        self.W = None
        self.M = None
        if assemble:
            self.assemble()

    @property
    def ndof(self) -> int:
        return self.top.ndof

    def assemble(self):
        self.V = core.assemble_V(self.geom.xyz, self.geom.tri, self.far_order, self.ss_order)
        self.W = assemble_W(self.top, self.V)
        self.W0, self.Z, self.rho, self.Q = augment_cells(self.top, self.W)
        if self.Z.shape[1]:
            self.W = self.W0 + self.rho * (self.Q @ self.Q.T)
        return self.W

    def rhs(self, g=None) -> np.ndarray:
        return rhs(self.top, self.geom.g if g is None else g)

    def factor(self, wire_basket: str = "exact"):
        self.M = build_preconditioner(self.top, self.W, self.coarse, self.geom.parent,
                                      self.geom.patch, wire_basket)
        return self.M

    def solve(self, g=None, rtol=1e-8, maxit=1000, fixed=False, precondition=True) -> PCGResult:
        if precondition and self.M is None:
            self.factor()
        L = self.rhs(g)
        return pcg(self.W, L, self.M.apply if precondition else None, rtol, maxit, fixed)

    def direct(self, g=None) -> np.ndarray:
        L = self.rhs(g)
        return sla.cho_solve(sla.cho_factor(self.W, lower=True), L)
