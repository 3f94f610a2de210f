"""Double-layer potential of a computed jump (test infrastructure only).

Lemma lemrepDL (eq. formulaDL): for x off the screen,

    DL u (x) = sum over oriented triangles t of
               int_t  n_t . (y - x) / (4 pi |x - y|^3)  gamma_t u(y)  dsigma(y).

For u = sum_nu Phi_nu psi_nu the trace on t = (T, +/-) is sum_a c_{+/-}(a) Phi
lambda_a and n_(T,-) = -n_T, so the two sides of T combine into the jump
J_{T,a} = sum_nu Phi_nu (c_+ - c_-)(T, a, nu):

    U(x) = sum_T sum_a J_{T,a} int_T n_T . (y - x) lambda_a(y) / (4 pi |x-y|^3) dy.

Each triangle is integrated with the 6-point degree-4 rule, optionally on its
4^refine congruent sub-triangles (uniform midpoint subdivision), for targets
close to the screen.  Plain FP64 numpy; nothing here is shared with the CUDA
path.
"""
from __future__ import annotations

import numpy as np

from . import core
from .topology import Topology


def jump_values(top: Topology, phi) -> np.ndarray:
    """J[T, a] = sum_nu Phi_nu (c_+ - c_-)(T, a, nu), summed in curl-list order."""
    J = np.zeros((top.nt, 3))
    np.add.at(J, (top.s_tri, top.s_loc), np.asarray(phi, float)[top.s_dof] * top.s_coef)
    return J


def _reference_subtriangles(refine: int):
    """Barycentric corners of the 4^refine sub-triangles of the reference
    triangle (uniform subdivision into m^2 = 4^refine similar triangles)."""
    m = 2 ** refine
    out = []
    for j in range(m):
        for i in range(m - j):
            def B(a, b):
                return np.array([1.0 - (a + b) / m, a / m, b / m])
            out.append((B(i, j), B(i + 1, j), B(i, j + 1)))
            if i + j + 1 < m:
                out.append((B(i + 1, j), B(i + 1, j + 1), B(i, j + 1)))
    return out


def dl_potential(top: Topology, phi, targets, refine: int = 0, chunk: int = 64) -> np.ndarray:
    bary, w = core.dunavant6()                      # weights sum to 1
    J = jump_values(top, phi)
    X = top.xyz[top.tri]                            # [nt, 3, 3]
    subs = _reference_subtriangles(refine)
    pts, chg = [], []
    for (B0, B1, B2) in subs:
        for p in range(6):
            beta = bary[p, 0] * B0 + bary[p, 1] * B1 + bary[p, 2] * B2       # barycentrics in T
            pts.append(np.einsum("a,tak->tk", beta, X))
            chg.append(w[p] * top.area / len(subs) * (J @ beta))
    P = np.stack(pts, axis=1)                       # [nt, q, 3]
    C = np.stack(chg, axis=1)                       # [nt, q]
    nrm = top.normal
    targets = np.atleast_2d(np.asarray(targets, float))
    out = np.zeros(targets.shape[0])
    for s in range(0, targets.shape[0], chunk):
        x = targets[s:s + chunk]
        d = P[None] - x[:, None, None, :]           # y - x
        r2 = np.einsum("mtqk,mtqk->mtq", d, d)
        nd = np.einsum("mtqk,tk->mtq", d, nrm)
        out[s:s + chunk] = np.einsum("mtq,tq->m", nd / (4.0 * np.pi * r2 * np.sqrt(r2)), C)
    return out
