"""The cube with its three mid-planes (eight closed cells): the library
assembles W + rho Z Z^T (closed-cell reading), and its solves are held to the
oracle's augmented system."""
import math

import numpy as np
import pytest

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import build as B
from paper_2310_09204_gb300 import workloads as WL
from oracle import solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _build():
    B.build()
    M.lib()


def _energy_rel(x, ref, W):
    e = x - ref
    return math.sqrt(max(e @ W @ e, 0.0)) / math.sqrt(ref @ W @ ref)


@pytest.mark.parametrize("n", [4, 6, 12])
def test_cube_against_oracle(n):
    geom = WL.cube_midplanes(n, 2 if n < 12 else 6)
    pb = solver.Problem(geom)
    pb.factor()
    with M.Solver(geom) as S:
        S.assemble()
        Z, rho = S.cells()
        assert Z.shape[1] == 8 and np.array_equal(Z, pb.Z)
        assert abs(rho - pb.rho) <= 1e-13 * pb.rho
        Wg = S.matrix()
        scale = np.abs(pb.W).max()
        assert np.abs(Wg - pb.W).max() <= 1e-12 * scale
        d = np.abs(np.diag(Wg) - np.diag(pb.W)) / np.abs(np.diag(pb.W))
        assert d.max() <= 1e-12
        S.factor()
        for g in (geom.g, np.array([0.2, -0.9, 0.4])):
            ref = pb.solve(g, rtol=1e-8)
            out = S.solve(g, rtol=1e-8)
            assert abs(out["iters"] - ref.iters) <= 1
            fx = S.solve(g, rtol=0.0, maxit=ref.iters, fixed=True)
            assert np.linalg.norm(fx["density"] - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
            assert _energy_rel(fx["density"], ref.x, pb.W) <= 1e-8
            assert np.abs(Z.T @ out["density"]).max() <= 1e-7 * np.linalg.norm(out["density"])
            mx = S.solve(g, rtol=1e-8, precision="mixed")
            L = pb.rhs(g)
            assert np.linalg.norm(L - pb.W @ mx["density"]) <= 1.05e-8 * np.linalg.norm(L)
            # the augmented solution solves the original singular system
            assert np.linalg.norm(L - pb.W0 @ out["density"]) <= 1e-7 * np.linalg.norm(L)


@pytest.mark.parametrize("geom,rows", [(WL.book(8, 2, jitter=True, seed=3), 64), (WL.cube_midplanes(6, 2), 128),
                                       (WL.panels(7, n=8, n_coarse=2), 192)], ids=lambda x: getattr(x, "name", x))
def test_panel_assembly(geom, rows):
    """V in row panels: W equals the one-piece assembly to rounding and the
    oracle to the parity bar; the solves agree."""
    pb = solver.Problem(geom)
    with M.Solver(geom) as S:
        S.assemble()
        W1 = S.matrix()
        S.assemble(panel_rows=rows)
        Wp = S.matrix()
        scale = np.abs(W1).max()
        # another summation order of the same double-float terms (each entry sums
        # ~100 terms with cancellation at 2^-48 per operation), and the panels
        # sum W[nu, nu'] and W[nu', nu] in different orders: both at rounding
        # level, ten times below the parity bar
        assert np.abs(Wp - W1).max() <= 1e-13 * scale
        assert np.abs(Wp - Wp.T).max() <= 1e-13 * scale
        assert np.abs(Wp - pb.W).max() <= 1e-12 * scale
        d = np.abs(np.diag(Wp) - np.diag(pb.W)) / np.abs(np.diag(pb.W))
        assert d.max() <= 1e-12
        S.factor()
        out = S.solve(geom.g, rtol=1e-8)
        pb.factor()
        ref = pb.solve(geom.g, rtol=1e-8)
        assert abs(out["iters"] - ref.iters) <= 1
        with pytest.raises(M.MsbemError) as e:
            S.assemble(panel_rows=100)
        assert e.value.status == -1
        with pytest.raises(M.MsbemError) as e:
            S.assemble(panel_rows=64, far_kernel=1)
        assert e.value.status == -1


def _oracle_rows(top, xyz, tri, rows, Q, rho):
    """Rows of W + rho Q Q^T from the oracle's pair integrals: for dof nu,
    W[nu, :] = sum_{k in J(nu)} s_k . (V[T_k, :] S), S the curl matrices."""
    from oracle import core
    s = top.curl_vectors()
    S = top.S_matrices()
    starts = np.searchsorted(top.s_dof, np.arange(top.ndof + 1))
    out = []
    for nu in rows:
        ks = np.arange(starts[nu], starts[nu + 1])
        R = np.repeat(top.s_tri[ks], top.nt)
        C = np.tile(np.arange(top.nt), len(ks))
        Vr = core.V_entries(xyz, tri, R, C).reshape(len(ks), top.nt)
        row = np.zeros(top.ndof)
        for c in range(3):
            row += S[c].T @ (s[ks, c] @ Vr)
        out.append(row + rho * (Q @ Q[nu]))
    return np.array(out)


def _oracle_diag(top, xyz, tri):
    """diag(W) from the oracle's pair integrals (each distinct near pair once)."""
    from oracle import core
    s = top.curl_vectors()
    starts = np.searchsorted(top.s_dof, np.arange(top.ndof + 1))
    cnt = np.diff(starts)
    owner = np.repeat(np.arange(top.ndof), cnt * cnt)
    off = np.arange(owner.size) - np.repeat(np.cumsum(cnt * cnt) - cnt * cnt, cnt * cnt)
    a = starts[owner] + off // cnt[owner]
    b = starts[owner] + off % cnt[owner]
    ta, tb = top.s_tri[a], top.s_tri[b]
    key = np.minimum(ta, tb) * top.nt + np.maximum(ta, tb)
    uk, inv = np.unique(key, return_inverse=True)
    v = core.V_entries(xyz, tri, uk // top.nt, uk % top.nt)[inv]
    d = np.zeros(top.ndof)
    np.add.at(d, owner, v * np.einsum("ij,ij->i", s[a], s[b]))
    return d


def test_cube_config_full_size():
    """The cube with mid-planes at h = 1/96 (N = 83,817, W 56 GB, V assembled in
    panels): Z and rho against the oracle (rho from all 83,817 FP64 diagonal
    entries), three sampled rows of W + rho Q Q^T, and the solves (true
    residual, the plain FP64 comparator's iteration count, mixed precision)."""
    from oracle.topology import Topology
    geom = WL.cube_config()
    top = Topology(geom.xyz, geom.tri)
    Zo = top.cells()
    xyz, tri = geom.xyz, geom.tri.astype(np.int32)
    diag_o = _oracle_diag(top, xyz, tri)
    rho_o = float(np.mean(diag_o))
    Lc = np.linalg.cholesky(Zo.T @ Zo)
    import scipy.linalg as sla
    Qo = sla.solve_triangular(Lc, Zo.T, lower=True).T
    with M.Solver(geom) as S:
        S.assemble()
        Z, rho = S.cells()
        assert np.array_equal(Z, Zo)
        # rho is the mean of 83,817 diagonal entries, each held to the 1e-12 bar
        assert abs(rho - rho_o) <= 1e-11 * rho_o
        rows = [0, 40000, S.n - 1]
        Wo = _oracle_rows(top, xyz, tri, rows, Qo, rho_o)
        scale = float(np.max(diag_o)) + rho_o
        for r, wo in zip(rows, Wo):
            wg = S.matrix(r, 1)[0]
            print("row", r, "max |dW| / scale", np.abs(wg - wo).max() / scale, "diag rel", abs(wg[r] - wo[r]) / abs(wo[r]))
            assert np.abs(wg - wo).max() <= 1e-12 * scale
            assert abs(wg[r] - wo[r]) <= 1e-12 * abs(wo[r])
        S.factor()
        df = S.solve(geom.g, rtol=1e-8)
        assert df["iters"] < 60
        Y, _ = S.apply(df["density"][None, :])
        L = S.rhs(geom.g)
        assert np.linalg.norm(L - Y[0]) <= 1.05e-8 * np.linalg.norm(L)
        assert np.abs(Z.T @ df["density"]).max() <= 1e-7 * np.linalg.norm(df["density"])
        pl = S.solve(geom.g, rtol=1e-8, precision="fp64")
        assert abs(pl["iters"] - df["iters"]) <= 1
        mx = S.solve(geom.g, rtol=1e-8, precision="mixed")
        assert np.linalg.norm(mx["density"] - df["density"]) <= 1e-7 * np.linalg.norm(df["density"])
        # the tensor-core products at this size (84 GB of slices): sampled rows
        # against the exactly rounded product of the device's own rows, and the
        # tensor-core solve forms to the true residual
        import math
        rng = np.random.default_rng(4)
        X = rng.standard_normal((16, S.n))
        Ytc, _ = S.apply(X, precision="tc")
        for r in rows:
            wg = S.matrix(r, 1)[0]
            for c in range(16):
                t = wg * X[c]
                ex = math.fsum(np.concatenate([t] + _two_prod_err(wg, X[c], t)))
                assert abs(Ytc[c, r] - ex) <= 2.0 ** -42 * np.abs(wg).max() * np.abs(X[c]).sum()
        for prec in ("tc", "mixed-tc"):
            o = S.solve(geom.g, rtol=1e-8, precision=prec)
            Y, _ = S.apply(o["density"][None, :])
            assert np.linalg.norm(L - Y[0]) <= 1.05e-8 * np.linalg.norm(L), prec
        # density bar of the mixed forms with the refinement's density test,
        # against the double-float PCG (held to the oracle above) run to 1e-13
        tight = S.solve(geom.g, rtol=1e-13, maxit=3000)["density"]
        for prec in ("mixed", "mixed-tc"):
            o = S.solve(geom.g, rtol=1e-8, precision=prec, density_tol=1e-9)
            e = np.linalg.norm(o["density"] - tight) / np.linalg.norm(tight)
            print(prec, "relative l2 error against the tight solve", e)
            assert e <= 1e-8, (prec, e)
        # W + rho Q Q^T on a wider sample: 300 rows stratified by the number of
        # sheets at their vertex (faces, mid-planes, junction lines, the centre),
        # each against the oracle's entries at its diagonal, its neighbours
        # (dofs sharing a triangle) and eight random columns
        _sampled_entries(S, top, geom, Qo, rho_o, scale)


def _sampled_entries(S, top, geom, Qo, rho_o, scale):
    rng = np.random.default_rng(5)
    q_of = top.q[top.dof_vertex]
    rows = []
    for qv in np.unique(q_of):
        pool = np.flatnonzero(q_of == qv)
        rows.extend(rng.choice(pool, min(len(pool), 75), replace=False).tolist())
    rows = np.array(sorted(set(rows)))[:300]
    # neighbours: dofs at the vertices of the triangles around the row's vertex
    tri = geom.tri
    nv = len(top.xyz)
    vt = [[] for _ in range(nv)]
    for t in range(top.nt):
        for v in tri[t]:
            vt[v].append(t)
    first = top.first_dof
    R, C, near = [], [], []
    for r in rows:
        vs = set(tri[vt[top.dof_vertex[r]]].ravel().tolist())
        nb = sorted({d for v in vs for d in range(first[v], first[v + 1])})
        far = rng.integers(0, top.ndof, 8).tolist()
        for c in nb:
            R.append(r); C.append(c); near.append(True)
        for c in far:
            R.append(r); C.append(c); near.append(False)
    R, C, near = np.array(R), np.array(C), np.array(near)
    wo = solver.W_entries(top, R, C) + rho_o * np.einsum("ij,ij->i", Qo[R], Qo[C])
    wg = np.empty_like(wo)
    for r in rows:
        m = R == r
        wg[m] = S.matrix(int(r), 1)[0][C[m]]
    err = np.abs(wg - wo)
    print("sampled entries:", len(wo), "rows:", len(rows), "max |dW| / scale", err.max() / scale)
    assert err.max() <= 1e-12 * scale
    big = near & (np.abs(wo) >= 1e-2 * scale)
    assert big.sum() >= len(rows)
    assert (err[big] <= 1e-12 * np.abs(wo[big])).all(), (err[big] / np.abs(wo[big])).max()


def _two_prod_err(a, b, p):
    """Terms whose exact sum is the rounding error a*b - p of the products
    p = a*b (Veltkamp splitting; each term exact in FP64 barring underflow)."""
    def split(x):
        c = x * 134217729.0
        hi = c - (c - x)
        return hi, x - hi
    ah, al = split(a)
    bh, bl = split(b)
    return [ah * bh - p, ah * bl, al * bh, al * bl]
