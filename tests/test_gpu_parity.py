"""GPU parity of the CUDA path against the CPU FP64 oracle (calls go through
the C ABI via the ctypes binding).

Tolerances (stated for the workload, derived in the design notes):
* W: max |W_gpu - W_oracle| <= 1e-12 max |W| (normwise); the diagonal and
  the nearest-neighbour couplings (dofs whose vertices share a triangle) of
  size >= 1e-2 max|W| also entry-wise within 1e-12 relative.
* RHS: 1e-14 relative (max norm).
* PCG: iteration counts within +-1; at the same (fixed) iteration count the
  densities agree to 1e-8 relative in l2 and in the W-energy norm.
"""
import math

import numpy as np
import pytest

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import build as B
from paper_2310_09204_gb300 import workloads as WL
from oracle import solver

pytestmark = pytest.mark.gpu

FAR_KERNELS = [0, 1]           # 0 double-float on the FP32 pipe, 1 native FP64
_ORACLE = {}


@pytest.fixture(scope="module", autouse=True)
def _build():
    B.build()
    M.lib()


def oracle(geom, **kw):
    key = (geom.name, tuple(sorted(kw.items())))
    if key not in _ORACLE:
        pb = solver.Problem(geom, **kw)
        pb.factor()
        _ORACLE[key] = pb
    return _ORACLE[key]


SMALL = [WL.flat_config(), WL.book(8, 2, jitter=True, seed=3), WL.bowtie(6, 2), WL.disk(5, fin=True),
         WL.unit_square(12, 3, "coarse_tri")]


def _neighbour_mask(top):
    """Dof pairs whose vertices lie in a common triangle (nearest neighbours)."""
    import scipy.sparse as sp
    nv = top.nv
    t = top.tri
    rows = np.repeat(t, 3, axis=1).ravel()
    cols = np.tile(t, (1, 3)).ravel()
    A = sp.csr_matrix((np.ones(rows.size), (rows, cols)), shape=(nv, nv))
    dv = top.dof_vertex
    return np.asarray(A[dv][:, dv].todense()) > 0


def _w_close(Wg, Wo, top=None):
    """W tolerance: max |dW| <= 1e-12 max |W| (normwise), and entry-wise 1e-12
    on the diagonal and on the nearest-neighbour couplings of size >= 1e-2
    max|W|.  Neighbour entries that cancel to below that (zero by symmetry at
    junctions, for instance) are held to the normwise bar: their relative error
    grows with the cancellation ratio in any finite-precision evaluation."""
    scale = np.abs(Wo).max()
    assert np.abs(Wg - Wo).max() <= 1e-12 * scale, np.abs(Wg - Wo).max() / scale
    d = np.abs(np.diag(Wg) - np.diag(Wo)) / np.abs(np.diag(Wo))
    assert d.max() <= 1e-12, d.max()
    if top is not None:
        nb = _neighbour_mask(top) & (np.abs(Wo) >= 1e-2 * scale)
        rel = np.abs(Wg - Wo)[nb] / np.abs(Wo)[nb]
        assert rel.max() <= 1e-12, rel.max()


@pytest.mark.parametrize("far_kernel", FAR_KERNELS)
@pytest.mark.parametrize("geom", SMALL, ids=lambda g: g.name)
def test_matrix_parity(geom, far_kernel):
    pb = oracle(geom)
    with M.Solver(geom) as S:
        assert S.n == pb.ndof
        v, s = S.dof_map()
        assert np.array_equal(v, pb.top.dof_vertex) and np.array_equal(s, pb.top.dof_sector)
        S.assemble(far_kernel=far_kernel)
        Wg = S.matrix()
    assert np.array_equal(Wg, Wg.T)
    _w_close(Wg, pb.W, pb.top)


@pytest.mark.parametrize("ss_order", [3, 8])
def test_matrix_parity_other_singular_orders(ss_order):
    geom = WL.book(6, 2, jitter=False)
    pb = solver.Problem(geom, ss_order=ss_order)
    with M.Solver(geom) as S:
        S.assemble(ss_order=ss_order, far_kernel=1)
        _w_close(S.matrix(), pb.W, pb.top)


@pytest.mark.parametrize("geom", SMALL[:3], ids=lambda g: g.name)
def test_rhs_parity(geom):
    pb = oracle(geom)
    rng = np.random.default_rng(5)
    with M.Solver(geom) as S:
        for g in (geom.g, rng.uniform(-1, 1, 3)):
            Lg = S.rhs(g)
            Lo = pb.rhs(g)
            assert np.abs(Lg - Lo).max() <= 1e-14 * max(np.abs(Lo).max(), 1e-300)


def _rel(a, b, W=None):
    if W is None:
        return np.linalg.norm(a - b) / np.linalg.norm(b)
    e = a - b
    return math.sqrt(max(e @ W @ e, 0.0)) / math.sqrt(b @ W @ b)


@pytest.mark.parametrize("geom", SMALL, ids=lambda g: g.name)
def test_pcg_parity(geom):
    pb = oracle(geom)
    ref = pb.solve(rtol=1e-8)
    with M.Solver(geom) as S:
        S.assemble().factor()
        out = S.solve(geom.g, rtol=1e-8)
        assert abs(out["iters"] - ref.iters) <= 1
        assert out["hist"][-1] <= 1e-8
        # same iteration count: densities agree to 1e-8 (l2 and energy)
        k = ref.iters
        fixed = S.solve(geom.g, rtol=0.0, maxit=k, fixed=True)
        assert _rel(fixed["density"], ref.x) <= 1e-8
        assert _rel(fixed["density"], ref.x, pb.W) <= 1e-8
        # residual histories agree; residuals at rounding level (< 1e-12) only in size
        np.testing.assert_allclose(fixed["hist"][: k + 1], ref.hist[: k + 1], rtol=1e-6, atol=1e-12)
        if k >= 3:
            assert abs(fixed["kappa"] - ref.kappa) <= 1e-6 * ref.kappa


def test_plain_cg_and_options():
    geom = WL.book(8, 2, jitter=True, seed=3)
    pb = oracle(geom)
    plain = solver.pcg(pb.W, pb.rhs(), None, rtol=1e-8)
    Mdiag = solver.build_preconditioner(pb.top, pb.W, pb.coarse, geom.parent, geom.patch, "diagonal")
    wbd = solver.pcg(pb.W, pb.rhs(), Mdiag.apply, rtol=1e-8)
    Mnoc = solver.build_preconditioner(pb.top, pb.W, None, geom.parent, geom.patch)
    noc = solver.pcg(pb.W, pb.rhs(), Mnoc.apply, rtol=1e-8)
    with M.Solver(geom) as S:
        S.assemble()
        out = S.solve(geom.g, precondition=False)
        assert abs(out["iters"] - plain.iters) <= 1
        assert _rel(out["density"], plain.x) <= 1e-7
        S.factor(wire_basket=1)
        out = S.solve(geom.g)
        assert abs(out["iters"] - wbd.iters) <= 1
        S.factor(use_coarse=0)
        out = S.solve(geom.g)
        assert abs(out["iters"] - noc.iters) <= 1


def test_status_codes_and_outputs():
    geom = WL.flat_config()
    pb = oracle(geom)
    with M.Solver(geom) as S:
        with pytest.raises(M.MsbemError) as e:
            S.solve(geom.g)
        assert e.value.status == -9                    # NOT_READY
        S.assemble()
        with pytest.raises(M.MsbemError) as e:
            S.solve(geom.g)                            # factor missing
        assert e.value.status == -9
        S.factor()
        out = S.solve(geom.g, maxit=1, raise_on_status=False)
        assert out["status"] == -5 and out["iters"] == 1   # NOT_CONVERGED, density written
        one = solver.pcg(pb.W, pb.rhs(), pb.M.apply, rtol=0.0, maxit=1, fixed=True)
        assert _rel(out["density"], one.x) <= 1e-10
        with pytest.raises(M.MsbemError) as e:
            S.assemble(ss_order=40)
        assert e.value.status == -1
        # device output buffer
        import torch
        dev = torch.empty(S.n, dtype=torch.float64, device="cuda")
        out = S.solve(geom.g, out=dev)
        torch.cuda.synchronize()
        ref = pb.solve()
        assert _rel(dev.cpu().numpy(), ref.x) <= 1e-7
        # g along no normal component gives the zero solution
        out = S.solve(np.zeros(3))
        assert out["iters"] == 0 and np.all(out["density"] == 0)


def test_geometry_without_dofs():
    # one coarse triangle refined once: every fine vertex lies on the boundary
    # or has a single sector except the interior ones; use the coarse mesh itself
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    tri = np.array([[0, 1, 2]], np.int32)
    with M.Solver(None) as S:
        S.upload(xyz, tri, xyz, tri, np.zeros(1, np.int32), np.zeros(1, np.int32))
        assert S.n == 0
        S.assemble().factor()
        out = S.solve(np.array([0.0, 0.0, 1.0]))
        assert out["iters"] == 0 and out["density"].size == 0


def test_upload_rejects_non_nested_coarse_mesh():
    geom = WL.unit_square(8, 2)
    bad_coarse = geom.coarse_xyz + np.array([0.01, 0.0, 0.0])
    with M.Solver(None) as S:
        with pytest.raises(M.MsbemError) as e:
            S.upload(geom.xyz, geom.tri, bad_coarse, geom.coarse_tri, geom.parent, geom.patch)
        assert e.value.status == -2


@pytest.mark.parametrize("far_kernel", FAR_KERNELS)
def test_book_config_full_size(far_kernel):
    """Full-size three-page book (h = 1/64, N = 12,033) in the launch
    configuration the benchmark times: the whole W, the RHS, and the PCG
    iteration count and density against the oracle."""
    geom = WL.book_config()
    pb = oracle(geom)
    ref = pb.solve(rtol=1e-8)
    with M.Solver(geom) as S:
        S.assemble(far_kernel=far_kernel)
        Wg = S.matrix()
        _w_close(Wg, pb.W)
        del Wg
        S.factor()
        out = S.solve(geom.g, rtol=1e-8)
        assert abs(out["iters"] - ref.iters) <= 1
        fixed = S.solve(geom.g, rtol=0.0, maxit=ref.iters, fixed=True)
        assert _rel(fixed["density"], ref.x) <= 1e-8
        assert _rel(fixed["density"], ref.x, pb.W) <= 1e-8
        info = S.split_info()
        assert info["n_coarse"] == 33 and info["n_faces"] == 48


def test_solve_beyond_the_history_capacity():
    """maxit above the geometry's persistent history (1,024 iterations): the
    iterations run launch by launch on the caller's stream (here the legacy
    default stream) with a temporary history, and give bit for bit the result
    of the graph-launched chunks."""
    geom = WL.flat_config()
    with M.Solver(geom) as S:
        S.assemble().factor()
        a = S.solve(geom.g, rtol=1e-8)
        b = S.solve(geom.g, rtol=1e-8, maxit=1500)
        assert a["iters"] == b["iters"] > 0
        assert np.array_equal(a["density"], b["density"])
        assert np.array_equal(a["hist"], b["hist"])
