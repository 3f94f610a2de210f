"""GPU test of msbem_spd_inverse_noalloc, the inversion entry point that
allocates no device memory (for callers that cannot allocate: a process whose
GPU memory is all reserved by its own pool, or a loop that cannot afford the
device synchronisation of cudaMalloc/cudaFree).

The existing path inverts the same kind of matrix inside msbem_factor: with a
single patch covering the whole mesh and no coarse space, the preconditioner is
exactly W^{-1}, so one fixed PCG iteration returns W^{-1} L.  The allocation-free
inverse applied to L must agree with it to the density tolerance of the parity
tests (1e-8 relative), on two calls in a row, on two different matrices.  This
file is collected last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import build as B
from paper_2310_09204_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def _single_patch(geom):
    geom.patch = np.zeros(geom.nt, np.int32)
    return geom


def _existing_path(geom):
    """W, L and W^{-1} L from msbem_factor + one PCG iteration."""
    with M.Solver(geom) as S:
        S.assemble().factor(use_coarse=0)
        info = S.split_info()
        assert info["n_faces"] == 1 and info["n_wire_basket"] == 0
        W = S.matrix()
        L = S.rhs(geom.g)
        out = S.solve(geom.g, rtol=0.0, maxit=1, fixed=True)
    return W, L, out["density"]


def test_noalloc_inverse_matches_factor_path():
    import torch
    B.build()
    M.lib()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [_single_patch(WL.unit_square(12, 3)), _single_patch(WL.book(6, 2, jitter=False))]
    for geom in cases:                       # two calls in a row, two matrices
        W, L, ref = _existing_path(geom)
        n = W.shape[0]
        assert 1 <= n <= M.NOALLOC_MAX_N
        A = torch.from_numpy(W).cuda()
        Ainv = torch.empty_like(A)
        st = M.msbem_spd_inverse_noalloc(A, Ainv, stream)
        torch.cuda.synchronize()
        assert st == 0
        x = Ainv.cpu().numpy() @ L
        assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)
        # the inverse itself is a two-sided inverse of W
        assert np.abs(Ainv.cpu().numpy() @ W - np.eye(n)).max() <= 1e-8


def _spd(n, seed):
    """Seeded symmetric, strictly diagonally dominant (hence SPD) matrix."""
    rng = np.random.default_rng(seed)
    G = rng.uniform(-1.0, 1.0, (n, n))
    A = 0.5 * (G + G.T)
    A[np.diag_indices(n)] = np.abs(A).sum(axis=1) + 1.0
    return A


def test_noalloc_at_the_maximum_order_and_in_place():
    """n = MSBEM_NOALLOC_MAX_N, where the fixed scratch has no slack (every
    panel and the largest offsets run), then the same matrix in place."""
    import torch
    B.build()
    n = M.NOALLOC_MAX_N
    A_h = _spd(n, 11)
    A = torch.from_numpy(A_h).cuda()
    Ainv = torch.empty_like(A)
    assert M.msbem_spd_inverse_noalloc(A, Ainv) == 0
    torch.cuda.synchronize()
    X = Ainv.cpu().numpy()
    assert np.abs(X @ A_h - np.eye(n)).max() <= 1e-8
    A2 = A.clone()
    assert M.msbem_spd_inverse_noalloc(A2, A2) == 0          # in place
    torch.cuda.synchronize()
    assert np.abs(A2.cpu().numpy() - X).max() <= 1e-12 * np.abs(X).max()


def test_noalloc_breakdown_then_recovers():
    """An indefinite matrix reports MSBEM_BREAKDOWN; the next call on an SPD
    matrix succeeds (the shared breakdown flag starts at zero every call)."""
    import torch
    B.build()
    n = 70
    D = torch.from_numpy(np.diag([1.0 if i % 2 == 0 else -1.0 for i in range(n)])).cuda()
    assert M.msbem_spd_inverse_noalloc(D, torch.empty_like(D)) == -6        # BREAKDOWN
    A_h = _spd(n, 3)
    A = torch.from_numpy(A_h).cuda()
    Ainv = torch.empty_like(A)
    assert M.msbem_spd_inverse_noalloc(A, Ainv) == 0
    torch.cuda.synchronize()
    assert np.abs(Ainv.cpu().numpy() @ A_h - np.eye(n)).max() <= 1e-10


def test_noalloc_rejects_oversize_and_empty():
    import torch
    B.build()
    A = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    # the C side rejects an order beyond the maximum before touching memory
    assert M.lib().msbem_spd_inverse_noalloc(A.data_ptr(), M.NOALLOC_MAX_N + 1, A.data_ptr(), None) == -1
    assert M.lib().msbem_spd_inverse_noalloc(None, 4, None, None) == -1
    assert M.lib().msbem_spd_inverse_noalloc(A.data_ptr(), 0, A.data_ptr(), None) == -1


def test_noalloc_binding_rejects_bad_tensors():
    """The binding checks what the raw pointers cannot carry: dtype, shape,
    layout and device."""
    import torch
    B.build()
    good = torch.eye(8, dtype=torch.float64, device="cuda")
    bad = [
        (good.float(), good),                                    # float32
        (good, torch.empty((9, 9), dtype=torch.float64, device="cuda")),   # shapes differ
        (torch.empty((8, 4), dtype=torch.float64, device="cuda"), good),   # not square
        (torch.empty((16, 16), dtype=torch.float64, device="cuda")[::2, ::2], good),   # strided
        (good.cpu(), good),                                      # host tensor
        (torch.empty((M.NOALLOC_MAX_N + 1,) * 2, dtype=torch.float64, device="cuda"),) * 2,
    ]
    for A, Ainv in bad:
        with pytest.raises(ValueError):
            M.msbem_spd_inverse_noalloc(A, Ainv)
