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


def test_noalloc_rejects_oversize_and_empty():
    import torch
    B.build()
    big = torch.empty((M.NOALLOC_MAX_N + 1, 1), dtype=torch.float64, device="cuda")
    assert M.msbem_spd_inverse_noalloc(big, big) == -1          # INVALID_ARG
    assert M.lib().msbem_spd_inverse_noalloc(None, 4, None, None) == -1
