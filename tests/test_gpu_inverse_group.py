"""Grouped SPD inversion (msbem_spd_inverse_group): the blocked Gauss-Jordan
recursion of the preconditioner set-up (Sec. 5, eq. jumpSplit: the face,
wire-basket and coarse blocks of M(H;h) inverted explicitly), double-float
through the tensor-core update, or FP32.

The bar: the inverse of the plain definition A X = I, within the rounding
bound of the arithmetic (||X - A^-1|| <= c u cond(A) ||A^-1||, u = 2^-48 for
double-float, 2^-24 for FP32), at orders that span several 128 x 64 output
tiles and ragged last panels; grouping changes no bit; the exponent cases of
the operand slicing (row maxima in [1/4, 1/2), which gives exponent 0; zero
panel rows of a block-diagonal matrix; rows many binades apart) are covered;
a matrix that is not positive definite is reported without disturbing the
others."""
import numpy as np
import pytest

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import build as B

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _build():
    B.build()
    M.lib()


def _spd(n, seed, scale=1.0, kind="gram"):
    rng = np.random.default_rng(seed)
    if kind == "gram":
        Bm = rng.uniform(-1, 1, (n, n))
        A = Bm @ Bm.T + 0.1 * n * np.eye(n)
    elif kind == "decay":          # 1/(1+|i-j|^2) off the diagonal: hypersingular-like decay
        d = np.abs(np.subtract.outer(np.arange(n), np.arange(n))).astype(float)
        A = -1.0 / (1.0 + d * d)
        A[np.diag_indices(n)] = 4.0 + 2.0 * n / 50.0
    elif kind == "blockdiag":      # zero off-diagonal blocks: zero panel rows
        A = np.zeros((n, n))
        h = n // 2
        for lo, hi in ((0, h), (h, n)):
            Bm = rng.uniform(-1, 1, (hi - lo, hi - lo))
            A[lo:hi, lo:hi] = Bm @ Bm.T + 0.1 * (hi - lo) * np.eye(hi - lo)
    elif kind == "graded":         # rows and columns scaled over many binades
        Bm = rng.uniform(-1, 1, (n, n))
        D = np.diag(2.0 ** rng.integers(-20, 20, n))
        A = D @ (Bm @ Bm.T + 0.1 * n * np.eye(n)) @ D
    return A * scale


def _inv_group(mats, precision="df"):
    T = [torch.tensor(A, device="cuda:0") for A in mats]
    st = M.msbem_spd_inverse_group(T, precision=precision)
    return [t.cpu().numpy() for t in T], st


def _rel(X, A):
    Ai = np.linalg.inv(A)
    return np.linalg.norm(X - Ai) / np.linalg.norm(Ai), np.linalg.cond(A)


ORDERS = [1, 7, 31, 32, 33, 49, 100, 130, 200, 257]


@pytest.mark.parametrize("kind", ["gram", "decay"])
def test_df_inverse_against_the_definition(kind):
    mats = [_spd(n, 10 + n, kind=kind) for n in ORDERS]
    X, st = _inv_group(mats)
    assert st == [0] * len(mats)
    for A, Xi in zip(mats, X):
        rel, cond = _rel(Xi, A)
        assert rel <= 64 * 2.0 ** -48 * cond * max(1.0, A.shape[0] / 32), (A.shape[0], rel, cond)


def test_exponent_cases_of_the_slicing():
    # whole matrices scaled so that row maxima of the operands land in
    # [1/4, 1/2) (exponent 0), in [1/2, 1), far below 1 and far above it
    mats = []
    for j, sc in enumerate([0.3 / 40.0, 0.7 / 40.0, 2.0 ** -30, 2.0 ** 30, 1.0]):
        mats.append(_spd(96, 70 + j, scale=sc))
    mats += [_spd(130, 80, kind="blockdiag"), _spd(75, 81, kind="graded")]
    X, st = _inv_group(mats)
    assert st == [0] * len(mats)
    for A, Xi in zip(mats, X):
        Ai = np.linalg.inv(A)
        if A.shape[0] == 75:
            # graded: the error of each entry against the scales of its row and column
            d = np.sqrt(np.abs(np.diag(Ai)))
            E = np.abs(Xi - Ai) / np.outer(d, d)
            assert E.max() <= 1e-9, E.max()
        else:
            rel, cond = _rel(Xi, A)
            assert rel <= 64 * 2.0 ** -48 * cond * 4, (A.shape[0], rel, cond)


def test_grouping_changes_no_bit():
    mats = [_spd(n, 30 + n) for n in (200, 33, 130, 7, 64)]
    G, _ = _inv_group(mats)
    for A, Xg in zip(mats, G):
        (Xa,), _ = _inv_group([A])
        assert np.array_equal(Xa, Xg)


def test_fp32_inverse():
    mats = [_spd(n, 50 + n) for n in (40, 100, 257)]
    X, st = _inv_group(mats, precision="fp32")
    assert st == [0, 0, 0]
    for A, Xi in zip(mats, X):
        rel, cond = _rel(Xi, A)
        assert rel <= 64 * 2.0 ** -24 * cond * 8, (A.shape[0], rel, cond)
        assert np.array_equal(Xi, Xi.T)


def test_breakdown_is_reported_per_matrix():
    good = _spd(50, 3)
    bad = _spd(40, 4)
    bad[5, 5] = -abs(bad[5, 5]) * 100.0      # a negative diagonal entry: not positive definite
    X, st = _inv_group([good, bad])
    assert st[0] == 0 and st[1] == -6
    rel, cond = _rel(X[0], good)
    assert rel <= 64 * 2.0 ** -48 * cond * 2


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        M.msbem_spd_inverse_group([])
    with pytest.raises(ValueError):
        M.msbem_spd_inverse_group([torch.zeros(4, 5, dtype=torch.float64, device="cuda:0")])
    with pytest.raises(ValueError):
        M.msbem_spd_inverse_group([torch.eye(4, dtype=torch.float32, device="cuda:0")])
    t = torch.eye(4, dtype=torch.float64, device="cuda:0")
    with pytest.raises(ValueError):
        M.msbem_spd_inverse_group([t, t])
    with pytest.raises(ValueError):
        M.msbem_spd_inverse_group([t], precision="fp16")


def test_tensor_core_update_against_the_definition():
    # orders >= 2048 take the tensor-core update (exact 8-bit slices of both
    # operands, 26 slice pairs in tensor memory, folded into double-float),
    # smaller ones the CUDA-core update, in the same grouped steps
    mats = [_spd(2100, 91), _spd(2333, 92, kind="decay"), _spd(130, 93), _spd(33, 94)]
    X, st = _inv_group(mats)
    assert st == [0] * len(mats)
    for A, Xi in zip(mats, X):
        rel, cond = _rel(Xi, A)
        assert rel <= 64 * 2.0 ** -48 * cond * max(1.0, A.shape[0] / 32), (A.shape[0], rel, cond)
    # the large ones alone: the same bits (the path depends on a matrix's own order)
    (X0,), _ = _inv_group([mats[0]])
    assert np.array_equal(X0, X[0])
    (X3,), _ = _inv_group([mats[3]])
    assert np.array_equal(X3, X[3])


def test_tensor_core_update_on_a_graded_matrix():
    # rows and columns over 2^+-20: the equilibration keeps the sliced
    # products' error at the scale of the entries
    A = _spd(2050, 95, kind="graded")
    (X,), st = _inv_group([A])
    assert st == [0]
    Ai = np.linalg.inv(A)
    d = np.sqrt(np.abs(np.diag(Ai)))
    assert (np.abs(X - Ai) / np.outer(d, d)).max() <= 1e-9
