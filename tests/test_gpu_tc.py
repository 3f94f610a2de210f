"""The double-float product on the tensor cores (msbem_apply precision 3).

W and X are cut into six signed 8-bit integer slices under a power-of-two
scale per row of W and per vector; the slice products are summed on the
tensor cores, exactly, and folded into double-float sums.  The reference is
the exactly rounded product of the device's own W (msbem_copy_matrix) with X,
formed on the host from error-free products (Veltkamp splitting) and math.fsum;
the bound per entry is

    |Y_ic - (W X)_ic| <= 2^-42 max_j |W_ij| sum_j |X_cj|,

which covers the slices' remainders (2^-49 of the scales), the levels left out
(2^-56 N of the scales) and the double-float fold, with margin, for vectors
of any magnitude within FP64's range.  The same bound holds for the CUDA-core
double-float product (precision 0) on vectors within FP32's range."""
import math

import numpy as np
import pytest

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import build as B
from paper_2310_09204_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

BOUND = 2.0 ** -42


@pytest.fixture(scope="module", autouse=True)
def _build():
    B.build()
    M.lib()


def _split(a):
    c = a * 134217729.0          # 2^27 + 1
    hi = c - (c - a)
    return hi, a - hi


def _exact_rows(W, X, rows):
    """Correctly rounded (W X^T)[rows] from error-free products and fsum."""
    wh, wl = _split(W[rows])
    out = np.empty((len(rows), X.shape[0]))
    for c in range(X.shape[0]):
        xh, xl = _split(X[c])
        p = W[rows] * X[c]
        # p exactly = wh*xh + wh*xl + wl*xh + wl*xl; e = that - p (exact terms)
        terms = np.stack([p, wh * xh - p, wh * xl, wl * xh, wl * xl], axis=-1)
        for k, i in enumerate(rows):
            out[k, c] = math.fsum(terms[k].ravel())
    return out


def _check(W, X, Y, rows):
    Ye = _exact_rows(W, X, rows)
    scale = np.abs(W[rows]).max(axis=1)[:, None] * np.abs(X).sum(axis=1)[None, :]
    err = np.abs(Y[:, rows].T - Ye)
    assert np.all(err <= BOUND * scale + 1e-300), float((err / np.maximum(scale, 1e-300)).max())
    return float((err / np.maximum(scale, 1e-300)).max())


@pytest.mark.parametrize("geom", [WL.book(8, 2, jitter=True, seed=3), WL.bowtie(6, 2), WL.panels(7, n=6)],
                         ids=lambda g: g.name)
def test_tc_product_exactly_rounded_reference(geom):
    rng = np.random.default_rng(41)
    with M.Solver(geom) as S:
        S.assemble()
        W = S.matrix()
        n = S.n
        X = rng.standard_normal((16, n))
        X[3] *= 1e-30
        X[4] *= 1e25
        X[5, : n // 2] = 0.0
        X[6] = 0.0
        X[7] = np.where(rng.random(n) < 0.1, rng.standard_normal(n) * 1e8, X[7])
        X[8] *= 1e-200
        X[9] *= 1e200
        rows = np.arange(n)
        Ytc, ms = S.apply(X, precision="tc")
        assert ms > 0.0
        Ydf, _ = S.apply(X, precision="df")
        e_tc = _check(W, X, Ytc, rows)
        # the CUDA-core product holds X as FP32 pairs: only vectors within
        # FP32's range there (the sliced product scales in FP64)
        keep = [c for c in range(16) if c not in (3, 8, 9)]
        e_df = _check(W, X[keep], Ydf[keep], rows)
        assert np.all(Ytc[6] == 0.0)
        print(f"{geom.name}: N={n} max rel err tc {e_tc:.2e} df {e_df:.2e}")


def test_tc_product_does_not_depend_on_the_batch():
    """A vector's product is bitwise the same alone or among 16, and scaling a
    vector by a power of two scales its product exactly (the slices are
    taken under a per-vector power-of-two scale)."""
    geom = WL.book(8, 2, jitter=True, seed=3)
    rng = np.random.default_rng(5)
    with M.Solver(geom) as S:
        S.assemble()
        X = rng.standard_normal((16, S.n))
        Y16, _ = S.apply(X, precision="tc")
        for k in (1, 3, 9):
            Yk, _ = S.apply(X[:k], precision="tc")
            assert np.array_equal(Yk, Y16[:k])
        for c in (0, 7, 15):
            Y1, _ = S.apply(X[c:c + 1], precision="tc")
            assert np.array_equal(Y1[0], Y16[c])
        Ys, _ = S.apply(np.ldexp(X, 37), precision="tc")
        assert np.array_equal(Ys, np.ldexp(Y16, 37))
        import torch
        Xd = torch.from_numpy(X[:5].copy()).cuda()
        Yd = torch.empty_like(Xd)
        S.apply(Xd, precision="tc", out=Yd)
        torch.cuda.synchronize()
        assert np.array_equal(Yd.cpu().numpy(), Y16[:5])


def test_tc_slices_follow_reassembly():
    """The slices are rebuilt after W changes (a second assembly with the
    FP64 far field gives a slightly different W)."""
    geom = WL.bowtie(6, 2)
    rng = np.random.default_rng(6)
    with M.Solver(geom) as S:
        S.assemble()
        X = rng.standard_normal((4, S.n))
        S.apply(X, precision="tc")
        S.assemble(far_kernel=1)
        W = S.matrix()
        Y, _ = S.apply(X, precision="tc")
        _check(W, X, Y, np.arange(S.n))


def test_tc_product_full_size_book():
    """The full-size book (N = 12,033): 16 vectors against the exactly
    rounded product at sampled rows, and against the CUDA-core product."""
    geom = WL.book_config()
    rng = np.random.default_rng(8)
    with M.Solver(geom) as S:
        S.assemble()
        n = S.n
        X = rng.standard_normal((16, n))
        Ytc, ms_tc = S.apply(X, precision="tc")
        Ydf, ms_df = S.apply(X, precision="df")
        rows = np.arange(0, n, 97)
        W = S.matrix()
        _check(W, X, Ytc, rows)
        scale = np.abs(W).max(axis=1)[None, :] * np.abs(X).sum(axis=1)[:, None]
        assert np.all(np.abs(Ytc - Ydf) <= 2 * BOUND * scale)
        print(f"book N={n}: tc {ms_tc:.3f} ms, df {ms_df:.3f} ms (16 vectors)")
        # the column split the autotuner picked at assembly serves every batch
        # size alike: a vector's product is the same alone and among 16
        for prec in ("df", "fp32", "tc"):
            Y16, _ = S.apply(X, precision=prec)
            Y1, _ = S.apply(X[5:6], precision=prec)
            assert np.array_equal(Y1[0], Y16[5]), prec


@pytest.mark.parametrize("geom", [WL.book(8, 2, jitter=True, seed=3), WL.panels(7, n=6)], ids=lambda g: g.name)
def test_fp16_product_bound(geom):
    """Scaled FP16 on the tensor cores: W rounded to 11 bits under its row's
    power-of-two scale (at most 2^-10 of the row's largest entry), the vectors
    to 22 bits, FP32 accumulation: within 2^-9 max_j |W_ij| sum_j |X_cj|."""
    rng = np.random.default_rng(42)
    with M.Solver(geom) as S:
        S.assemble()
        W = S.matrix()
        X = rng.standard_normal((16, S.n))
        X[2] *= 1e-150
        X[5] *= 1e150
        Y, ms = S.apply(X, precision="fp16-tc")
        assert ms > 0.0
        Ye = _exact_rows(W, X, np.arange(S.n))
        scale = np.abs(W).max(axis=1)[:, None] * np.abs(X).sum(axis=1)[None, :]
        err = np.abs(Y.T - Ye) / scale
        assert err.max() <= 2.0 ** -9, err.max()
        assert err.max() >= 2.0 ** -40            # it is the low-precision product
        Y1, _ = S.apply(X[4:5], precision="fp16-tc")
        assert np.array_equal(Y1[0], Y[4])


SMALL = [WL.flat_config(), WL.book(8, 2, jitter=True, seed=3), WL.bowtie(6, 2)]


@pytest.mark.parametrize("geom", SMALL, ids=lambda g: g.name)
def test_tc_solve_against_oracle(geom):
    """Double-float PCG with the tensor-core products: the parity bar of the
    default path (iterations within +-1, densities to 1e-8 at a fixed count)."""
    from oracle import solver
    pb = solver.Problem(geom)
    pb.factor()
    ref = pb.solve(rtol=1e-8)
    with M.Solver(geom) as S:
        S.assemble().factor()
        out = S.solve(geom.g, rtol=1e-8, precision="tc")
        assert abs(out["iters"] - ref.iters) <= 1
        fx = S.solve(geom.g, rtol=0.0, maxit=ref.iters, fixed=True, precision="tc")
        assert np.linalg.norm(fx["density"] - ref.x) <= 1e-8 * np.linalg.norm(ref.x)
        df = S.solve(geom.g, rtol=0.0, maxit=ref.iters, fixed=True)
        assert np.linalg.norm(fx["density"] - df["density"]) <= 1e-11 * np.linalg.norm(df["density"])


def test_tc_batch_column_independent():
    geom = WL.book(8, 2, jitter=True, seed=3)
    G = np.random.default_rng(12).uniform(-1, 1, (19, 3))
    with M.Solver(geom) as S:
        S.assemble().factor()
        full = S.solve_batch(G, rtol=1e-9, precision="tc")
        for c in (0, 9, 17):
            alone = S.solve_batch(G[c:c + 1], rtol=1e-9, precision="tc")
            assert alone["iters"][0] == full["iters"][c]
            assert np.array_equal(alone["density"][0], full["density"][c])
        one = S.solve(G[4], rtol=1e-9, precision="tc")
        assert np.array_equal(one["density"], full["density"][4])
        df = S.solve_batch(G[:16], rtol=1e-9)
        assert np.abs(df["iters"] - full["iters"][:16]).max() <= 1
        assert np.linalg.norm(df["density"] - full["density"][:16]) <= 1e-8 * np.linalg.norm(df["density"])


@pytest.mark.parametrize("prec", ["mixed-tc", "mixed-fp16"])
@pytest.mark.parametrize("geom", SMALL, ids=lambda g: g.name)
def test_mixed_tc_reaches_true_residual(geom, prec):
    """Mixed precision with the refinement residual on the tensor cores
    (double-float product), the inner PCG in FP32 on the CUDA cores or in
    scaled FP16 on the tensor cores; the TRUE residual with the oracle's W
    meets the tolerance."""
    from oracle import solver
    pb = solver.Problem(geom)
    rng = np.random.default_rng(21)
    with M.Solver(geom) as S:
        S.assemble().factor()
        for g in (geom.g, rng.uniform(-1, 1, 3)):
            L = pb.rhs(g)
            out = S.solve(g, rtol=1e-8, precision=prec)
            rel = np.linalg.norm(L - pb.W @ out["density"]) / np.linalg.norm(L)
            assert rel <= 1.05e-8, rel
            assert out["hist"][-1] <= 1e-8 and len(out["hist"]) >= 2
            assert np.all(np.diff(out["hist"]) < 0)


@pytest.mark.parametrize("prec", ["mixed-tc", "mixed-fp16"])
def test_mixed_tc_batch_alone_and_in_the_mix(prec):
    geom = WL.book(8, 2, jitter=True, seed=3)
    from oracle import solver
    pb = solver.Problem(geom)
    G = np.random.default_rng(22).uniform(-1, 1, (6, 3))
    G[3] = 0.0
    with M.Solver(geom) as S:
        S.assemble().factor()
        bt = S.solve_batch(G, rtol=1e-8, precision=prec)
        for c in range(len(G)):
            if c == 3:
                assert bt["iters"][c] == 0 and np.all(bt["density"][c] == 0.0)
                continue
            L = pb.rhs(G[c])
            assert np.linalg.norm(L - pb.W @ bt["density"][c]) <= 1.05e-8 * np.linalg.norm(L)
        alone = S.solve_batch(G[1:2], rtol=1e-8, precision=prec)
        assert np.array_equal(alone["density"][0], bt["density"][1])


def test_tensor_modes_full_size_book():
    """The full-size book: 16 right-hand sides in the tensor-core modes;
    true residuals with the device's own W, densities against the default
    double-float batch."""
    geom = WL.book_config()
    G = np.random.default_rng(31).uniform(-1, 1, (16, 3))
    with M.Solver(geom) as S:
        S.assemble().factor()
        ref = S.solve_batch(G, rtol=1e-8)
        W = S.matrix()
        L = np.stack([S.rhs(g) for g in G])
        for prec in ("tc", "mixed-tc", "mixed-fp16"):
            out = S.solve_batch(G, rtol=1e-8, precision=prec)
            R = L - out["density"] @ W
            rel = np.linalg.norm(R, axis=1) / np.linalg.norm(L, axis=1)
            assert rel.max() <= 1.05e-8, (prec, rel.max())
            d = np.linalg.norm(out["density"] - ref["density"], axis=1) / np.linalg.norm(ref["density"], axis=1)
            assert d.max() <= 1e-6, (prec, d.max())
