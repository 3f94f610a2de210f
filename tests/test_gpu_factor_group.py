"""One grouped inversion for the preconditioners of several geometries
(msbem_factor_group, the Sec. 5 blocks of every geometry in one sequence of
launches): the inverses are those of factoring each geometry alone, bit for
bit, and the sixteen hinged-panel instances, factored as one group, solve to
a true relative residual of 1e-8 with tensor-core products inside
double-float refinement."""
import numpy as np
import pytest

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import build as B
from paper_2310_09204_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

SMALL = [WL.panels(7, n=8, n_coarse=2), WL.book(8, 2, jitter=True, seed=3), WL.panels(11, n=12),
         WL.bowtie(6, 2), WL.cube_midplanes(6, 2)]


@pytest.fixture(scope="module", autouse=True)
def _build():
    B.build()
    M.lib()


def _group(geoms):
    first = M.Solver(geoms[0])
    return [first] + [M.Solver(g, share=first) for g in geoms[1:]]


def _close(group):
    for S in reversed(group):      # the context's owner last
        S.close()


def test_group_equals_alone():
    # a fixed number of PCG steps is a deterministic function of W and of the
    # inverses, so equal densities mean equal inverses
    alone = []
    for geom in SMALL:
        with M.Solver(geom) as S:
            S.assemble().factor()
            alone.append(S.solve(geom.g, rtol=0.0, maxit=6, fixed=True)["density"])
    group = _group(SMALL)
    try:
        for S in group:
            S.assemble()
        st = M.msbem_factor_group(group)
        assert st.tolist() == [0] * len(SMALL)
        for S, geom, ref in zip(group, SMALL, alone):
            out = S.solve(geom.g, rtol=0.0, maxit=6, fixed=True)["density"]
            assert np.array_equal(out, ref), geom.name
        # without the coarse space, and factored again in a different group
        st = M.msbem_factor_group(group[::-1], use_coarse=0)
        assert st.tolist() == [0] * len(SMALL)
        for S, geom in zip(group, SMALL):
            with M.Solver(geom) as A:
                A.assemble().factor(use_coarse=0)
                ref = A.solve(geom.g, rtol=0.0, maxit=6, fixed=True)["density"]
            assert np.array_equal(S.solve(geom.g, rtol=0.0, maxit=6, fixed=True)["density"], ref)
    finally:
        _close(group)


def test_group_rejects_bad_groups():
    group = _group(SMALL[:2])
    try:
        with pytest.raises(M.MsbemError) as e:
            M.msbem_factor_group([group[0], group[0]])
        assert e.value.status == -1                          # repeated geometry
        with pytest.raises(M.MsbemError) as e:
            M.msbem_factor_group(group)
        assert e.value.status == -9                          # not assembled
        with M.Solver(SMALL[2]) as other:
            other.assemble()
            group[0].assemble()
            with pytest.raises(M.MsbemError) as e:
                M.msbem_factor_group([group[0], other])
            assert e.value.status == -1                      # two contexts
    finally:
        _close(group)


def test_sixteen_instances_grouped_mixed_tc():
    geoms = WL.panels_config()
    group = _group(geoms)
    try:
        for S in group:
            S.assemble()
        assert (M.msbem_factor_group(group) == 0).all()
        worst = 0.0
        for S, geom in zip(group, geoms):
            rng = np.random.default_rng(geom.meta["seed"])
            G = rng.uniform(-1, 1, (4, 3))
            G[0] = geom.g
            mx = S.solve_batch(G, rtol=1e-8, precision="mixed-tc")
            Y, _ = S.apply(mx["density"])
            for c in range(len(G)):
                L = S.rhs(G[c])
                r = np.linalg.norm(L - Y[c]) / np.linalg.norm(L)
                worst = max(worst, r)
                assert r <= 1.05e-8, (geom.name, c, r)
        print("grouped factorisation, mixed-tc: worst true relative residual", worst)
    finally:
        _close(group)


def test_rejected_factor_keeps_inverses():
    # options are checked before anything of the geometry changes
    geom = SMALL[1]
    with M.Solver(geom) as S:
        S.assemble().factor()
        ref = S.solve(geom.g, rtol=0.0, maxit=6, fixed=True)["density"]
        with pytest.raises(M.MsbemError) as e:
            S.factor(wire_basket=2, use_coarse=0)
        assert e.value.status == -1
        out = S.solve(geom.g, rtol=0.0, maxit=6, fixed=True)["density"]
        assert np.array_equal(out, ref)
