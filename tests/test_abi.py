"""C-ABI checks that need no GPU: the library builds and loads, exports every
symbol include/msbem.h declares, and its host topology (the same code that
msbem_upload runs) reproduces the oracle's dof numbering bit for bit."""
import math
import re
import os

import numpy as np
import pytest

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import build as B
from paper_2310_09204_gb300 import workloads as WL
from oracle.topology import Topology

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return M.lib()


def test_exports_every_declared_symbol(L):
    hdr = open(os.path.join(ROOT, "include", "msbem.h")).read()
    names = re.findall(r"^\w[\w\s\*]*?\b(msbem_\w+)\s*\(", hdr, re.M)
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("geom", [WL.flat_config(), WL.book(8, 2), WL.disk(5, fin=True), WL.bowtie(6, 2),
                                  WL.panels(7, n=6), WL.panels(5, n=6),
                                  WL.book_config()], ids=lambda g: g.name)
def test_dof_map_matches_oracle(L, geom):
    n, v, s = M.msbem_mesh_dofs(geom.xyz, geom.tri)
    top = Topology(geom.xyz, geom.tri)
    assert n == top.ndof
    assert np.array_equal(v, top.dof_vertex)
    assert np.array_equal(s, top.dof_sector)


def test_rejects_bad_meshes(L):
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0.5], [0, -1, 0.5]], float)
    with pytest.raises(M.MsbemError) as e:
        M.msbem_mesh_dofs(xyz, np.array([[0, 1, 2], [0, 3, 4]]))
    assert e.value.status == -3                               # point contact
    with pytest.raises(M.MsbemError) as e:
        M.msbem_mesh_dofs(xyz, np.array([[0, 1, 2], [1, 2, 0]]))
    assert e.value.status == -2                               # duplicate triangle
    with pytest.raises(M.MsbemError) as e:
        M.msbem_mesh_dofs(np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0]], float), np.array([[0, 1, 2]]))
    assert e.value.status == -2                               # degenerate
    with pytest.raises(M.MsbemError) as e:
        M.msbem_mesh_dofs(xyz, np.array([[0, 1, 7]]))
    assert e.value.status == -1                               # bad vertex id


def test_single_triangle_has_no_dofs(L):
    n, v, s = M.msbem_mesh_dofs(np.eye(3), np.array([[0, 1, 2]]))
    assert n == 0


@pytest.mark.parametrize("geom", [WL.cube_midplanes(4, 2), WL.cube_midplanes(6, 2), WL.book(4, 2),
                                  WL.panels(7, n=4)], ids=lambda g: g.name)
def test_cells_match_oracle(L, geom):
    """The library's closed cells (its own C++ code) equal the oracle's bit for bit."""
    from oracle.topology import Topology
    Zg = M.msbem_mesh_cells(geom.xyz, geom.tri)
    Zo = Topology(geom.xyz, geom.tri).cells()
    assert Zg.shape == Zo.shape
    assert np.array_equal(Zg, Zo)


def test_factor_group_rejects_empty_groups(L):
    # argument checks that return before any device call
    import ctypes
    assert L.msbem_factor_group(None, 1, None, None) == -1
    geoms = (ctypes.c_void_p * 1)(None)
    assert L.msbem_factor_group(ctypes.cast(geoms, ctypes.c_void_p), 0, None, None) == -1
    assert L.msbem_factor_group(ctypes.cast(geoms, ctypes.c_void_p), 1, None, None) == -1


@pytest.mark.parametrize("ang,ok", [(0.0, False), (5e-11, False), (2e-10, True), (1e-8, True), (1e-3, True),
                                    (math.pi, True), (2 * math.pi - 5e-11, False), (2 * math.pi - 2e-10, True)])
@pytest.mark.parametrize("scale", [1.0, 3.0])
def test_two_triangle_fold_threshold(L, ang, ok, scale):
    # two triangles on one edge, the second turned by `ang` about it: they
    # overlap (NONCONFORMING) when the angle is within 1e-10 of 0 or 2 pi
    xyz = np.array([[0.1, 0.2, 0.3], [0.1, 1.7, 0.3], [1.3, 0.9, 0.3],
                    [0.1 + scale * math.cos(ang), 0.9, 0.3 + scale * math.sin(ang)]])
    tri = np.array([[0, 1, 2], [0, 1, 3]])
    if ok:
        n, v, s = M.msbem_mesh_dofs(xyz, tri)
        assert n == 0          # an open screen of two triangles has no interior vertex
    else:
        with pytest.raises(M.MsbemError) as e:
            M.msbem_mesh_dofs(xyz, tri)
        assert e.value.status == -2


def test_test_hooks_check_their_arguments():
    """The error-path test hooks reject bad arguments before any CUDA call."""
    M.lib()
    assert M.msbem_test_fail_alloc(-2) == -1
    assert M.msbem_test_fail_alloc(-1) == 0          # off: nothing pending
    assert M.msbem_test_expire_waits(-1) == -1
