"""Host logic of the Python binding's shared contexts (no GPU): the C calls
are replaced by a fake that tracks contexts and geometries, so that freeing a
geometry twice, or after its context, is caught whatever the order in which
Solvers are closed or collected."""
import gc
import itertools

import pytest

import paper_2310_09204_gb300 as M


class FakeLib:
    def __init__(self):
        self.ctx_alive = set()
        self.geom_ctx = {}          # live geometry -> its context
        self.errors = []
        self.ids = itertools.count(1)

    def msbem_destroy(self, ctx):
        c = ctx.value
        if c not in self.ctx_alive:
            self.errors.append(("destroy of a dead context", c))
        self.ctx_alive.discard(c)
        for g, gc_ in list(self.geom_ctx.items()):
            if gc_ == c:
                del self.geom_ctx[g]
        return 0

    def msbem_geom_free(self, geom):
        g = geom.value
        if g not in self.geom_ctx:
            self.errors.append(("free of a dead geometry", g))
            return -1
        del self.geom_ctx[g]
        return 0

    def msbem_last_error(self, ctx):
        return b"fake"


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()

    def create(device=0, stream=0):
        c = next(f.ids)
        f.ctx_alive.add(c)
        return M.ctypes.c_void_p(c)

    def upload(ctx, *a):
        g = next(f.ids)
        f.geom_ctx[g] = ctx.value
        return M.ctypes.c_void_p(g)

    monkeypatch.setattr(M, "lib", lambda: f)
    monkeypatch.setattr(M, "msbem_create", create)
    monkeypatch.setattr(M, "msbem_upload", upload)
    monkeypatch.setattr(M, "msbem_ndofs", lambda g: 0)
    yield f
    # Solvers still reachable (e.g. from a failed test's traceback) must never
    # reach the real library with the fake handles once the fake is removed
    for obj in gc.get_objects():
        if type(obj) is M.Solver:
            obj.ctx, obj.geom, obj._root = None, None, None


def _group(n):
    owner = M.Solver(None, stream=0)
    owner.upload(None, None, None, None, None, None)
    rest = [M.Solver(None, share=owner) for _ in range(n - 1)]
    for S in rest:
        S.upload(None, None, None, None, None, None)
    return [owner] + rest


@pytest.mark.parametrize("order", ["sharers_first", "owner_first", "mixed"])
def test_close_orders(fake, order):
    group = _group(4)
    if order == "sharers_first":
        seq = group[1:] + group[:1]
    elif order == "owner_first":
        seq = group
    else:
        seq = [group[2], group[0], group[3], group[1]]
    for S in seq:
        S.close()
    for S in group:
        S.close()                      # closing again is harmless
    assert fake.errors == []
    assert not fake.ctx_alive and not fake.geom_ctx


def test_sharer_keeps_owner_alive(fake):
    group = _group(3)
    sharer = group[2]
    del group
    gc.collect()
    # the other sharer was collected (its geometry freed); the owner lives on
    # through the remaining sharer, with its context and geometry
    assert len(fake.ctx_alive) == 1 and len(fake.geom_ctx) == 2
    # closing the last sharer drops the last reference to the owner, which
    # then destroys the context
    sharer.close()
    gc.collect()
    assert not fake.ctx_alive and not fake.geom_ctx and fake.errors == []


def test_share_of_a_sharer_uses_the_owner(fake):
    group = _group(2)
    third = M.Solver(None, share=group[1])
    assert third.ctx.value == group[0].ctx.value and third._root is group[0]
    group[0].close()
    assert third.ctx is None and third.geom is None
    with pytest.raises(ValueError):
        M.Solver(None, share=group[1])
    assert fake.errors == []


def test_factor_group_rejects_closed_solvers(fake):
    group = _group(2)
    group[1].close()
    with pytest.raises(ValueError):
        M.msbem_factor_group(group)
    with pytest.raises(ValueError):
        M.msbem_factor_group([])
    group[0].close()
    assert fake.errors == []


def test_noalloc_binding_rejects_host_and_mistyped_tensors(monkeypatch):
    """msbem_spd_inverse_noalloc's binding refuses what raw pointers cannot
    describe (host memory, wrong dtype or shape) before reaching the library:
    a library call would fail this test."""
    import torch

    class NoCall:
        def __getattr__(self, name):
            raise AssertionError(f"library called: {name}")

    monkeypatch.setattr(M, "_lib", NoCall())
    eye = torch.eye(4, dtype=torch.float64)
    for A, Ainv in ((eye, eye), (eye.float(), eye), (torch.zeros(4, 3, dtype=torch.float64),) * 2):
        with pytest.raises(ValueError):
            M.msbem_spd_inverse_noalloc(A, Ainv)


def test_inverse_group_binding_rejects_before_the_library(monkeypatch):
    """msbem_spd_inverse_group's binding refuses an empty list, host or
    mistyped or non-square matrices, a repeated matrix and an unknown
    precision before reaching the library (a library call fails this test)."""
    import torch

    class NoCall:
        def __getattr__(self, name):
            raise AssertionError(f"library called: {name}")

    monkeypatch.setattr(M, "_lib", NoCall())
    eye = torch.eye(4, dtype=torch.float64)
    with pytest.raises(ValueError):
        M.msbem_spd_inverse_group([])
    for mats in ([eye], [eye.float()], [torch.zeros(4, 3, dtype=torch.float64)], [eye, eye]):
        with pytest.raises(ValueError):
            M.msbem_spd_inverse_group(mats)
    with pytest.raises(ValueError):
        M.msbem_spd_inverse_group([eye], precision="bf16")
