"""Failure detection without a GPU fault.

* A bounded device-side wait that runs out: the test hook
  msbem_test_expire_waits makes every CTA of the matrix-vector product kernels
  (CUDA-core and tensor-core) wait about a millisecond on a device flag that
  nothing sets.  Each CTA then takes its timeout path -- lets its copies in
  flight land, frees its tensor memory, raises the error flag and returns --
  and the call reports DEVICE_TIMEOUT.  The context must stay usable: after
  the hook is cleared the same calls give bit for bit the results they gave
  before.
* An allocation that fails on the host side: msbem_test_fail_alloc makes the
  k-th device allocation of the library fail as if the device were out of
  memory.  The assembly and the preconditioner set-up must return OOM, leave
  the geometry not assembled (not factored), and a later clean call must give
  the same results as a geometry that never failed.
"""
import numpy as np
import pytest

import paper_2310_09204_gb300 as M
from paper_2310_09204_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

DEVICE_TIMEOUT, OOM, NOT_READY = -7, -4, -9


def test_expired_wait_reports_timeout_and_context_recovers():
    geom = WL.flat_config()
    X = np.random.default_rng(3).standard_normal((3, 225))
    with M.Solver(geom) as S:
        S.assemble().factor()
        Y0, _ = S.apply(X, "df")
        T0, _ = S.apply(X, "tc")
        ref = S.solve(geom.g)
        try:
            assert M.msbem_test_expire_waits(1_000_000) == 0        # 1 ms
            for prec in ("df", "tc"):
                with pytest.raises(M.MsbemError) as ei:
                    S.apply(X, prec)
                assert ei.value.status == DEVICE_TIMEOUT, prec
            out = S.solve(geom.g, raise_on_status=False)
            assert out["status"] == DEVICE_TIMEOUT
        finally:
            assert M.msbem_test_expire_waits(0) == 0
        Y1, _ = S.apply(X, "df")
        T1, _ = S.apply(X, "tc")
        assert np.array_equal(Y0, Y1) and np.array_equal(T0, T1)
        out = S.solve(geom.g)
        assert out["iters"] == ref["iters"]
        assert np.array_equal(out["density"], ref["density"])


def test_injected_allocation_failure_in_assembly_and_setup():
    geom = WL.book(8, 2, jitter=False)
    with M.Solver(geom) as S0:
        S0.assemble().factor()
        ref = S0.solve(geom.g)
    with M.Solver(geom) as S:
        # the assembly's first allocation (the pair matrix V) fails
        try:
            assert M.msbem_test_fail_alloc(0) == 0
            with pytest.raises(M.MsbemError) as ei:
                S.assemble()
            assert ei.value.status == OOM
        finally:
            M.msbem_test_fail_alloc(-1)
        with pytest.raises(M.MsbemError) as ei:
            S.factor()
        assert ei.value.status == NOT_READY           # left unassembled
        S.assemble()
        # each allocation of the preconditioner set-up in turn
        failures = 0
        for after in range(24):
            M.msbem_test_fail_alloc(after)
            try:
                S.factor()
                failed = False
            except M.MsbemError as e:
                assert e.status == OOM, (after, e)
                failed = True
            finally:
                M.msbem_test_fail_alloc(-1)
            if not failed:
                break
            failures += 1
            with pytest.raises(M.MsbemError) as ei:
                S.solve(geom.g)
            assert ei.value.status == NOT_READY       # left unfactored
        assert failures >= 3
        S.factor()
        out = S.solve(geom.g)
    assert out["iters"] == ref["iters"]
    assert np.array_equal(out["density"], ref["density"])

