"""GB300-native multiscreen hypersingular BEM: Python binding of libmsbem.

Argument marshalling only: every step of the solve runs in the CUDA library
(``csrc/``, C ABI in ``include/msbem.h``).  There is no CPU fallback; if the
library is missing or cannot be loaded, ``lib()`` raises.

Low-level names mirror the C ABI (``msbem_create``, ``msbem_upload``, ...);
``Solver`` wraps one context + one geometry for convenience.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmsbem.so")
_lib = None

MSBEM_OK = 0
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "NONCONFORMING", -3: "POINT_CONTACT", -4: "OOM",
          -5: "NOT_CONVERGED", -6: "BREAKDOWN", -7: "DEVICE_TIMEOUT", -8: "CUDA_ERROR",
          -9: "NOT_READY"}


class MsbemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class AssembleOpts(ctypes.Structure):
    _fields_ = [("ss_order", ctypes.c_int), ("far_kernel", ctypes.c_int), ("panel_rows", ctypes.c_int64)]


class PrecondOpts(ctypes.Structure):
    _fields_ = [("wire_basket", ctypes.c_int), ("use_coarse", ctypes.c_int), ("precision", ctypes.c_int)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("maxit", ctypes.c_int), ("fixed_iters", ctypes.c_int),
                ("precondition", ctypes.c_int), ("precision", ctypes.c_int), ("inner_rtol", ctypes.c_double),
                ("density_tol", ctypes.c_double)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_double), ("precision", ctypes.c_int), ("rtol", ctypes.c_double),
                ("inner_rtol", ctypes.c_double), ("maxit", ctypes.c_int), ("chunk", ctypes.c_int),
                ("admission_threads", ctypes.c_int), ("density_tol", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("admissions", ctypes.c_int64),
                ("evictions", ctypes.c_int64), ("resident_bytes", ctypes.c_double),
                ("resident_geometries", ctypes.c_int), ("far_ms", ctypes.c_double), ("far_pairs", ctypes.c_int64),
                ("assemble_ms", ctypes.c_double), ("factor_ms", ctypes.c_double), ("launches", ctypes.c_int64)]


#: arithmetic of the solve's matrix-vector products (msbem_solve_opts.precision)
PRECISION = {"df": 0, "fp64": 1, "mixed": 2, "tc": 3, "mixed-tc": 4, "mixed-fp16": 5}


def lib():
    """Load libmsbem.so (built by ``paper_2310_09204_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libmsbem.so not built ({LIB_PATH}); run paper_2310_09204_gb300/build.py")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "msbem_create": ([ctypes.POINTER(P), i32, P], i32),
        "msbem_destroy": ([P], i32),
        "msbem_last_error": ([P], ctypes.c_char_p),
        "msbem_upload": ([P, P, i64, P, i64, P, i64, P, i64, P, P, ctypes.POINTER(P)], i32),
        "msbem_geom_free": ([P], i32),
        "msbem_ndofs": ([P, ctypes.POINTER(i64)], i32),
        "msbem_dof_map": ([P, P, P], i32),
        "msbem_split_info": ([P, P, P, P, P], i32),
        "msbem_assemble": ([P, ctypes.POINTER(AssembleOpts)], i32),
        "msbem_copy_matrix": ([P, i64, i64, P], i32),
        "msbem_rhs": ([P, P, P], i32),
        "msbem_factor": ([P, ctypes.POINTER(PrecondOpts)], i32),
        "msbem_factor_group": ([P, i32, ctypes.POINTER(PrecondOpts), P], i32),
        "msbem_solve": ([P, P, ctypes.POINTER(SolveOpts), P, ctypes.POINTER(i32), P, i32,
                         ctypes.POINTER(d)], i32),
        "msbem_last_timings": ([P, P], i32),
        "msbem_counters": ([P, ctypes.POINTER(i64), ctypes.POINTER(i64)], i32),
        "msbem_spd_inverse_noalloc": ([P, i64, P, P], i32),
        "msbem_spd_inverse_group": ([P, P, P, i32, i32, P], i32),
        "msbem_solve_batch": ([P, P, i32, ctypes.POINTER(SolveOpts), P, P, P, P], i32),
        "msbem_apply": ([P, P, i32, i32, P, P], i32),
        "msbem_cells": ([P, ctypes.POINTER(i32), P, ctypes.POINTER(ctypes.c_double)], i32),
        "msbem_dl_potential": ([P, P, P, i64, i32, P, P], i32),
        "msbem_mesh_cells": ([P, i64, P, i64, ctypes.POINTER(i32), P, i64], i32),
        "msbem_server_create": ([P, ctypes.POINTER(ServerOpts), ctypes.POINTER(P)], i32),
        "msbem_server_destroy": ([P], i32),
        "msbem_server_add_geometry": ([P, ctypes.c_uint64, P, i64, P, i64, P, i64, P, i64, P, P], i32),
        "msbem_server_now": ([], ctypes.c_double),
        "msbem_server_footprint": ([P, ctypes.c_uint64], ctypes.c_double),
        "msbem_server_submit": ([P, ctypes.c_uint64, P, P, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)], i32),
        "msbem_server_progress": ([P, i32, ctypes.POINTER(i32)], i32),
        "msbem_server_result": ([P, ctypes.c_uint64, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(i32)], i32),
        "msbem_server_stats_get": ([P, ctypes.POINTER(ServerStats)], i32),
        "msbem_mesh_dofs": ([P, i64, P, i64, ctypes.POINTER(i64), P, P, i64, ctypes.c_char_p, i32], i32),
        "msbem_test_fail_alloc": ([i64], i32),
        "msbem_test_expire_waits": ([i64], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return _lib


def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a.data_ptr())


def _check(ctx, st: int):
    if st != MSBEM_OK:
        raise MsbemError(st, lib().msbem_last_error(ctx).decode())


# ---- low-level wrappers with the C names ------------------------------------

def msbem_create(device: int = 0, stream: int = 0):
    h = ctypes.c_void_p()
    st = lib().msbem_create(ctypes.byref(h), device, stream)
    if st != MSBEM_OK:
        raise MsbemError(st, "msbem_create failed")
    return h


def msbem_destroy(ctx):
    return lib().msbem_destroy(ctx)


def msbem_upload(ctx, xyz, tri, coarse_xyz, coarse_tri, parent, patch):
    xyz = np.ascontiguousarray(xyz, np.float64)
    tri = np.ascontiguousarray(tri, np.int32)
    cxyz = np.ascontiguousarray(coarse_xyz, np.float64)
    ctri = np.ascontiguousarray(coarse_tri, np.int32)
    parent = np.ascontiguousarray(parent, np.int32)
    patch = np.ascontiguousarray(patch, np.int32)
    g = ctypes.c_void_p()
    st = lib().msbem_upload(ctx, _ptr(xyz), xyz.shape[0], _ptr(tri), tri.shape[0], _ptr(cxyz),
                            cxyz.shape[0], _ptr(ctri), ctri.shape[0], _ptr(parent), _ptr(patch),
                            ctypes.byref(g))
    _check(ctx, st)
    return g


def msbem_mesh_cells(xyz, tri):
    """Host-only closed cells of a mesh: Z (N x ncells), the cells' indicators in the psi basis."""
    xyz = np.ascontiguousarray(xyz, np.float64)
    tri = np.ascontiguousarray(tri, np.int32)
    n = msbem_mesh_dofs(xyz, tri)[0]
    nc = ctypes.c_int()
    st = lib().msbem_mesh_cells(_ptr(xyz), xyz.shape[0], _ptr(tri), tri.shape[0], ctypes.byref(nc), None, 0)
    if st != MSBEM_OK:
        raise MsbemError(st, "msbem_mesh_cells")
    Z = np.zeros((n, nc.value))
    if nc.value:
        lib().msbem_mesh_cells(_ptr(xyz), xyz.shape[0], _ptr(tri), tri.shape[0], ctypes.byref(nc), _ptr(Z), Z.size)
    return Z


def msbem_mesh_dofs(xyz, tri):
    """Host-only topology of a mesh: (ndof, vertex_of_dof, sector_of_dof)."""
    xyz = np.ascontiguousarray(xyz, np.float64)
    tri = np.ascontiguousarray(tri, np.int32)
    n = ctypes.c_int64()
    buf = ctypes.create_string_buffer(256)
    st = lib().msbem_mesh_dofs(_ptr(xyz), xyz.shape[0], _ptr(tri), tri.shape[0], ctypes.byref(n),
                               None, None, 0, buf, 256)
    if st != MSBEM_OK:
        raise MsbemError(st, buf.value.decode())
    v = np.zeros(n.value, np.int32)
    s = np.zeros(n.value, np.int32)
    st = lib().msbem_mesh_dofs(_ptr(xyz), xyz.shape[0], _ptr(tri), tri.shape[0], ctypes.byref(n),
                               _ptr(v), _ptr(s), n.value, buf, 256)
    if st != MSBEM_OK:
        raise MsbemError(st, buf.value.decode())
    return int(n.value), v, s


NOALLOC_MAX_N = 2048


def msbem_spd_inverse_noalloc(A, Ainv, stream: int = 0) -> int:
    """Inverse of an SPD matrix without any device allocation; returns the C
    status (0 on success, MSBEM_BREAKDOWN for a non-positive pivot).

    A and Ainv are CUDA tensors of shape (n, n), float64, contiguous, on one
    device (Ainv may be A itself: in place); stream is a raw cudaStream_t of
    that device (0: the legacy default stream).  Anything else raises
    ValueError before the library is called, since the C side only sees raw
    pointers and would read or write past a smaller or differently laid out
    tensor.  The call runs with A's device current, so the library uses that
    device's scratch array."""
    import torch
    for name, t in (("A", A), ("Ainv", Ainv)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"msbem_spd_inverse_noalloc: {name} must be a CUDA tensor")
        if t.dtype != torch.float64:
            raise ValueError(f"msbem_spd_inverse_noalloc: {name} must be float64, got {t.dtype}")
        if t.dim() != 2 or t.shape[0] != t.shape[1]:
            raise ValueError(f"msbem_spd_inverse_noalloc: {name} must be square, got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"msbem_spd_inverse_noalloc: {name} must be contiguous")
    if A.shape != Ainv.shape:
        raise ValueError(f"msbem_spd_inverse_noalloc: shapes differ: {tuple(A.shape)} and {tuple(Ainv.shape)}")
    if A.device != Ainv.device:
        raise ValueError(f"msbem_spd_inverse_noalloc: tensors on {A.device} and {Ainv.device}")
    n = int(A.shape[0])
    if not 1 <= n <= NOALLOC_MAX_N:
        raise ValueError(f"msbem_spd_inverse_noalloc: order {n} outside 1..{NOALLOC_MAX_N}")
    with torch.cuda.device(A.device):
        return lib().msbem_spd_inverse_noalloc(_ptr(A), n, _ptr(Ainv), stream)


def msbem_spd_inverse_group(mats, precision: str = "df", device: int = 0):
    """In-place inverses of a list of SPD matrices (CUDA float64 tensors,
    square, contiguous, on `device`) by the grouped Gauss-Jordan recursion of
    the preconditioner set-up; precision "df" (tensor-core update, double-float
    accuracy) or "fp32".  Returns the per-matrix C status list (0, or
    MSBEM_BREAKDOWN for a matrix whose recursion met a non-positive pivot).
    Shapes, dtypes and devices are checked before the library is called."""
    import torch
    if precision not in ("df", "fp32"):
        raise ValueError(f"msbem_spd_inverse_group: precision must be 'df' or 'fp32', got {precision!r}")
    mats = list(mats)
    if not mats:
        raise ValueError("msbem_spd_inverse_group: no matrices")
    dev = torch.device("cuda", device)
    for i, t in enumerate(mats):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device != dev:
            raise ValueError(f"msbem_spd_inverse_group: matrix {i} must be a CUDA tensor on {dev}")
        if t.dtype != torch.float64 or t.dim() != 2 or t.shape[0] != t.shape[1] or t.shape[0] < 1:
            raise ValueError(f"msbem_spd_inverse_group: matrix {i} must be square float64, got {t.dtype} {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"msbem_spd_inverse_group: matrix {i} must be contiguous")
    ptrs = set(t.data_ptr() for t in mats)
    if len(ptrs) != len(mats):
        raise ValueError("msbem_spd_inverse_group: repeated matrix")
    k = len(mats)
    A = (ctypes.c_void_p * k)(*[t.data_ptr() for t in mats])
    n = (ctypes.c_int64 * k)(*[int(t.shape[0]) for t in mats])
    st = (ctypes.c_int * k)()
    with torch.cuda.device(dev):
        ctx = msbem_create(device, torch.cuda.current_stream(dev).cuda_stream)
        try:
            rc = lib().msbem_spd_inverse_group(ctx, A, n, k, 0 if precision == "df" else 1, st)
            if rc not in (MSBEM_OK, -6):   # -6: BREAKDOWN, reported per matrix
                _check(ctx, rc)
        finally:
            lib().msbem_destroy(ctx)
    return list(st)


def msbem_test_fail_alloc(after: int) -> int:
    """Test hook: the (after + 1)-th device allocation of the library from now
    fails as if out of memory, once (-1: off).  Returns the C status."""
    return lib().msbem_test_fail_alloc(int(after))


def msbem_test_expire_waits(ns: int) -> int:
    """Test hook: the product kernels' bounded waits run out after ns
    nanoseconds on a flag nothing sets (0: off; current device)."""
    return lib().msbem_test_expire_waits(int(ns))


def msbem_factor_group(solvers, wire_basket: int = 0, use_coarse: int = 1, precision: str = "df"):
    """Factor the preconditioners of several Solvers that share one context
    (Solver(share=...)) with one grouped inversion; returns the per-geometry
    C statuses (0, or MSBEM_BREAKDOWN) and raises when any is not 0."""
    solvers = list(solvers)
    if not solvers:
        raise ValueError("msbem_factor_group: no solvers")
    if any(S.ctx is None or S.geom is None for S in solvers):
        raise ValueError("msbem_factor_group: a Solver is closed or has no geometry")
    geoms = (ctypes.c_void_p * len(solvers))(*[S.geom.value for S in solvers])
    status = np.zeros(len(solvers), np.int32)
    o = PrecondOpts(wire_basket, use_coarse, {"df": 0, "fp32": 1}[precision])
    _check(solvers[0].ctx, lib().msbem_factor_group(ctypes.cast(geoms, ctypes.c_void_p), len(solvers),
                                                    ctypes.byref(o), _ptr(status)))
    return status


def msbem_ndofs(geom) -> int:
    n = ctypes.c_int64()
    lib().msbem_ndofs(geom, ctypes.byref(n))
    return int(n.value)


class Solver:
    """One context + one uploaded geometry.  share=another Solver: use its
    context (and memory pool) instead of a new one; closing this Solver then
    frees only its geometry.  The Solver that created the context stays alive
    while any Solver shares it, and closing it first also invalidates the
    geometries of the Solvers sharing its context (the context frees them)."""

    def __init__(self, geom=None, device: int = 0, stream: int | None = None, share=None, **arrays):
        self.ctx, self.geom, self._owns_ctx = None, None, False
        self._sharers = weakref.WeakSet()   # Solvers using this one's context
        self._root = None                   # the Solver owning the shared context
        if share is not None:
            root = share._root if share._root is not None else share
            if root.ctx is None:
                raise ValueError("Solver(share=...): that Solver is closed")
            self.ctx, self._root = root.ctx, root
            root._sharers.add(self)
        else:
            if stream is None:
                try:
                    import torch
                    stream = torch.cuda.current_stream(device).cuda_stream
                except Exception:  # pragma: no cover - torch without CUDA
                    stream = 0
            self.ctx, self._owns_ctx = msbem_create(device, stream), True
        self.geom = None
        if geom is not None:
            self.upload(geom.xyz, geom.tri, geom.coarse_xyz, geom.coarse_tri, geom.parent, geom.patch)
        elif arrays:
            self.upload(**arrays)

    def upload(self, xyz, tri, coarse_xyz, coarse_tri, parent, patch):
        self.free_geometry()
        self.geom = msbem_upload(self.ctx, xyz, tri, coarse_xyz, coarse_tri, parent, patch)
        self.n = msbem_ndofs(self.geom)
        return self

    def close(self):
        if self.ctx is not None:
            if self._owns_ctx:
                # msbem_destroy frees every geometry of the context, the
                # sharers' included: they must not free theirs again
                for other in list(self._sharers):
                    other.ctx, other.geom = None, None
                self._sharers.clear()
                lib().msbem_destroy(self.ctx)
            else:
                self.free_geometry()
                if self._root is not None:
                    self._root._sharers.discard(self)
            self.ctx = None
            self.geom = None
            self._root = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- queries
    def dof_map(self):
        v = np.zeros(self.n, np.int32)
        s = np.zeros(self.n, np.int32)
        _check(self.ctx, lib().msbem_dof_map(self.geom, _ptr(v), _ptr(s)))
        return v, s

    def split_info(self):
        vals = [ctypes.c_int64() for _ in range(4)]
        _check(self.ctx, lib().msbem_split_info(self.geom, *[ctypes.byref(v) for v in vals]))
        return dict(zip(("n_faces", "n_wire_basket", "n_coarse", "max_face"), (v.value for v in vals)))

    def counters(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(self.ctx, lib().msbem_counters(self.geom, ctypes.byref(a), ctypes.byref(b)))
        return {"launches": int(a.value), "far_pairs": int(b.value)}

    def free_geometry(self):
        if self.geom is not None:
            _check(self.ctx, lib().msbem_geom_free(self.geom))
            self.geom = None

    def timings(self):
        t = np.zeros(5)
        lib().msbem_last_timings(self.geom, _ptr(t))
        return dict(zip(("far_ms", "near_ms", "contract_ms", "factor_ms", "solve_ms"), t.tolist()))

    # --- the hot path
    def assemble(self, ss_order: int = 5, far_kernel: int = 0, panel_rows: int = 0):
        """W; panel_rows > 0 forces the pair matrix V into row panels of that
        many triangles (0: in one piece when it fits)."""
        o = AssembleOpts(ss_order, far_kernel, panel_rows)
        _check(self.ctx, lib().msbem_assemble(self.geom, ctypes.byref(o)))
        return self

    def matrix(self, row0: int = 0, nrows: int | None = None, out=None):
        nrows = self.n - row0 if nrows is None else nrows
        if out is None:
            out = np.empty((nrows, self.n), np.float64)
        _check(self.ctx, lib().msbem_copy_matrix(self.geom, row0, nrows, _ptr(out)))
        return out

    def rhs(self, g, out=None):
        gv = np.ascontiguousarray(g, np.float64)
        if out is None:
            out = np.empty(self.n, np.float64)
        _check(self.ctx, lib().msbem_rhs(self.geom, _ptr(gv), _ptr(out)))
        return out

    def factor(self, wire_basket: int = 0, use_coarse: int = 1, precision: str = "df"):
        """Set up M(H;h).  precision "df" (default): double-float inverses;
        "fp32": FP32 inverses of the face and wire-basket blocks (for the
        mixed-precision solves)."""
        o = PrecondOpts(wire_basket, use_coarse, {"df": 0, "fp32": 1}[precision])
        _check(self.ctx, lib().msbem_factor(self.geom, ctypes.byref(o)))
        return self

    def potential(self, density, targets, refine: int = 0, out=None):
        """U = DL Phi at target points (M x 3); returns (U, kernel_ms)."""
        if isinstance(density, np.ndarray):
            density = np.ascontiguousarray(density, np.float64)
        if isinstance(targets, np.ndarray):
            targets = np.ascontiguousarray(targets, np.float64).reshape(-1, 3)
        M = targets.shape[0]
        if out is None:
            out = np.empty(M, np.float64)
        ms = ctypes.c_double()
        _check(self.ctx, lib().msbem_dl_potential(self.geom, _ptr(density), _ptr(targets), M, refine, _ptr(out),
                                                  ctypes.byref(ms)))
        return out, float(ms.value)

    def cells(self):
        """(Z, rho): the closed cells' indicators in the psi basis (N x ncells)
        and the augmentation weight (after assemble)."""
        nc = ctypes.c_int()
        rho = ctypes.c_double()
        _check(self.ctx, lib().msbem_cells(self.geom, ctypes.byref(nc), None, ctypes.byref(rho)))
        Z = np.zeros((self.n, nc.value))
        if nc.value:
            _check(self.ctx, lib().msbem_cells(self.geom, None, _ptr(Z), None))
        return Z, rho.value

    def apply(self, X, precision="df", out=None):
        """Y = W X for up to 16 vectors (rows of X); returns (Y, kernel_ms)."""
        prec = {"df": 0, "fp64": 1, "fp32": 2, "tc": 3, "fp16-tc": 4}[precision]
        if isinstance(X, np.ndarray):
            X = np.ascontiguousarray(X, np.float64).reshape(-1, self.n)
        k = X.shape[0]
        if out is None:
            out = np.empty((k, self.n), np.float64)
        ms = ctypes.c_double()
        _check(self.ctx, lib().msbem_apply(self.geom, _ptr(X), k, prec, _ptr(out), ctypes.byref(ms)))
        return out, float(ms.value)

    def solve_batch(self, G, rtol: float = 1e-8, maxit: int = 1000, fixed: bool = False,
                    precondition: bool = True, out=None, raise_on_status=True, precision="df",
                    inner_rtol: float = 0.0, density_tol: float = 0.0):
        """k solves sharing the matrix-vector products; G is k x 3.
        density_tol (mixed precisions): also stop only when the refinement's
        estimated relative error is below it (0: residual test alone)."""
        G = np.ascontiguousarray(G, np.float64).reshape(-1, 3)
        k = G.shape[0]
        if out is None:
            out = np.empty((k, self.n), np.float64)
        iters = np.zeros(k, np.int32)
        rel = np.zeros(k, np.float64)
        kap = np.zeros(k, np.float64)
        o = SolveOpts(rtol, maxit, int(fixed), int(precondition), PRECISION[precision], inner_rtol, density_tol)
        st = lib().msbem_solve_batch(self.geom, _ptr(G), k, ctypes.byref(o), _ptr(out), _ptr(iters),
                                     _ptr(rel), _ptr(kap))
        if raise_on_status:
            _check(self.ctx, st)
        return {"density": out, "iters": iters, "relres": rel, "kappa": kap, "status": st}

    def solve(self, g, rtol: float = 1e-8, maxit: int = 1000, fixed: bool = False,
              precondition: bool = True, out=None, hist_cap: int = 4096, raise_on_status=True,
              precision="df", inner_rtol: float = 0.0, density_tol: float = 0.0):
        """One solve.  precision: "df" (double-float products, default), "fp64"
        (the plain FP64 comparator) or "mixed" (FP32 inner PCG inside
        double-float iterative refinement; hist then holds the true relative
        residual after each refinement step and iters the inner iterations)."""
        gv = np.ascontiguousarray(g, np.float64)
        if out is None:
            out = np.empty(self.n, np.float64)
        it = ctypes.c_int()
        kap = ctypes.c_double()
        hist = np.full(hist_cap, np.nan)
        o = SolveOpts(rtol, maxit, int(fixed), int(precondition), PRECISION[precision], inner_rtol, density_tol)
        st = lib().msbem_solve(self.geom, _ptr(gv), ctypes.byref(o), _ptr(out), ctypes.byref(it),
                               _ptr(hist), hist_cap, ctypes.byref(kap))
        if raise_on_status:
            _check(self.ctx, st)
        n_it = int(it.value)
        nh = int(np.argmax(np.isnan(hist))) if np.isnan(hist).any() else hist_cap
        return {"density": out, "iters": n_it, "hist": hist[:nh].copy(),
                "kappa": float(kap.value), "status": st}


class Server:
    """The serving engine (msbem_server_*): geometries registered by key stay
    resident on the device once admitted; requests (key, g) are answered by a
    continuously refilled 16-slot multi-vector PCG per geometry."""

    def __init__(self, device: int = 0, stream=None, precision="mixed", rtol: float = 1e-8,
                 inner_rtol: float = 0.0, hbm_budget: float = 0.0, maxit: int = 1000, chunk: int = 4,
                 admission_threads: int = 0, density_tol: float = 0.0):
        self.ctx = msbem_create(device, stream)
        o = ServerOpts(float(hbm_budget), PRECISION[precision], rtol, inner_rtol, maxit, chunk, admission_threads,
                       density_tol)
        h = ctypes.c_void_p()
        st = lib().msbem_server_create(self.ctx, ctypes.byref(o), ctypes.byref(h))
        if st:
            msbem_destroy(self.ctx)
            raise MsbemError(st, "msbem_server_create failed")
        self.h = h.value
        self.ndof = {}

    def add_geometry(self, key: int, geom, ndof: int | None = None) -> None:
        """Register a geometry (host copies; nothing goes to the device until a
        request for it is admitted).  ndof: its dof count when the caller knows
        it already (else computed here from the mesh)."""
        xyz = np.ascontiguousarray(geom.xyz, np.float64)
        tri = np.ascontiguousarray(geom.tri, np.int32)
        cxyz = np.ascontiguousarray(geom.coarse_xyz, np.float64)
        ctri = np.ascontiguousarray(geom.coarse_tri, np.int32)
        par = np.ascontiguousarray(geom.parent, np.int32)
        pat = np.ascontiguousarray(geom.patch, np.int32)
        _check(self.ctx, lib().msbem_server_add_geometry(self.h, key, _ptr(xyz), len(xyz), _ptr(tri), len(tri),
                                                         _ptr(cxyz), len(cxyz), _ptr(ctri), len(ctri),
                                                         _ptr(par), _ptr(pat)))
        self.ndof[key] = int(ndof) if ndof is not None else msbem_mesh_dofs(xyz, tri)[0]

    def footprint(self, key: int) -> float:
        """Bytes the admission of geometry `key` asks of the HBM budget."""
        return float(lib().msbem_server_footprint(self.h, key))

    @staticmethod
    def now() -> float:
        return float(lib().msbem_server_now())

    def submit(self, key: int, g, out=None, t_arrival: float = 0.0) -> int:
        gv = np.ascontiguousarray(g, np.float64)
        rid = ctypes.c_uint64()
        _check(self.ctx, lib().msbem_server_submit(self.h, key, _ptr(gv), None if out is None else _ptr(out),
                                                   t_arrival, ctypes.byref(rid)))
        return int(rid.value)

    def progress(self, block: bool = False) -> int:
        n = ctypes.c_int()
        st = lib().msbem_server_progress(self.h, int(block), ctypes.byref(n))
        if st:
            raise MsbemError(st, "msbem_server_progress")
        return int(n.value)

    def result(self, rid: int) -> dict:
        st, it, rf = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        rel, lat = ctypes.c_double(), ctypes.c_double()
        _check(self.ctx, lib().msbem_server_result(self.h, rid, ctypes.byref(st), ctypes.byref(it),
                                                   ctypes.byref(rel), ctypes.byref(lat), ctypes.byref(rf)))
        return {"status": st.value, "iters": it.value, "relres": rel.value, "latency_ms": lat.value,
                "refinements": rf.value}

    def stats(self) -> dict:
        s = ServerStats()
        lib().msbem_server_stats_get(self.h, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().msbem_server_destroy(self.h)
            self.h = None
        if getattr(self, "ctx", None):
            msbem_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
