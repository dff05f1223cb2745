"""Thin Python binding of the C ABI in ``include/ndhss.h``.

Argument marshalling only: every step of the preconditioner (tree, fronts,
apply, sparse product, GMRES) runs inside ``lib/libndhss.so``.  Functions
carry the C names.  Device buffers are torch CUDA tensors (PyTorch provides
memory and streams); host buffers are numpy arrays.  There is no CPU
fallback: if the library is missing the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

NDHSS_R64, NDHSS_C128 = 0, 1
NDHSS_FP64, NDHSS_FP32, NDHSS_FP32_TF32, NDHSS_FP32_BF16 = 0, 1, 2, 3
NODE_FIELDS = ("level", "parent", "child0", "child1", "i_off", "m_i", "b_off", "m_b",
               "x0", "x1", "y0", "y1", "axis", "cut")
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "SINGULAR", 4: "RANK_CAP", 5: "NOT_CONVERGED",
          6: "TIMEOUT", 7: "CUDA", 8: "INTERNAL"}

EXPORTED = ("ndhss_version", "ndhss_last_error", "ndhss_kernel_launches", "ndhss_build_tree", "ndhss_tree_sizes", "ndhss_tree_export",
            "ndhss_tree_destroy", "ndhss_factor", "ndhss_factor_stats_get", "ndhss_factor_get_block",
            "ndhss_factor_destroy", "ndhss_apply", "ndhss_apply_noalloc", "ndhss_spmv", "ndhss_gmres",
            "ndhss_testing_stall_apply", "ndhss_elem_qform", "ndhss_build_tree_batched", "ndhss_apply_multi",
            "ndhss_gmres_batched", "ndhss_measure_fma_peak")


class NdhssError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ndhss error {STATUS.get(code, code)}: {msg}")
        self.code = code


class FactorOpts(C.Structure):
    _fields_ = [("prec", C.c_int32), ("hss_levels", C.c_int32), ("eps_hss", C.c_double), ("beta", C.c_int32),
                ("k0", C.c_int32), ("r", C.c_int32), ("rank_cap", C.c_int32), ("panel", C.c_int32),
                ("seed", C.c_uint64), ("timing", C.c_int32), ("ulv", C.c_int32)]


class GmresOpts(C.Structure):
    _fields_ = [("restart", C.c_int32), ("maxit", C.c_int32), ("tol", C.c_double), ("timing", C.c_int32),
                ("conj_transpose", C.c_int32), ("inner", C.c_double), ("cycle_rtol", C.c_double)]


class GmresStats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("cycles", C.c_int32), ("converged", C.c_int32), ("pad", C.c_int32),
                ("true_relres", C.c_double), ("precond_relres", C.c_double), ("napply", C.c_int32),
                ("nspmv", C.c_int32), ("apply_ms", C.c_double), ("spmv_ms", C.c_double)]

    def as_dict(self):
        return dict(iters=self.iters, cycles=self.cycles, converged=bool(self.converged),
                    true_relres=self.true_relres, precond_relres=self.precond_relres, napply=self.napply,
                    nspmv=self.nspmv, apply_ms=self.apply_ms, spmv_ms=self.spmv_ms)


class FactorStats(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnodes", C.c_int32), ("depth", C.c_int32), ("front_elems", C.c_int64),
                ("apply_bytes", C.c_int64), ("factor_bytes", C.c_int64), ("factor_ms", C.c_double),
                ("kmax", C.c_int32), ("prec", C.c_int32), ("launches", C.c_int64),
                ("class_ms", C.c_double * 8), ("class_launches", C.c_int64 * 8), ("update_flops", C.c_double),
                ("tc_flops", C.c_double), ("host_setup_ms", C.c_double), ("host_tail_ms", C.c_double)]

    CLASSES = ("assemble", "scatter", "panel", "prep", "update", "finalize", "compress", "tensor")

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("class_ms", "class_launches")}
        d["class_ms"] = {c: self.class_ms[i] for i, c in enumerate(self.CLASSES)}
        d["class_launches"] = {c: self.class_launches[i] for i, c in enumerate(self.CLASSES)}
        return d


_lib = None


def load(path: str | None = None):
    """Load (never build) the shared library; raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (paper_2105_07791_gb300.build.build())")
    L = C.CDLL(path)
    P, I32, I64, V = C.c_void_p, C.c_int32, C.c_int64, C.c_void_p
    sig = {
        "ndhss_version": (C.c_char_p, []),
        "ndhss_last_error": (C.c_char_p, []),
        "ndhss_kernel_launches": (C.c_int64, []),
        "ndhss_measure_fma_peak": (I32, [I32, V, C.POINTER(C.c_double)]),
        "ndhss_build_tree": (I32, [I32, P, P, P, I32, C.POINTER(C.c_void_p)]),
        "ndhss_tree_sizes": (I32, [P, C.POINTER(I32), C.POINTER(I32), C.POINTER(I64), C.POINTER(I64)]),
        "ndhss_tree_export": (I32, [P] + [P] * 8),
        "ndhss_tree_destroy": (None, [P]),
        "ndhss_factor": (I32, [P, I32, P, P, P, C.POINTER(FactorOpts), V, C.POINTER(C.c_void_p)]),
        "ndhss_factor_stats_get": (I32, [P, C.POINTER(FactorStats)]),
        "ndhss_factor_get_block": (I32, [P, I32, I32, P, I64]),
        "ndhss_factor_destroy": (None, [P]),
        "ndhss_apply": (I32, [P, I32, P, I64, P, I64, V]),
        "ndhss_apply_noalloc": (I32, [P, P, P, V]),
        "ndhss_testing_stall_apply": (I32, [P]),
        "ndhss_elem_qform": (I32, [I32, P, I32, P, P, P, P, P, V]),
        "ndhss_spmv": (I32, [I32, I32, P, P, P, P, P, V]),
        "ndhss_gmres": (I32, [P, P, P, P, I32, P, I64, P, I64, C.POINTER(GmresOpts), C.POINTER(GmresStats), V]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(code):
    if code != 0:
        raise NdhssError(code, load().ndhss_last_error().decode())


def _ptr(a):
    """Raw address of a torch tensor or numpy array (must be contiguous)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"] and not a.flags["F_CONTIGUOUS"]:
        raise ValueError("array must be contiguous")
    return C.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def ndhss_version() -> str:
    return load().ndhss_version().decode()


class Tree:
    """Owning wrapper of an ``ndhss_tree*``."""

    def __init__(self, handle, n):
        self.handle = handle
        self.n = n
        nn, dp, nnz, smb = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int64()
        _check(load().ndhss_tree_sizes(handle, C.byref(nn), C.byref(dp), C.byref(nnz), C.byref(smb)))
        self.nnodes, self.depth, self.nnz, self.sum_mb = nn.value, dp.value, nnz.value, smb.value

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ndhss_tree_destroy(self.handle)
            self.handle = None


def ndhss_build_tree(coords, rowptr, col, leaf_size: int) -> Tree:
    coords = np.ascontiguousarray(coords, dtype=np.int32)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    n = coords.shape[0]
    h = C.c_void_p()
    _check(load().ndhss_build_tree(n, _ptr(coords), _ptr(rowptr), _ptr(col), int(leaf_size), C.byref(h)))
    return Tree(h, n)


def ndhss_build_tree_batched(problems, leaf_size: int) -> Tree:
    """Forest of independent problems; ``problems`` is a sequence of
    (coords, rowptr, col) host arrays, one per problem.  The tree's DOFs are
    the problems' DOFs concatenated in order."""
    keep = []
    for (coords, rowptr, col) in problems:
        keep.append((np.ascontiguousarray(coords, dtype=np.int32), np.ascontiguousarray(rowptr, dtype=np.int32),
                     np.ascontiguousarray(col, dtype=np.int32)))
    ns = len(keep)
    n = np.array([k[0].shape[0] for k in keep], dtype=np.int32)
    P = C.POINTER(C.c_int32)
    arr = lambda j: (P * ns)(*[k[j].ctypes.data_as(P) for k in keep])
    h = C.c_void_p()
    _check(load().ndhss_build_tree_batched(ns, _ptr(n), arr(0), arr(1), arr(2), int(leaf_size), C.byref(h)))
    return Tree(h, int(n.sum()))


def batch_csr(mats):
    """The block-diagonal CSR of scipy matrices ``mats`` (the layout the
    batched tree describes) and the DOF offsets [nsys + 1]."""
    import scipy.sparse as sp
    mats = [m.tocsr() for m in mats]
    off = np.zeros(len(mats) + 1, dtype=np.int64)
    off[1:] = np.cumsum([m.shape[0] for m in mats])
    eoff = np.zeros(len(mats) + 1, dtype=np.int64)
    eoff[1:] = np.cumsum([m.nnz for m in mats])
    indptr = np.concatenate([np.zeros(1, np.int64)] + [m.indptr[1:].astype(np.int64) + eoff[s]
                                                      for s, m in enumerate(mats)])
    indices = np.concatenate([m.indices.astype(np.int64) + off[s] for s, m in enumerate(mats)])
    data = np.concatenate([m.data for m in mats])
    n = int(off[-1])
    A = sp.csr_matrix((data, indices.astype(np.int32), indptr.astype(np.int32)), shape=(n, n))
    return A, off


def ndhss_tree_export(tree: Tree) -> dict:
    out = dict(perm=np.empty(tree.n, np.int32), node_info=np.empty((tree.nnodes, 14), np.int32),
               blist=np.empty(tree.sum_mb, np.int32), emap=np.empty(tree.sum_mb, np.int32),
               e_off=np.empty(tree.nnodes + 1, np.int32), e_row=np.empty(tree.nnz, np.int32),
               e_col=np.empty(tree.nnz, np.int32), e_idx=np.empty(tree.nnz, np.int32))
    keys = ("perm", "node_info", "blist", "emap", "e_off", "e_row", "e_col", "e_idx")
    _check(load().ndhss_tree_export(tree.handle, *[_ptr(out[k]) for k in keys]))
    return out


class Factor:
    """Owning wrapper of an ``ndhss_factorization*`` (device memory)."""

    def __init__(self, handle, tree, vtype, prec):
        self.handle = handle
        self.tree = tree
        self.vtype = vtype
        self.prec = prec

    @property
    def n(self):
        return self.tree.n

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ndhss_factor_destroy(self.handle)
            self.handle = None


def make_factor_opts(prec=NDHSS_FP64, hss_levels=-1, eps_hss=1e-6, beta=64, k0=32, r=16, rank_cap=512,
                     panel=0, seed=0, timing=False, ulv=False) -> FactorOpts:
    return FactorOpts(prec, hss_levels, eps_hss, beta, k0, r, rank_cap, panel, seed, int(bool(timing)), int(bool(ulv)))


def ndhss_factor(tree: Tree, vtype: int, d_rowptr, d_col, d_vals, opts: FactorOpts | None = None,
                 stream=None) -> Factor:
    h = C.c_void_p()
    o = opts if opts is not None else make_factor_opts()
    _check(load().ndhss_factor(tree.handle, int(vtype), _ptr(d_rowptr), _ptr(d_col), _ptr(d_vals), C.byref(o),
                               _stream(stream), C.byref(h)))
    return Factor(h, tree, vtype, o.prec)


def ndhss_factor_stats_get(f: Factor) -> dict:
    st = FactorStats()
    _check(load().ndhss_factor_stats_get(f.handle, C.byref(st)))
    return st.as_dict()


def ndhss_factor_get_block(f: Factor, node: int, which: int, m_i: int, m_b: int) -> np.ndarray:
    rows = m_i if which in (0, 1) else m_b
    cols = m_i if which in (0, 2) else m_b
    dt = np.complex128 if f.vtype == NDHSS_C128 else np.float64
    out = np.zeros((cols, max(rows, 1)), dtype=dt)          # column-major storage, ld = rows
    _check(load().ndhss_factor_get_block(f.handle, int(node), int(which), _ptr(out), max(rows, 1)))
    return out[:, :rows].T.copy()


def _check_vector(f: Factor, v, name: str, device_only: bool = False):
    """Refuse a buffer the C side would read or write out of bounds: it must
    hold exactly f.n contiguous values of the factor's value type
    (float64 / complex128), on the device where the call needs one."""
    want = "complex128" if f.vtype == NDHSS_C128 else "float64"
    if hasattr(v, "data_ptr"):
        if device_only and not v.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if not v.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        dt = str(v.dtype).replace("torch.", "")
        size = v.numel()
    else:
        if device_only:
            raise ValueError(f"{name} must be a CUDA tensor")
        if not (v.flags["C_CONTIGUOUS"] or v.flags["F_CONTIGUOUS"]):
            raise ValueError(f"{name} must be contiguous")
        dt = str(v.dtype)
        size = v.size
    if dt != want:
        raise ValueError(f"{name} has dtype {dt}; this factor takes {want}")
    if size != f.n:
        raise ValueError(f"{name} has {size} values; this factor takes n = {f.n}")


def ndhss_apply(f: Factor, x, y, stream=None):
    """y = P^{-1} x.  x, y: (n,) vectors (torch CUDA or numpy) of the factor's value type."""
    n = f.n
    if x.ndim == 2:
        raise ValueError("pass one right-hand side per call, or several as rows of a block via ndhss_apply_block")
    _check_vector(f, x, "x")
    _check_vector(f, y, "y")
    _check(load().ndhss_apply(f.handle, 1, _ptr(x), n, _ptr(y), n, _stream(stream)))
    return y


def ndhss_apply_block(f: Factor, X, Y, stream=None):
    """Y[j] = P^{-1} X[j] for the rows j of contiguous (nrhs, n) blocks, i.e.
    column-major n x nrhs with leading dimension n (one C-ABI call)."""
    n = f.n
    if X.ndim != 2 or X.shape[1] != n or tuple(Y.shape) != tuple(X.shape):
        raise ValueError("X and Y must both have shape (nrhs, n)")
    _check(load().ndhss_apply(f.handle, int(X.shape[0]), _ptr(X), n, _ptr(Y), n, _stream(stream)))
    return Y


def ndhss_apply_noalloc(f: Factor, d_x, d_y, stream=None):
    """y = P^{-1} x without any allocation (device tensors of n values; see include/ndhss.h)."""
    _check_vector(f, d_x, "d_x", device_only=True)
    _check_vector(f, d_y, "d_y", device_only=True)
    _check(load().ndhss_apply_noalloc(f.handle, _ptr(d_x), _ptr(d_y), _stream(stream)))
    return d_y


def ndhss_testing_stall_apply(f: Factor):
    """Failure-detection hook: makes the next apply's bounded waits run out."""
    _check(load().ndhss_testing_stall_apply(f.handle))


def ndhss_elem_qform(d_goff, nloc: int, d_idx, d_mats, d_lam, d_x, d_q, stream=None):
    """q[g] = sum over the elements of group g of conj(lam_e)^T M_e x_e (device tensors)."""
    _check(load().ndhss_elem_qform(int(d_goff.numel()) - 1, _ptr(d_goff), int(nloc), _ptr(d_idx), _ptr(d_mats),
                                   _ptr(d_lam), _ptr(d_x), _ptr(d_q), _stream(stream)))
    return d_q


def ndhss_spmv(n: int, vtype: int, d_rowptr, d_col, d_vals, d_x, d_y, stream=None):
    _check(load().ndhss_spmv(int(n), int(vtype), _ptr(d_rowptr), _ptr(d_col), _ptr(d_vals), _ptr(d_x), _ptr(d_y),
                             _stream(stream)))
    return d_y


def ndhss_kernel_launches() -> int:
    return int(load().ndhss_kernel_launches())


def ndhss_measure_fma_peak(which: int, stream=None) -> float:
    """Sustained FMA rate of the device's CUDA cores in TFLOP/s: which = 0
    FP64, 1 FP32 (measurement aid, no counterpart in the paper)."""
    if which not in (0, 1):
        raise ValueError("which must be 0 (FP64) or 1 (FP32)")
    out = C.c_double(0.0)
    _check(load().ndhss_measure_fma_peak(int(which), _stream(stream), C.byref(out)))
    return float(out.value)


def ndhss_gmres(f: Factor, d_rowptr, d_col, d_vals, b, x, restart=30, maxit=300, tol=1e-8, stream=None,
                raise_on_nonconvergence=False, timing=False, inner=0.1, cycle_rtol=-1.0, conj_transpose=False):
    """Solve A x = b (A^H x = b with conj_transpose); b, x are (n,) torch CUDA
    tensors or numpy arrays.  Returns the stats dict."""
    n = f.n
    st = GmresStats()
    o = GmresOpts(int(restart), int(maxit), float(tol), int(bool(timing)), int(bool(conj_transpose)), float(inner),
                  float(cycle_rtol))
    code = load().ndhss_gmres(f.handle, _ptr(d_rowptr), _ptr(d_col), _ptr(d_vals), 1, _ptr(b), n, _ptr(x), n,
                              C.byref(o), C.byref(st), _stream(stream))
    if code == 5 and not raise_on_nonconvergence:
        return st.as_dict()
    _check(code)
    return st.as_dict()


def ndhss_apply_multi(f: Factor, X, Y, stream=None):
    """Y = P^{-1} X for up to 32 right-hand sides stored interleaved: X, Y
    contiguous (n, nrhs) torch CUDA tensors (row = DOF, column = right-hand side)."""
    if X.ndim != 2 or X.shape[0] != f.n or tuple(Y.shape) != tuple(X.shape):
        raise ValueError("X and Y must both have shape (n, nrhs)")
    nrhs = int(X.shape[1])
    _check(load().ndhss_apply_multi(f.handle, nrhs, _ptr(X), nrhs, _ptr(Y), nrhs, _stream(stream)))
    return Y


def ndhss_gmres_batched(f: Factor, d_rowptr, d_col, d_vals, sys_off, B, X, restart=30, maxit=300, tol=1e-8,
                        stream=None, raise_on_nonconvergence=False, inner=0.1, cycle_rtol=-1.0):
    """Solve the batch's systems in lockstep.  B, X: (nrhs, n) contiguous torch
    CUDA tensors (column-major n x nrhs); ``sys_off`` the problems' row offsets
    [nsys + 1].  Returns a list (per problem) of lists (per right-hand side)
    of stats dicts."""
    n = f.n
    off = np.ascontiguousarray(sys_off, dtype=np.int64)
    nsys = off.size - 1
    nrhs = int(B.shape[0]) if B.ndim == 2 else 1
    st = (GmresStats * max(nsys * nrhs, 1))()
    o = GmresOpts(int(restart), int(maxit), float(tol), 0, 0, float(inner), float(cycle_rtol))
    code = load().ndhss_gmres_batched(f.handle, _ptr(d_rowptr), _ptr(d_col), _ptr(d_vals), nsys, _ptr(off), nrhs,
                                      _ptr(B), n, _ptr(X), n, C.byref(o), st, _stream(stream))
    if not (code == 5 and not raise_on_nonconvergence):
        _check(code)
    return [[st[s * nrhs + c].as_dict() for c in range(nrhs)] for s in range(nsys)]


class DeviceCSR:
    """A scipy CSR matrix copied to torch CUDA tensors (int32 pattern, float64/complex128 values)."""

    def __init__(self, A, device="cuda"):
        import torch
        self.n = A.shape[0]
        self.nnz = A.nnz
        self.vtype = NDHSS_C128 if np.iscomplexobj(A.data) else NDHSS_R64
        self.rowptr = torch.from_numpy(np.ascontiguousarray(A.indptr, dtype=np.int32)).to(device)
        self.col = torch.from_numpy(np.ascontiguousarray(A.indices, dtype=np.int32)).to(device)
        dt = np.complex128 if self.vtype == NDHSS_C128 else np.float64
        self.vals = torch.from_numpy(np.ascontiguousarray(A.data, dtype=dt)).to(device)
