"""ctypes binding of libcmsvd.so (include/cmsvd.h): argument marshalling only.

Every computation happens in the CUDA library. PyTorch supplies device memory
and the stream; tensors are passed as raw device pointers. If the library is
missing, ``lib()`` raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcmsvd.so")

OK, INVALID_ARG, INVALID_MATRIX, OUT_OF_MEMORY, WORKSPACE_TOO_SMALL, NOT_CONVERGED, BREAKDOWN, \
    SUBSPACE_SATURATED, CUDA_ERROR, NOT_SUPPORTED, PENDING = range(11)
LINEAR, NT = 0, 1
SOLVER_AUTO, SOLVER_KRYLOV, SOLVER_DIRECT, SOLVER_DENSE = 0, 1, 2, 3
FP64, MIXED = 0, 1
STORE_FP64, STORE_FP32, STORE_BF16 = 0, 1, 2
STORAGES = {"fp64": STORE_FP64, "fp32": STORE_FP32, "bf16": STORE_BF16}
VARIANTS = {"linear": LINEAR, "nt": NT}
SOLVERS = {"auto": SOLVER_AUTO, "krylov": SOLVER_KRYLOV, "direct": SOLVER_DIRECT, "dense": SOLVER_DENSE}


class cmsvd_params(C.Structure):
    _fields_ = [("N", C.c_int32), ("L", C.c_int32), ("M", C.c_int32), ("ell", C.c_int32),
                ("delta", C.c_double), ("eps_tau", C.c_double), ("alpha", C.c_double),
                ("variant", C.c_int32), ("solver", C.c_int32), ("precision", C.c_int32),
                ("max_iter", C.c_int32), ("tol_solve", C.c_double), ("tol_triplet", C.c_double),
                ("norm_A", C.c_double), ("check_every", C.c_int32), ("direct_max_block", C.c_int32),
                ("profile", C.c_int32), ("refine", C.c_int32), ("estimate", C.c_int32),
                ("fault_breakdown_at", C.c_int32)]

PROFILE_CLASSES = ("spmm", "krylov", "direct", "gram", "gemm", "small_dense", "other", "jacobi")


class cmsvd_stats(C.Structure):
    _fields_ = [("found", C.c_int64), ("in_interval", C.c_int64), ("rank", C.c_int64),
                ("krylov_iters", C.c_int64), ("max_component", C.c_int64),
                ("solver_used", C.c_int32), ("converged", C.c_int32),
                ("norm_A", C.c_double), ("sigma_S1", C.c_double), ("max_res_u", C.c_double),
                ("max_res_v", C.c_double), ("ms_solve", C.c_double), ("ms_truncate", C.c_double),
                ("ms_qr", C.c_double), ("ms_ritz", C.c_double), ("kernel_launches", C.c_int64),
                ("refine_rounds", C.c_int32), ("pad_", C.c_int32), ("refine_residual", C.c_double),
                ("prof_ms", C.c_double * 8), ("prof_launches", C.c_int64 * 8), ("prof_bytes", C.c_double * 8),
                ("prof_flops", C.c_double * 8), ("ms_components", C.c_double)]

    def as_dict(self) -> dict:
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if k.startswith("prof_") else v
        return d


_P = C.c_void_p
_I64 = C.c_int64
_SIGS = {
    "cmsvd_status_string": (C.c_char_p, [C.c_int]),
    "cmsvd_last_error": (C.c_char_p, []),
    "cmsvd_params_default": (C.c_int, [C.POINTER(cmsvd_params)]),
    "cmsvd_context_create": (C.c_int, [_P, C.POINTER(_P)]),
    "cmsvd_context_destroy": (C.c_int, [_P]),
    "cmsvd_context_set_dense_arith": (C.c_int, [_P, C.c_int32]),
    "cmsvd_csr_create": (C.c_int, [_P, _I64, _I64, _I64, _P, _P, _P, C.c_int, C.c_int32, C.POINTER(_P)]),
    "cmsvd_csr_destroy": (C.c_int, [_P]),
    "cmsvd_csr_shape": (C.c_int, [_P, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64)]),
    "cmsvd_spmm": (C.c_int, [_P, C.c_int, _I64, _P, _I64, _P, _I64]),
    "cmsvd_spmm_f32": (C.c_int, [_P, C.c_int, _I64, _P, _I64, _P, _I64]),
    "cmsvd_spmm_df": (C.c_int, [_P, C.c_int, _I64, _P, _I64, _P, _I64]),
    "cmsvd_spmm_tuning": (C.c_int, [_P, C.c_int, C.c_int32, _I64, _P, C.POINTER(C.c_float)]),
    "cmsvd_quadrature": (C.c_int, [_P, C.c_double, C.c_double, C.c_int32, C.c_int32, C.c_double, _P, _P, _P]),
    "cmsvd_workspace_size": (C.c_int, [_P, C.POINTER(cmsvd_params), C.POINTER(C.c_size_t)]),
    "cmsvd_gram_workspace_size": (C.c_int, [_P, _I64, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]),
    "cmsvd_gram": (C.c_int, [_P, _I64, C.c_int32, C.c_int32, _P, _I64, _P, _I64, _P, _P, C.c_size_t]),
    "cmsvd_gram_noalloc": (C.c_int, [_P, _I64, C.c_int32, C.c_int32, _P, _I64, _P, _I64, _P]),
    "cmsvd_gemm": (C.c_int, [_P, _I64, C.c_int32, C.c_int32, _P, _I64, _P, _I64, _P, _I64]),
    "cmsvd_moments": (C.c_int, [_P, C.c_double, C.c_double, C.POINTER(cmsvd_params), _P, _P, _P, C.c_size_t,
                                C.POINTER(cmsvd_stats)]),
    "cmsvd_solve_interval": (C.c_int, [_P, C.c_double, C.c_double, C.POINTER(cmsvd_params), _P, _P, C.c_size_t,
                                       C.POINTER(_P)]),
    "cmsvd_result_count": (C.c_int, [_P, C.POINTER(_I64)]),
    "cmsvd_result_copy": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "cmsvd_result_copy_estimate": (C.c_int, [_P, _P]),
    "cmsvd_server_create": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(_P)]),
    "cmsvd_server_destroy": (C.c_int, [_P]),
    "cmsvd_server_add_matrix": (C.c_int, [_P, C.c_int64, C.c_int64, C.c_int64, _P, _P, _P, C.c_int, C.c_int32,
                                          C.POINTER(C.c_int)]),
    "cmsvd_server_submit": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.POINTER(cmsvd_params), _P,
                                      C.POINTER(C.c_int64)]),
    "cmsvd_server_wait": (C.c_int, [_P, C.c_int64, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "cmsvd_server_take": (C.c_int, [_P, C.c_int64, C.c_int64, _P, _P, _P, _P, _P, _P, C.POINTER(cmsvd_stats)]),
    "cmsvd_solve_batch": (C.c_int, [C.c_int, C.POINTER(_P), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(cmsvd_params), C.POINTER(_P), C.POINTER(_P), C.POINTER(C.c_size_t),
                                    C.POINTER(_P), C.POINTER(C.c_int)]),
    "cmsvd_result_stats": (C.c_int, [_P, C.POINTER(cmsvd_stats)]),
    "cmsvd_result_destroy": (C.c_int, [_P]),
}
EXPORTED = tuple(_SIGS)

_lib = None


def lib() -> C.CDLL:
    """Load libcmsvd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        h = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib = h
    return _lib


class CmsvdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().cmsvd_last_error().decode(errors="replace")
        name = lib().cmsvd_status_string(status).decode()
        super().__init__(f"{where}: {name} ({status}): {msg}")


def _check(status: int, where: str, allow=()) -> int:
    if status != OK and status not in allow:
        raise CmsvdError(status, where)
    return status


def _ptr(t) -> int:
    """Device or host address of a torch tensor or numpy array (must be contiguous)."""
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


def params(**kw) -> cmsvd_params:
    """cmsvd_params with the library defaults, overridden by keyword arguments.
    variant / solver accept the strings of VARIANTS / SOLVERS."""
    p = cmsvd_params()
    _check(lib().cmsvd_params_default(C.byref(p)), "cmsvd_params_default")
    for k, v in kw.items():
        if k == "variant" and isinstance(v, str):
            v = VARIANTS[v]
        if k == "solver" and isinstance(v, str):
            v = SOLVERS[v]
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


# ----------------------------------------------------------------------------- raw entry points
def cmsvd_context_create(stream: int = 0) -> int:
    h = _P()
    _check(lib().cmsvd_context_create(_P(stream), C.byref(h)), "cmsvd_context_create")
    return h.value


def cmsvd_context_destroy(ctx: int) -> None:
    _check(lib().cmsvd_context_destroy(_P(ctx)), "cmsvd_context_destroy")


def cmsvd_csr_create(ctx: int, m: int, n: int, rowptr, colidx, vals, storage=STORE_FP64) -> int:
    """rowptr int64[m+1], colidx int32[nnz], vals float64[nnz]: numpy (host) or torch CUDA tensors.
    storage: STORE_FP64 / STORE_FP32 / STORE_BF16 (or "fp64", "fp32", "bf16")."""
    storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
    on_dev = 0 if isinstance(rowptr, np.ndarray) else 1
    if on_dev == 0:
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        colidx = np.ascontiguousarray(colidx, dtype=np.int32)
        vals = np.ascontiguousarray(vals, dtype=np.float64)
    nnz = int(rowptr[-1])
    h = _P()
    _check(lib().cmsvd_csr_create(_P(ctx), m, n, nnz, _ptr(rowptr), _ptr(colidx) if nnz else None,
                                  _ptr(vals) if nnz else None, on_dev, storage, C.byref(h)), "cmsvd_csr_create")
    return h.value


def cmsvd_csr_destroy(A: int) -> None:
    _check(lib().cmsvd_csr_destroy(_P(A)), "cmsvd_csr_destroy")


def cmsvd_csr_shape(A: int):
    m, n, z = _I64(), _I64(), _I64()
    _check(lib().cmsvd_csr_shape(_P(A), C.byref(m), C.byref(n), C.byref(z)), "cmsvd_csr_shape")
    return m.value, n.value, z.value


def cmsvd_spmm(A: int, transpose: bool, X, Y) -> None:
    """Y = A X (or A^T X); X, Y float64 CUDA tensors, row-major blocks."""
    L = X.shape[1]
    _check(lib().cmsvd_spmm(_P(A), int(transpose), L, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0)), "cmsvd_spmm")


def cmsvd_spmm_f32(A: int, transpose: bool, X, Y) -> None:
    """Y = A X (or A^T X) in FP32; X, Y float32 CUDA tensors, row-major blocks."""
    L = X.shape[1]
    _check(lib().cmsvd_spmm_f32(_P(A), int(transpose), L, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0)), "cmsvd_spmm_f32")


def cmsvd_spmm_df(A: int, transpose: bool, X, Y) -> None:
    """Y = A X (or A^T X) in double-float arithmetic; X, Y float32 CUDA tensors of shape
    (rows, 2 L): each row holds the L high parts, then the L low parts."""
    L = X.shape[1] // 2
    _check(lib().cmsvd_spmm_df(_P(A), int(transpose), L, _ptr(X), X.stride(0), _ptr(Y), Y.stride(0)), "cmsvd_spmm_df")


def cmsvd_spmm_tuning(A: int, transpose: bool, kind: int, L: int):
    """The autotuner's pick: dict(lanes_per_row, gathers, slices, natural_order, ms), or None
    when that product has not run yet. kind: 0 FP64, 1 FP32, 2 double-float."""
    cfg = np.zeros(4, dtype=np.int32)
    ms = C.c_float()
    s = lib().cmsvd_spmm_tuning(_P(A), int(transpose), kind, L, _P(cfg.ctypes.data), C.byref(ms))
    if s == NOT_SUPPORTED:
        return None
    _check(s, "cmsvd_spmm_tuning")
    return {"lanes_per_row": int(cfg[0]), "gathers_in_flight": int(cfg[1]), "column_slices": int(cfg[2]),
            "row_order": "storage" if cfg[3] else "first-column", "ms_in_tuning": float(ms.value)}


def cmsvd_quadrature(ctx: int, a: float, b: float, N: int, variant="linear", alpha: float = 0.1):
    """(shift, weight, scaled) for j = 1..N/2 as complex128 numpy arrays."""
    J = N // 2
    out = [np.zeros(2 * J) for _ in range(3)]
    v = VARIANTS[variant] if isinstance(variant, str) else variant
    _check(lib().cmsvd_quadrature(_P(ctx), a, b, N, v, alpha, *(o.ctypes.data for o in out)), "cmsvd_quadrature")
    return tuple(o[0::2] + 1j * o[1::2] for o in out)


def cmsvd_gram_workspace_size(ctx: int, n: int, c1: int, c2: int) -> int:
    b = C.c_size_t()
    _check(lib().cmsvd_gram_workspace_size(_P(ctx), n, c1, c2, C.byref(b)), "cmsvd_gram_workspace_size")
    return b.value


def _gram_operands(X, Y, G):
    """Shape, dtype and device checks of a Gram call, before anything reaches the library:
    a wrong shape would make the kernels read or write outside the tensors."""
    import torch
    if X.dim() != 2 or Y.dim() != 2 or G.dim() != 2:
        raise ValueError("X, Y and G must be 2-D")
    n, c1 = X.shape
    c2 = Y.shape[1]
    if Y.shape[0] != n:
        raise ValueError(f"Y has {Y.shape[0]} rows, X has {n}")
    if tuple(G.shape) != (c1, c2):
        raise ValueError(f"G must be {c1} x {c2}, got {tuple(G.shape)}")
    for name, t in (("X", X), ("Y", Y), ("G", G)):
        if t.dtype != torch.float64:
            raise ValueError(f"{name} must be float64")
        if t.stride(1) != 1:
            raise ValueError(f"{name} rows must be contiguous")
    if not G.is_contiguous():
        raise ValueError("G must be contiguous")
    if not (X.is_cuda and Y.is_cuda and G.is_cuda):
        raise ValueError("X, Y and G must be CUDA tensors")
    return n, c1, c2


def cmsvd_gram(ctx: int, X, Y, G, workspace) -> None:
    """G (c1 x c2) = X^T Y for float64 CUDA tensors X (n x c1), Y (n x c2) (row strides as leading dims)."""
    n, c1, c2 = _gram_operands(X, Y, G)
    _check(lib().cmsvd_gram(_P(ctx), n, c1, c2, _ptr_any(X), X.stride(0), _ptr_any(Y), Y.stride(0), _ptr(G),
                            _ptr(workspace), workspace.numel() * workspace.element_size()), "cmsvd_gram")


def cmsvd_gemm(ctx: int, X, W, Z) -> None:
    """Z (n x c2) = X (n x c1) W (c1 x c2), float64 CUDA tensors with contiguous rows."""
    import torch
    n, c1 = X.shape
    if W.shape[0] != c1 or tuple(Z.shape) != (n, W.shape[1]):
        raise ValueError("shapes must be X n x c1, W c1 x c2, Z n x c2")
    for name, t in (("X", X), ("W", W), ("Z", Z)):
        if t.dtype != torch.float64 or not t.is_cuda or t.stride(1) != 1:
            raise ValueError(f"{name} must be a float64 CUDA tensor with contiguous rows")
    _check(lib().cmsvd_gemm(_P(ctx), n, c1, W.shape[1], _ptr_any(X), X.stride(0), _ptr_any(W), W.stride(0),
                            _ptr_any(Z), Z.stride(0)), "cmsvd_gemm")


def cmsvd_gram_noalloc(ctx: int, X, Y, G) -> None:
    """G = X^T Y like cmsvd_gram, using the library's fixed device scratch (no workspace)."""
    n, c1, c2 = _gram_operands(X, Y, G)
    _check(lib().cmsvd_gram_noalloc(_P(ctx), n, c1, c2, _ptr_any(X), X.stride(0), _ptr_any(Y), Y.stride(0), _ptr(G)),
           "cmsvd_gram_noalloc")


def _ptr_any(t) -> int:
    """Device address of a row-strided tensor (unit column stride)."""
    assert t.stride(1) == 1
    return t.data_ptr()


def cmsvd_workspace_size(A: int, p: cmsvd_params) -> int:
    n = C.c_size_t()
    _check(lib().cmsvd_workspace_size(_P(A), C.byref(p), C.byref(n)), "cmsvd_workspace_size")
    return n.value


def cmsvd_moments(A: int, a: float, b: float, p: cmsvd_params, V_in, S_out, workspace) -> tuple[int, dict]:
    st = cmsvd_stats()
    s = lib().cmsvd_moments(_P(A), a, b, C.byref(p), _ptr(V_in), _ptr(S_out), _ptr(workspace),
                            workspace.numel() * workspace.element_size(), C.byref(st))
    _check(s, "cmsvd_moments", allow=(NOT_CONVERGED,))
    return s, st.as_dict()


def cmsvd_solve_interval(A: int, a: float, b: float, p: cmsvd_params, V_in, workspace) -> tuple[int, int]:
    r = _P()
    s = lib().cmsvd_solve_interval(_P(A), a, b, C.byref(p), _ptr(V_in), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), C.byref(r))
    _check(s, "cmsvd_solve_interval", allow=(NOT_CONVERGED, SUBSPACE_SATURATED))
    return s, r.value


def cmsvd_result_count(r: int) -> int:
    t = _I64()
    _check(lib().cmsvd_result_count(_P(r), C.byref(t)), "cmsvd_result_count")
    return t.value


def cmsvd_result_copy(r: int, sigma=None, U=None, V=None, res_u=None, res_v=None, tau=None) -> None:
    args = [_P(_ptr(x)) if x is not None else None for x in (sigma, U, V, res_u, res_v, tau)]
    _check(lib().cmsvd_result_copy(_P(r), *args), "cmsvd_result_copy")


def cmsvd_result_copy_estimate(r: int, res_est) -> None:
    _check(lib().cmsvd_result_copy_estimate(_P(r), _P(_ptr(res_est))), "cmsvd_result_copy_estimate")


def cmsvd_result_stats(r: int) -> dict:
    st = cmsvd_stats()
    _check(lib().cmsvd_result_stats(_P(r), C.byref(st)), "cmsvd_result_stats")
    return st.as_dict()


def cmsvd_result_destroy(r: int) -> None:
    _check(lib().cmsvd_result_destroy(_P(r)), "cmsvd_result_destroy")


def cmsvd_solve_batch(A: list, a: list, b: list, p: list, V_in: list, workspace: list) -> tuple[list, list]:
    """Raw batched call. Returns (status per problem, result handle per problem)."""
    n = len(A)
    arrP = (_P * n)(*[_P(x) for x in A])
    arrA = (C.c_double * n)(*a)
    arrB = (C.c_double * n)(*b)
    arrp = (cmsvd_params * n)(*p)
    arrV = (_P * n)(*[_P(_ptr(v)) for v in V_in])
    arrW = (_P * n)(*[_P(_ptr(w)) for w in workspace])
    arrS = (C.c_size_t * n)(*[w.numel() * w.element_size() for w in workspace])
    outs = (_P * n)()
    st = (C.c_int * n)()
    s = lib().cmsvd_solve_batch(n, arrP, arrA, arrB, arrp, arrV, arrW, arrS, outs, st)
    if s not in (OK, NOT_CONVERGED, SUBSPACE_SATURATED):
        for o in outs:
            if o:
                cmsvd_result_destroy(o)
    _check(s, "cmsvd_solve_batch", allow=(NOT_CONVERGED, SUBSPACE_SATURATED))
    return list(st), [o or 0 for o in outs]


def _triplets_from(r: int, m: int, n: int, status: int, want_estimate: bool) -> "Triplets":
    try:
        t = cmsvd_result_count(r)
        out = [np.zeros(t), np.zeros((t, m)), np.zeros((t, n)), np.zeros(t), np.zeros(t), np.zeros(t)]
        cmsvd_result_copy(r, *out)
        est = None
        if want_estimate:
            est = np.zeros(t)
            cmsvd_result_copy_estimate(r, est)
        st = cmsvd_result_stats(r)
    finally:
        cmsvd_result_destroy(r)
    return Triplets(out[0], out[1].T.copy(), out[2].T.copy(), out[3], out[4], out[5], st, status, est)


class Server:
    """Serving loop with continuous batching (cmsvd_server_*): resident matrices, requests
    with host V_in, admission by slot and HBM budget, results copied back to the host."""

    def __init__(self, slots: int = 4, hbm_budget: int = 0):
        h = _P()
        _check(lib().cmsvd_server_create(slots, hbm_budget, C.byref(h)), "cmsvd_server_create")
        self.handle = h.value
        self.shapes = []

    def add_matrix(self, A, storage=STORE_FP64) -> int:
        storage = STORAGES[storage] if isinstance(storage, str) else int(storage)
        i = C.c_int()
        rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
        ci = np.ascontiguousarray(A.colidx, dtype=np.int32)
        va = np.ascontiguousarray(A.vals, dtype=np.float64)
        _check(lib().cmsvd_server_add_matrix(_P(self.handle), A.m, A.n, A.nnz, _P(rp.ctypes.data), _P(ci.ctypes.data),
                                             _P(va.ctypes.data), 0, storage, C.byref(i)), "cmsvd_server_add_matrix")
        self.shapes.append((A.m, A.n))
        return i.value

    def submit(self, mid: int, a: float, b: float, p: cmsvd_params, V_in: np.ndarray) -> int:
        t = C.c_int64()
        V = np.ascontiguousarray(V_in, dtype=np.float64)
        n = self.shapes[mid][1] if 0 <= mid < len(self.shapes) else None
        if n is not None and V.shape != (n, p.L):
            raise ValueError(f"V_in must be {n} x {p.L}, got {V.shape}")   # the library copies n * L doubles
        _check(lib().cmsvd_server_submit(_P(self.handle), mid, a, b, C.byref(p), _P(V.ctypes.data), C.byref(t)),
               "cmsvd_server_submit")
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        """(done, t, solve_status, latency_ms, queue_ms)."""
        t, st, lat, q = C.c_int64(), C.c_int(), C.c_double(), C.c_double()
        s = lib().cmsvd_server_wait(_P(self.handle), ticket, timeout_ms, C.byref(t), C.byref(st), C.byref(lat),
                                    C.byref(q))
        if s == PENDING:
            return False, 0, PENDING, 0.0, 0.0
        _check(s, "cmsvd_server_wait")
        return True, t.value, st.value, lat.value, q.value

    def take(self, ticket: int, mid: int, t: int, status: int = 0) -> "Triplets":
        m, n = self.shapes[mid]
        out = [np.zeros(t), np.zeros((t, m)), np.zeros((t, n)), np.zeros(t), np.zeros(t), np.zeros(t)]
        st = cmsvd_stats()
        _check(lib().cmsvd_server_take(_P(self.handle), ticket, t, *[_P(x.ctypes.data) for x in out], C.byref(st)),
               "cmsvd_server_take")
        return Triplets(out[0], out[1].T.copy(), out[2].T.copy(), out[3], out[4], out[5], st.as_dict(), status)

    def close(self):
        if self.handle:
            lib().cmsvd_server_destroy(_P(self.handle))
        self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(problems: list) -> list:
    """problems: list of (Matrix, a, b, params, V_in device tensor). Spread the matrices over
    several Contexts for the problems to overlap on the GPU (see cmsvd_solve_batch)."""
    ws = [M.workspace(p) for (M, a, b, p, V) in problems]
    st, rs = cmsvd_solve_batch([M.handle for (M, *_r) in problems], [x[1] for x in problems],
                               [x[2] for x in problems], [x[3] for x in problems], [x[4] for x in problems], ws)
    return [_triplets_from(r, M.m, M.n, s, bool(p.estimate)) for r, s, (M, a, b, p, V) in zip(rs, st, problems)]


# ----------------------------------------------------------------------------- convenience
@dataclass
class Triplets:
    sigma: np.ndarray
    U: np.ndarray          # m x t
    V: np.ndarray          # n x t
    res_u: np.ndarray
    res_v: np.ndarray
    tau: np.ndarray
    stats: dict
    status: int
    res_est: np.ndarray | None = None   # Sec. 3.4.1 estimate, when solved with estimate=1


class Context:
    """A cmsvd context bound to torch's current CUDA stream (or a given one)."""

    def __init__(self, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.handle = cmsvd_context_create(stream.cuda_stream)
        self._matrices = weakref.WeakSet()

    def set_dense_arith(self, mode: int) -> None:
        """0: tall Grams and products emulated in FP64 on the BF16 tensor cores (default); 1: FP64 pipe."""
        _check(lib().cmsvd_context_set_dense_arith(_P(self.handle), int(mode)), "cmsvd_context_set_dense_arith")

    def close(self):
        """Destroy the context; matrices created on it are destroyed first."""
        if self.handle:
            for M in list(self._matrices):
                M.close()
            cmsvd_context_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Matrix:
    """A CSR matrix resident on the device (library-owned copy)."""

    def __init__(self, ctx: Context, m: int, n: int, rowptr, colidx, vals, storage=STORE_FP64):
        if not ctx.handle:
            raise RuntimeError("context is closed")
        self.ctx = ctx
        self.m, self.n = m, n
        self.handle = cmsvd_csr_create(ctx.handle, m, n, rowptr, colidx, vals, storage)
        ctx._matrices.add(self)

    @classmethod
    def from_csr(cls, ctx: Context, A, storage=STORE_FP64) -> "Matrix":
        return cls(ctx, A.m, A.n, A.rowptr, A.colidx, A.vals, storage)

    def close(self):
        if self.handle and self.ctx.handle:
            cmsvd_csr_destroy(self.handle)
        self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace(self, p: cmsvd_params):
        import torch
        return torch.empty(cmsvd_workspace_size(self.handle, p), dtype=torch.uint8, device="cuda")

    def spmm(self, X, transpose: bool = False):
        import torch
        rows = self.n if transpose else self.m
        Y = torch.empty((rows, X.shape[1]), dtype=torch.float64, device=X.device)
        cmsvd_spmm(self.handle, transpose, X, Y)
        return Y

    def spmm_f32(self, X, transpose: bool = False):
        import torch
        rows = self.n if transpose else self.m
        Y = torch.empty((rows, X.shape[1]), dtype=torch.float32, device=X.device)
        cmsvd_spmm_f32(self.handle, transpose, X, Y)
        return Y

    def spmm_df(self, X, transpose: bool = False):
        """X: float32 (cols, 2 L) double-float block; returns the (rows, 2 L) double-float product."""
        import torch
        rows = self.n if transpose else self.m
        Y = torch.empty((rows, X.shape[1]), dtype=torch.float32, device=X.device)
        cmsvd_spmm_df(self.handle, transpose, X, Y)
        return Y

    def moments(self, a, b, p: cmsvd_params, V_in, workspace=None):
        import torch
        ws = workspace if workspace is not None else self.workspace(p)
        S = torch.empty((self.n, p.L * (p.M + 1)), dtype=torch.float64, device=V_in.device)
        status, st = cmsvd_moments(self.handle, a, b, p, V_in, S, ws)
        return S, status, st

    def solve_interval(self, a, b, p: cmsvd_params, V_in, workspace=None) -> Triplets:
        ws = workspace if workspace is not None else self.workspace(p)
        status, r = cmsvd_solve_interval(self.handle, a, b, p, V_in, ws)
        return _triplets_from(r, self.m, self.n, status, bool(p.estimate))
