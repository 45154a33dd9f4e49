"""Host-side checks of the C ABI (no GPU work): the library loads, exports every
entry point declared in include/cmsvd.h, and its host-only calls behave."""
import os
import re

import pytest

from paper_2109_13655_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return B.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "cmsvd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cmsvd_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_boundary():
    names = declared_functions()
    for must in ("cmsvd_csr_create", "cmsvd_csr_destroy", "cmsvd_solve_interval", "cmsvd_moments", "cmsvd_spmm",
                 "cmsvd_result_copy", "cmsvd_workspace_size", "cmsvd_quadrature"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(B.EXPORTED) | {"cmsvd_status_string", "cmsvd_last_error"}


def test_status_strings(lib):
    assert lib.cmsvd_status_string(0) == b"ok"
    assert lib.cmsvd_status_string(B.NOT_CONVERGED) == b"not converged"
    assert lib.cmsvd_status_string(999) == b"unknown status"


def test_params_defaults(lib):
    p = B.params()
    assert (p.N, p.L, p.M, p.ell) == (32, 16, 4, 1)
    assert p.delta == 1e-12 and p.eps_tau == 1e-8 and p.alpha == 0.1
    assert p.tol_triplet == 1e-10 and p.tol_solve == 1e-12
    q = B.params(N=16, variant="nt", solver="direct")
    assert (q.N, q.variant, q.solver) == (16, B.NT, B.SOLVER_DIRECT)
    with pytest.raises(KeyError):
        B.params(bogus=1)


def test_null_arguments_rejected(lib):
    import ctypes as C
    assert lib.cmsvd_params_default(None) == B.INVALID_ARG
    assert lib.cmsvd_context_create(None, None) == B.INVALID_ARG
    assert lib.cmsvd_csr_create(None, 2, 2, 0, None, None, None, 0, C.byref(C.c_void_p())) == B.INVALID_ARG
    assert lib.cmsvd_result_count(None, None) == B.INVALID_ARG
    assert lib.cmsvd_context_destroy(None) == B.OK
    assert lib.cmsvd_csr_destroy(None) == B.OK
    assert lib.cmsvd_result_destroy(None) == B.OK


def test_context_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes as C
    h = C.c_void_p()
    st = lib.cmsvd_context_create(None, C.byref(h))
    assert st == B.CUDA_ERROR
    assert h.value is None
    assert len(lib.cmsvd_last_error()) > 0


def test_batch_and_server_argument_checks(lib):
    """Host-side argument validation of the batched and serving entry points (no GPU work)."""
    import ctypes as C
    st = (C.c_int * 1)()
    assert lib.cmsvd_solve_batch(-1, None, None, None, None, None, None, None, None, None) == B.INVALID_ARG
    assert lib.cmsvd_solve_batch(1, None, None, None, None, None, None, None, None, st) == B.INVALID_ARG
    assert lib.cmsvd_solve_batch(0, None, None, None, None, None, None, None, None, None) == B.OK
    h = C.c_void_p()
    assert lib.cmsvd_server_create(0, 0, C.byref(h)) == B.INVALID_ARG
    assert lib.cmsvd_server_create(65, 0, C.byref(h)) == B.INVALID_ARG
    assert lib.cmsvd_server_create(1, 0, None) == B.INVALID_ARG
    assert lib.cmsvd_server_destroy(None) == B.OK
    assert lib.cmsvd_server_wait(None, 1, 0, None, None, None, None) == B.INVALID_ARG
    assert lib.cmsvd_server_take(None, 1, 0, None, None, None, None, None, None, None) == B.INVALID_ARG
    assert lib.cmsvd_server_submit(None, 0, 0.1, 0.2, None, None, None) == B.INVALID_ARG
    assert lib.cmsvd_status_string(B.PENDING) == b"pending"
    assert lib.cmsvd_result_copy_estimate(None, None) == B.INVALID_ARG
