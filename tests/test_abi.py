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
    assert lib.cmsvd_csr_create(None, 2, 2, 0, None, None, None, 0, 0, C.byref(C.c_void_p())) == B.INVALID_ARG
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


def test_header_is_c99_and_matches_binding_layout(lib, tmp_path):
    """include/cmsvd.h compiles as strict C99 and links against the library, and the
    struct layouts the ctypes binding declares match the header field by field (sizes
    and offsets taken from the C compiler), as do the status and enum values."""
    import ctypes as C
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"cmsvd_params": B.cmsvd_params, "cmsvd_stats": B.cmsvd_stats}
    consts = {"CMSVD_OK": B.OK, "CMSVD_INVALID_ARG": B.INVALID_ARG, "CMSVD_INVALID_MATRIX": B.INVALID_MATRIX,
              "CMSVD_OUT_OF_MEMORY": B.OUT_OF_MEMORY, "CMSVD_WORKSPACE_TOO_SMALL": B.WORKSPACE_TOO_SMALL,
              "CMSVD_NOT_CONVERGED": B.NOT_CONVERGED, "CMSVD_BREAKDOWN": B.BREAKDOWN,
              "CMSVD_SUBSPACE_SATURATED": B.SUBSPACE_SATURATED, "CMSVD_CUDA_ERROR": B.CUDA_ERROR,
              "CMSVD_NOT_SUPPORTED": B.NOT_SUPPORTED, "CMSVD_PENDING": B.PENDING,
              "CMSVD_LINEAR": B.LINEAR, "CMSVD_NT": B.NT, "CMSVD_SOLVER_AUTO": B.SOLVER_AUTO,
              "CMSVD_SOLVER_KRYLOV": B.SOLVER_KRYLOV, "CMSVD_SOLVER_DIRECT": B.SOLVER_DIRECT,
              "CMSVD_SOLVER_DENSE": B.SOLVER_DENSE, "CMSVD_FP64": B.FP64, "CMSVD_MIXED": B.MIXED,
              "CMSVD_PROF_CLASSES": len(B.PROFILE_CLASSES)}
    body = ["#include <stdio.h>", "#include <stddef.h>", '#include "cmsvd.h"', "int main(void) {",
            "    cmsvd_params p;", "    if (cmsvd_params_default(&p) != CMSVD_OK) return 1;",
            '    printf("default %d %d %d %d\\n", (int)p.N, (int)p.L, (int)p.M, (int)p.ell);']
    for sname, st in structs.items():
        body.append(f'    printf("size {sname} %zu\\n", sizeof({sname}));')
        for f, _ in st._fields_:
            body.append(f'    printf("off {sname}.{f} %zu\\n", offsetof({sname}, {f}));')
    for k in consts:
        body.append(f'    printf("const {k} %d\\n", (int){k});')
    body += ["    return 0;", "}"]
    src = tmp_path / "abi_check.c"
    src.write_text("\n".join(body) + "\n")
    exe = tmp_path / "abi_check"
    libdir = os.path.dirname(B.LIB_PATH)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", libdir, "-lcmsvd", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in filter(None, out):
        kind, key, val = line.split(" ", 2)
        got[(kind, key)] = val
    assert got[("default", "32")] == "16 4 1"
    for sname, st in structs.items():
        assert int(got[("size", sname)]) == C.sizeof(st), sname
        for f, _ in st._fields_:
            assert int(got[("off", f"{sname}.{f}")]) == getattr(st, f).offset, f"{sname}.{f}"
    for k, v in consts.items():
        assert int(got[("const", k)]) == v, k


def test_readme_c_example_builds(lib, tmp_path):
    """The C usage example in README.md compiles as strict C99 against the header and links
    against the library and the CUDA runtime (built, not run: it needs a GPU)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    cuda = os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    if cc is None or not os.path.exists(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("no C compiler or CUDA headers")
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```c\n(.*?)```", text, flags=re.S)
    assert len(blocks) == 1
    src = tmp_path / "example.c"
    src.write_text(blocks[0])
    libdir = os.path.dirname(B.LIB_PATH)
    cudalib = next((d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"))
                    if os.path.isdir(d)), None)
    if cudalib is None:
        pytest.skip("no CUDA runtime library directory")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-fPIC", "-shared",
                        "-I", os.path.join(ROOT, "include"), "-isystem", os.path.join(cuda, "include"), str(src),
                        "-L", libdir, "-lcmsvd", "-L", cudalib, "-lcudart", "-Wl,--no-undefined",
                        "-o", str(tmp_path / "libexample.so")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_gram_operand_checks_before_any_launch():
    """The binding rejects mismatched Gram operands before the library (or a GPU) is touched."""
    torch = pytest.importorskip("torch")
    X = torch.zeros((10, 3), dtype=torch.float64)
    with pytest.raises(ValueError, match="rows"):
        B.cmsvd_gram_noalloc(0, X, torch.zeros((9, 4), dtype=torch.float64), torch.zeros((3, 4), dtype=torch.float64))
    with pytest.raises(ValueError, match="G must be"):
        B.cmsvd_gram_noalloc(0, X, torch.zeros((10, 4), dtype=torch.float64), torch.zeros((4, 3), dtype=torch.float64))
    with pytest.raises(ValueError, match="float64"):
        B.cmsvd_gram(0, X.float(), X.float(), torch.zeros((3, 3)), None)
    with pytest.raises(ValueError, match="CUDA"):
        B.cmsvd_gram_noalloc(0, X, X, torch.zeros((3, 3), dtype=torch.float64))
