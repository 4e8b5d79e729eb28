"""The C-ABI library builds, loads and exports every entry point include/imq.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(imq_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2205_04194_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("imq_plan", "imq_matvec", "imq_dense_matvec", "imq_plan_destroy", "imq_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_2205_04194_gb300 import _lib
    assert set(_declared()) <= set(_lib.SIGNATURES)


def test_status_strings_without_gpu(lib):
    from paper_2205_04194_gb300 import _lib
    L = _lib.load()
    assert L.imq_status_string(0) == b"IMQ_OK"
    assert L.imq_status_string(5) == b"IMQ_NOT_CONVERGED"
    assert L.imq_version().startswith(b"imq-gb300")


def test_invalid_arguments_rejected_before_any_gpu_work(lib):
    from paper_2205_04194_gb300 import _lib
    L = _lib.load()
    h = ctypes.c_void_p(0)
    pts = (ctypes.c_double * 4)(0.0, 0.0, 1.0, 1.0)
    assert L.imq_plan(pts, 2, -1.0, 8, 16, None, None, ctypes.byref(h)) == 1      # c <= 0
    assert L.imq_plan(pts, 0, 1.0, 8, 16, None, None, ctypes.byref(h)) == 1       # N < 1
    assert L.imq_plan(pts, 2, 1.0, 99, 16, None, None, ctypes.byref(h)) == 7      # p too large
    assert L.imq_plan(None, 2, 1.0, 8, 16, None, None, ctypes.byref(h)) == 1
    assert L.imq_plan(pts, 2, float("nan"), 8, 16, None, None, ctypes.byref(h)) == 1
    assert b"c must be" in L.imq_last_error()
    assert L.imq_matvec(None, None, None, 1, 0, None) == 1


def test_oracle_builds_and_is_not_linked_by_the_product(lib):
    from oracle import dense
    assert os.path.exists(dense.build())
    # the product library references no oracle symbol
    for name in ("oracle_dense_matvec", "oracle_evaluate"):
        assert not hasattr(lib, name)


def test_autotune_arguments_rejected_before_any_gpu_work(lib):
    from paper_2205_04194_gb300 import _lib
    L = _lib.load()
    res = _lib.TuneResult()
    pts = (ctypes.c_double * 4)(0.0, 0.0, 1.0, 1.0)
    offs = (ctypes.c_int64 * 2)(0, 2)
    cs = (ctypes.c_double * 1)(0.1)
    ps = (ctypes.c_int32 * 2)(8, 12)
    leaves = (ctypes.c_int32 * 1)(32)
    args = lambda **kw: [kw.get("pts", pts), kw.get("offs", offs), kw.get("nprob", 1), kw.get("cs", cs),
                         kw.get("target", 1e-6), kw.get("ps", ps), kw.get("n_p", 2), leaves, kw.get("n_leaf", 1),
                         kw.get("nrhs", 1), None, None, ctypes.byref(res)]
    assert L.imq_autotune(*args(target=0.0)) == 1
    assert L.imq_autotune(*args(target=float("nan"))) == 1
    assert L.imq_autotune(*args(n_p=0)) == 1
    assert L.imq_autotune(*args(n_leaf=17)) == 1
    assert L.imq_autotune(*args(nrhs=0)) == 1
    assert L.imq_autotune(*args(ps=(ctypes.c_int32 * 2)(8, 99))) == 1
    assert L.imq_autotune(*args(cs=(ctypes.c_double * 1)(-1.0))) == 1
    assert L.imq_autotune(*args(offs=(ctypes.c_int64 * 2)(0, 0))) == 1
    assert L.imq_autotune(*args(pts=None)) == 1


def test_ctypes_structs_match_the_c_header(tmp_path):
    """Every struct of include/imq.h has the size and field offsets of its ctypes mirror
    (a C program compiled with gcc prints them)."""
    import subprocess
    from paper_2205_04194_gb300 import _lib
    mirrors = {"imq_options": _lib.ImqOptions, "imq_cg_options": _lib.CgOptions, "imq_cg_info": _lib.CgInfo,
               "imq_tune_entry": _lib.TuneEntry, "imq_tune_result": _lib.TuneResult,
               "imq_plan_info": _lib.PlanInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "imq.h"', "int main(void) {"]
    for cname, cls in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "sizes"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.run(["gcc", "-I", os.path.join(root, "include"), "-o", str(exe), str(src)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, cls in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_treecode_options_checked_before_any_gpu_work(lib):
    from paper_2205_04194_gb300 import _lib
    L = _lib.load()
    h = ctypes.c_void_p(0)
    pts = (ctypes.c_double * 4)(0.0, 0.0, 1.0, 1.0)
    opt = _lib.ImqOptions()
    opt.struct_size = ctypes.sizeof(_lib.ImqOptions)
    opt.algorithm = 1
    opt.levels = 0                                   # the paper's L starts at 1
    assert L.imq_plan(pts, 2, 1.0, 8, 16, ctypes.byref(opt), None, ctypes.byref(h)) == 1
    opt.levels = 16
    assert L.imq_plan(pts, 2, 1.0, 8, 16, ctypes.byref(opt), None, ctypes.byref(h)) == 1
    opt.algorithm = 7
    assert L.imq_plan(pts, 2, 1.0, 8, 16, ctypes.byref(opt), None, ctypes.byref(h)) == 1
    assert b"unknown algorithm" in L.imq_last_error()
    # the struct layout itself is checked against the C header in test_ctypes_structs_match_the_c_header


def test_allocator_needs_both_functions(lib):
    from paper_2205_04194_gb300 import _lib
    L = _lib.load()
    h = ctypes.c_void_p(0)
    pts = (ctypes.c_double * 4)(0.0, 0.0, 1.0, 1.0)
    opt = _lib.ImqOptions()
    opt.struct_size = ctypes.sizeof(_lib.ImqOptions)
    keep = _lib.ALLOC_FN(lambda n, ctx: None)
    opt.alloc = keep                                  # free missing
    assert L.imq_plan(pts, 2, 1.0, 8, 16, ctypes.byref(opt), None, ctypes.byref(h)) == 1
    assert b"together" in L.imq_last_error()


def test_binding_names_match_the_header_enums(tmp_path):
    """The Python names of every option value (dtype, algorithm, translations, M2L kernel,
    preconditioner, inner operator, residual, Krylov method) map to the values include/imq.h
    gives those enum constants (a C program compiled with gcc prints them)."""
    import subprocess
    from paper_2205_04194_gb300 import imq
    pairs = {"IMQ_F32": imq.F32, "IMQ_F64": imq.F64,
             "IMQ_ALG_FMM": imq.ALGORITHMS["fmm"], "IMQ_ALG_TREECODE": imq.ALGORITHMS["treecode"],
             "IMQ_TRANS_FP32": imq.TRANSLATIONS["fp32"], "IMQ_TRANS_FP64": imq.TRANSLATIONS["fp64"],
             "IMQ_TRANS_MIXED": imq.TRANSLATIONS["mixed"],
             "IMQ_M2L_AUTO": imq.M2L_KERNELS["auto"], "IMQ_M2L_CUDA_CORES": imq.M2L_KERNELS["cuda_cores"],
             "IMQ_M2L_TENSOR": imq.M2L_KERNELS["tensor"],
             "IMQ_PRECOND_NONE": imq.PRECONDS["none"], "IMQ_PRECOND_SCHWARZ": imq.PRECONDS["schwarz"],
             "IMQ_PRECOND_SCHWARZ_2L": imq.PRECONDS["schwarz2"],
             "IMQ_OPERATOR_FAST_F32": imq.OPERATORS["fast_f32"], "IMQ_OPERATOR_FAST_F64": imq.OPERATORS["fast_f64"],
             "IMQ_OPERATOR_DENSE_F64": imq.OPERATORS["dense_f64"],
             "IMQ_RESIDUAL_PLAN_F64": imq.RESIDUALS["plan"], "IMQ_RESIDUAL_DENSE_F64": imq.RESIDUALS["dense"],
             "IMQ_KRYLOV_CG": imq.KRYLOVS["cg"], "IMQ_KRYLOV_GMRES": imq.KRYLOVS["gmres"]}
    lines = ["#include <stdio.h>", '#include "imq.h"', "int main(void) {"]
    lines += [f'printf("{name} %d\\n", (int){name});' for name in pairs]
    lines += ["return 0;", "}"]
    src = tmp_path / "enums.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "enums"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    got = {out[k]: int(out[k + 1]) for k in range(0, len(out), 2)}
    assert got == pairs
