"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function declared in include/klecgc.h (no compute calls here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "klecgc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(klecgc_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    import paper_2510_26180_gb300 as pkg
    lib = pkg.load()
    declared = _declared()
    assert len(declared) >= 11
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert set(pkg.klecgc.EXPORTS) == set(declared)


def test_status_strings_without_gpu():
    import paper_2510_26180_gb300 as pkg
    lib = pkg.load()
    assert lib.klecgc_status_string(0) == b"ok"
    assert b"converged" in lib.klecgc_status_string(3)
    lib.klecgc_free(None)  # NULL is allowed


def test_package_does_not_import_oracle():
    import ast
    pkg_dir = os.path.join(ROOT, "paper_2510_26180_gb300")
    for fn in os.listdir(pkg_dir):
        if fn.endswith(".py"):
            tree = ast.parse(open(os.path.join(pkg_dir, fn)).read())
            for node in ast.walk(tree):
                if isinstance(node, ast.Import):
                    assert not any(a.name.split(".")[0] == "oracle" for a in node.names), fn
                if isinstance(node, ast.ImportFrom):
                    assert (node.module or "").split(".")[0] != "oracle", fn


def test_load_rejects_files_that_are_not_contexts(tmp_path):
    # klecgc_load validates the file header before any CUDA call
    import ctypes
    import paper_2510_26180_gb300 as pkg
    lib = pkg.load()
    h = ctypes.c_void_p()
    missing = os.fsencode(str(tmp_path / "missing.ctx"))
    assert lib.klecgc_load(missing, ctypes.byref(h), None) == pkg.E_INVALID_ARG
    assert b"cannot open" in lib.klecgc_last_error()
    junk = tmp_path / "junk.ctx"
    junk.write_bytes(b"not a context file" * 20)
    assert lib.klecgc_load(os.fsencode(str(junk)), ctypes.byref(h), None) == pkg.E_INVALID_ARG
    assert h.value is None
    bad = tmp_path / "short.ctx"
    bad.write_bytes(b"KLECGCv1")
    assert lib.klecgc_load(os.fsencode(str(bad)), ctypes.byref(h), None) == pkg.E_INVALID_ARG


def test_batch_rejects_bad_arguments_before_any_cuda_call():
    import ctypes
    import paper_2510_26180_gb300 as pkg
    lib = pkg.load()
    inst = (pkg.klecgc.Instance * 1)()
    assert lib.klecgc_solve_batch(None, 1, inst, 1, None, 0.1, 1e-8, 5, 0, 0, None, None, None,
                                  None) == pkg.E_INVALID_ARG
    ctxs = (ctypes.c_void_p * 1)(None)
    assert lib.klecgc_solve_batch(ctxs, 0, inst, 1, None, 0.1, 1e-8, 5, 0, 0, None, None, None,
                                  None) == pkg.E_INVALID_ARG
    # the range checks of alpha, tol, kmax, precision and guess also come first
    buf = (ctypes.c_double * 4)()
    for alpha, tol, kmax, prec, guess in [(0.0, 1e-8, 5, 0, 0), (1.0, 1e-8, 5, 0, 0),
                                          (0.1, 0.0, 5, 0, 0), (0.1, 1e-8, 0, 0, 0),
                                          (0.1, 1e-8, 5, 3, 0), (0.1, 1e-8, 5, -1, 0),
                                          (0.1, 1e-8, 5, 0, pkg.GUESS_USER),
                                          (0.1, 1e-8, 5, 0, pkg.GUESS_MLP)]:
        got = lib.klecgc_solve_batch(ctxs, 1, inst, 1, buf, alpha, tol, kmax, prec, guess, buf,
                                     None, None, None)
        assert got == pkg.E_INVALID_ARG, (alpha, tol, kmax, prec, guess)


def test_setup_validates_problem_fields_before_any_cuda_call():
    # every rule of klecgc_setup's argument check, through the C ABI; the
    # check runs before the first CUDA call, so none of these touches a GPU
    import ctypes
    import math
    import numpy as np
    import paper_2510_26180_gb300 as pkg
    from synth import workload
    lib = pkg.load()
    w = workload("heat1d_nx63")
    xi_t = np.zeros((w.n_train, w.M))
    xp = xi_t.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    INV, UNS = pkg.E_INVALID_ARG, pkg.E_UNSUPPORTED
    cases = [
        (dict(dim=3), UNS), (dict(dim=0), UNS), (dict(dim=2, nx=2048), UNS),
        (dict(nx=0), INV), (dict(M=0), INV), (dict(gpc_degree=-1), INV),
        (dict(n_train=1), INV), (dict(T=0.0), INV), (dict(T=math.nan), INV),
        (dict(sigma=-0.1), INV), (dict(corr_len=0.0), INV), (dict(eps_kl=-1e-3), INV),
        (dict(J=0), INV), (dict(reaction=-1.0), INV), (dict(forcing=math.inf), INV),
        (dict(u0_kind=-1), INV), (dict(u0_kind=3), INV), (dict(reaction_kind=3), INV),
        (dict(reaction_kind=-1), INV), (dict(cgc_newton=-1), INV),
        (dict(advection=-0.1), INV), (dict(advection=math.inf), INV),
        (dict(u0_kind=2), UNS), (dict(advection=0.1), UNS),
        (dict(dim=2, nx=15, advection=0.1, reaction_kind=1), UNS),
        (dict(dim=2, nx=15, reaction_kind=1), UNS),
        (dict(N=12), UNS), (dict(N=1), UNS), (dict(N=128), UNS),
    ]
    for over, want in cases:
        pr = pkg.Problem.from_workload(w)
        for k, v in over.items():
            setattr(pr, k, v)
        out = ctypes.c_void_p(1)
        got = lib.klecgc_setup(ctypes.byref(pr), xp, ctypes.byref(out), None)
        assert got == want, (over, got, lib.klecgc_last_error().decode())
        assert out.value is None, over
        assert lib.klecgc_last_error().decode(), over
    pr = pkg.Problem.from_workload(w)
    out = ctypes.c_void_p(1)
    assert lib.klecgc_setup(ctypes.byref(pr), None, ctypes.byref(out), None) == INV
    assert lib.klecgc_setup(None, xp, ctypes.byref(out), None) == INV
    assert lib.klecgc_setup(ctypes.byref(pr), xp, None, None) == INV


def test_every_entry_point_rejects_a_null_context_without_cuda():
    # ctx = NULL (and NULL / zero for everything else): INVALID_ARG with a
    # message, checked before any CUDA call; klecgc_free(NULL) is a no-op
    import ctypes
    import paper_2510_26180_gb300 as pkg
    lib = pkg.load()
    skip = {"klecgc_setup", "klecgc_load", "klecgc_solve_batch",    # no context argument
            "klecgc_kl_basis", "klecgc_gpc_indices"}
    names = [n for n in pkg.klecgc.EXPORTS if n.startswith("klecgc_") and n not in skip]
    checked = 0
    for name in names:
        f = getattr(lib, name)
        if f.argtypes is None or f.restype is not ctypes.c_int:
            continue
        args = []
        for t in f.argtypes:
            if t in (ctypes.c_double,):
                args.append(0.0)
            elif t in (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int):
                args.append(0)
            else:
                args.append(None)
        assert f(*args) == pkg.E_INVALID_ARG, name
        assert lib.klecgc_last_error().decode(), name
        checked += 1
    assert checked >= 24
    lib.klecgc_free(None)


def test_missing_library_fails_loudly(tmp_path):
    # no CPU fallback: without the compiled library every call path raises
    import subprocess
    import sys
    code = (
        "import paper_2510_26180_gb300.klecgc as k\n"
        f"k.LIB_PATH = {str(tmp_path / 'absent.so')!r}\n"
        "k._lib = None\n"
        "try:\n"
        "    k.load()\n"
        "except RuntimeError as e:\n"
        "    assert 'missing' in str(e)\n"
        "    print('raised')\n"
    )
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "raised", r.stderr[-2000:]


def test_noalloc_device_array_rule_on_the_host(tmp_path):
    # the allocation-free entry point accepts device memory of the context's
    # own device and managed memory only; an array on another GPU would make
    # its kernel read that GPU's memory (a fault with peer access off).  The
    # rule is plain host code, checked here with g++ and no GPU.
    import shutil
    import subprocess
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "rule.cpp"
    src.write_text(
        '#include "ptr_rule.h"\n#include <cstdio>\n'
        "int main() {\n"
        "  using klecgc::device_array_usable;\n"
        "  int ok = device_array_usable(2, 0, 0) && device_array_usable(2, 3, 3)\n"
        "        && !device_array_usable(2, 1, 0) && !device_array_usable(2, 0, 1)\n"
        "        && device_array_usable(3, 1, 0) && device_array_usable(3, -2, 0)\n"
        "        && !device_array_usable(1, 0, 0) && !device_array_usable(0, 0, 0);\n"
        '  std::printf("%d\\n", ok);\n  return ok ? 0 : 1;\n}\n')
    exe = tmp_path / "rule"
    csrc = os.path.join(ROOT, "paper_2510_26180_gb300", "csrc")
    subprocess.run([gxx, "-std=c++17", "-I", csrc, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "1"
