"""The C-ABI library builds, loads and exports every entry point that
include/supcg.h declares; argument errors come back as status codes without
touching a GPU."""
import ctypes as C
import os
import re

import pytest

import paper_1807_10151_gb300 as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "supcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(supcg_\w+)\s*\(", src)))


def test_header_declares_the_binding_names():
    assert declared_symbols() == sorted(S.EXPORTED)


def test_library_exports_every_declared_symbol():
    L = S.load()
    for name in declared_symbols():
        assert hasattr(L, name), name
    out = os.popen(f"nm -D --defined-only {S.lib_path()}").read()
    for name in declared_symbols():
        assert re.search(rf"\bT {name}\b", out), name


def test_argument_errors_are_status_codes():
    L = S.load()
    assert L.supcg_project(None, None, None, 1, None) == -1
    assert L.supcg_backproject(None, None, None, 1, None) == -1
    assert L.supcg_destroy_geometry(None) == -1
    h = C.c_void_p()
    # invalid sizes are rejected before any CUDA call
    assert L.supcg_create_geometry(0, 4, 0.25, 4, None, 5, 0.0, 0.0, 0, C.byref(h)) == -1
    assert L.supcg_create_geometry(4, 4, -1.0, 4, None, 5, 0.0, 0.0, 0, C.byref(h)) == -1
    assert L.supcg_create_geometry(4, 4, 0.25, 4, None, 5, 0.0, 0.0, 7, C.byref(h)) == -1
    assert L.supcg_get_mirror_pairs(None, C.byref(C.c_int())) == -1
    assert S.supcg_status_string(-5).startswith("S_TV")
    assert S.supcg_status_string(0) == "ok"


def test_wait_limit_and_barrier_hook_check_their_arguments():
    """Host-only settings: out-of-range values are refused, valid ones accepted."""
    L = S.load()
    assert L.supcg_set_wait_limit(0) == -1
    assert L.supcg_set_barrier_shortfall(-1) == -1
    assert L.supcg_set_barrier_shortfall(1025) == -1
    try:
        assert L.supcg_set_wait_limit(1 << 10) == 0
        assert L.supcg_set_barrier_shortfall(2) == 0
    finally:
        assert L.supcg_set_barrier_shortfall(0) == 0
        assert L.supcg_set_wait_limit(S.DEFAULT_WAIT_LIMIT) == 0


def test_param_struct_layout_matches_header():
    # offsets follow the C layout of supcg_params / supcg_report on LP64
    assert S.Params.a.offset == 8 and S.Params.max_iter.offset == 48 and S.Params.max_trials.offset == 56
    assert S.Params.bayes_r.offset == 80 and S.Params.bayes_mu.offset == 88
    assert C.sizeof(S.Params) == 96
    assert S.Report.ell.offset == 8 and S.Report.n_learned.offset == 48 and C.sizeof(S.Report) == 56


def test_art_struct_layout_matches_the_compiled_header(tmp_path):
    """supcg_art_params / supcg_art_report as the C compiler lays them out from
    include/supcg.h, against the binding's ctypes structures."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "layout.c"
    src.write_text(
        "#include <stddef.h>\n#include <stdio.h>\n#include \"supcg.h\"\n"
        "int main(void) {\n"
        "  printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\", offsetof(supcg_art_params, r),\n"
        "         offsetof(supcg_art_params, lambda), offsetof(supcg_art_params, mu),\n"
        "         offsetof(supcg_art_params, cycles), offsetof(supcg_art_params, K),\n"
        "         offsetof(supcg_art_params, a), offsetof(supcg_art_params, gamma),\n"
        "         offsetof(supcg_art_params, max_trials), sizeof(supcg_art_params));\n"
        "  printf(\"%zu %zu %zu %zu %zu\\n\", offsetof(supcg_art_report, cycles), offsetof(supcg_art_report, ell),\n"
        "         offsetof(supcg_art_report, mu), offsetof(supcg_art_report, status), sizeof(supcg_art_report));\n"
        "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    p = [int(v) for v in lines[0].split()]
    r = [int(v) for v in lines[1].split()]
    A, R = S.ArtParams, S.ArtReport
    assert p == [A.r.offset, A.lam.offset, A.mu.offset, A.cycles.offset, A.K.offset, A.a.offset, A.gamma.offset,
                 A.max_trials.offset, C.sizeof(A)]
    assert r == [R.cycles.offset, R.ell.offset, R.mu.offset, R.status.offset, C.sizeof(R)]
