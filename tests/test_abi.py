"""Host-side checks of the C ABI (no GPU needed): libdemag.so builds for
sm_103a, loads, and exports every function include/demag.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "demag.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(demag_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1606_00247_gb300 import build
    from paper_1606_00247_gb300 import _lib

    build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("demag_plan_create", "demag_eval", "demag_plan_destroy", "demag_plan_stats",
              "demag_plan_export_tree", "demag_options_default", "demag_status_string", "demag_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in _declared():
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_options_default_and_status_strings(lib):
    from paper_1606_00247_gb300 import _lib

    o = _lib.demag_options_default()
    assert (o.p, o.leaf_size, o.theta, o.precision, o.near_mode, o.max_batch, o.autotune) == (4, 32, 0.5, 0, 0, 1, 0)
    assert (o.profile, o.m2l_targets_per_cta, o.m2l_kps, o.m2l_promote, o.m2l_promote_rows,
            o.m2l_table_batch, o.sources, o.near_tc, o.graph, o.m2l_split_degree) == (0,) * 10
    # the binding's struct matches the library's: the default fills exactly sizeof(demag_options)
    assert ctypes.sizeof(_lib.demag_options) == 16 * 4 + 8  # sixteen ints, one double
    for s in range(8):
        assert _lib.demag_status_string(s)
    assert _lib.demag_status_string(_lib.DEMAG_ERR_INTERNAL) == "plan audit failed"
    assert _lib.demag_status_string(99) == "unknown status"


def test_null_arguments_rejected_on_host(lib):
    from paper_1606_00247_gb300 import _lib

    st, h = _lib.demag_plan_create(None, 10, None, 1, 4, 32, 0.5, None)
    assert st == _lib.DEMAG_ERR_INVALID_ARG and not h.value
    assert _lib.demag_plan_destroy(None) == _lib.DEMAG_ERR_INVALID_ARG
    assert _lib.demag_plan_audit(None) == _lib.DEMAG_ERR_INVALID_ARG
    assert _lib.demag_eval(None, None, 1, None, None, None) == _lib.DEMAG_ERR_INVALID_ARG


def test_binding_structs_and_constants_match_the_header(tmp_path):
    """The ctypes mirrors of demag_options, demag_stats and demag_tree_export
    have the header's field offsets and sizes, and the binding's constants the
    header's values (a C program built against include/demag.h prints them)."""
    import shutil
    import subprocess

    from paper_1606_00247_gb300 import _lib

    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [("demag_options", _lib.demag_options), ("demag_stats", _lib.demag_stats),
               ("demag_tree_export", _lib.demag_tree_export)]
    consts = [n for n in dir(_lib) if n.startswith("DEMAG_") and isinstance(getattr(_lib, n), int)]
    # the stage order of the per-stage timers and the source models of the Python wrapper
    stages = {f"DEMAG_STAGE_{s.upper()}": k for k, s in enumerate(_lib.STAGES)}
    from paper_1606_00247_gb300 import api

    sources = {f"DEMAG_SOURCES_{k.upper()}": v for k, v in api._SOURCES.items()}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "demag.h"', "int main(void) {"]
    for sname, st in structs:
        lines.append(f'  printf("{sname} sizeof %zu\\n", sizeof({sname}));')
        for fname, _ in st._fields_:
            lines.append(f'  printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    for n in consts + list(stages) + list(sources):
        lines.append(f'  printf("const {n} %d\\n", (int)({n}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for sname, st in structs:
        assert got[(sname, "sizeof")] == ctypes.sizeof(st), sname
        for fname, _ in st._fields_:
            assert got[(sname, fname)] == getattr(st, fname).offset, (sname, fname)
    for n in consts:
        assert got[("const", n)] == getattr(_lib, n), n
    for n, v in {**stages, **sources}.items():
        assert got[("const", n)] == v, n
