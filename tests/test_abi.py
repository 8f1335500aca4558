"""C-ABI checks that need no GPU: the library builds and loads, exports
every entry point include/lbo.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import pytest

from paper_2503_09580_gb300 import lbo
from paper_2503_09580_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return lbo.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbo.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbo_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(lbo.EXPORTS)


def test_status_strings(lib):
    assert lib.lbo_status_string(0) == b"ok"
    assert lib.lbo_status_string(7) == b"unsupported configuration"


def test_argument_errors_before_any_launch(lib):
    h = ctypes.c_void_p()
    assert lib.lbo_plan_create(17, 8.0, 0.5, 16, ctypes.byref(h)) == 7   # odd / unbuilt N
    assert h.value is None
    assert lib.lbo_plan_create(32, -1.0, 0.5, 32, ctypes.byref(h)) == 1
    assert lib.lbo_plan_create(32, 8.0, 0.3, 32, ctypes.byref(h)) == 1  # omega outside [0.5, 1]
    assert lib.lbo_plan_create(32, 8.0, 0.5, 0, ctypes.byref(h)) == 1
    assert lib.lbo_plan_set(None, 0, 1.0) == 1
    assert lib.lbo_apply_linearized(None, None, None, None, 1) == 1
    assert lib.lbo_plan_sync(None) == 1
    lib.lbo_plan_destroy(None)


def test_binding_marshals_profile_and_noalloc_calls(lib):
    """The binding's wrappers call each entry point with its own argument
    list (no GPU needed: a NULL plan is rejected before any launch)."""
    plan = lbo.Plan.__new__(lbo.Plan)
    plan._h = ctypes.c_void_p()
    with pytest.raises(lbo.LboError):
        plan.profile(True)
    assert lib.lbo_plan_profile_count(None) == 0
    name, cnt, ms = ctypes.c_char_p(), ctypes.c_int(), ctypes.c_double()
    assert lib.lbo_plan_profile_get(None, 0, ctypes.byref(name), ctypes.byref(cnt), ctypes.byref(ms)) == 1
    assert lib.lbo_apply_linearized_noalloc(None, None, None, None, 1) == 1
    assert lib.lbo_noalloc_scratch_bytes() == 64 << 20
    plan._h = None


@pytest.mark.parametrize("cname,pystruct", [("lbo_problem", lbo.Problem), ("lbo_newton_stats", lbo.NewtonStats)])
def test_binding_structs_match_the_header_layout(cname, pystruct, tmp_path):
    """Every field of the ctypes mirrors sits at the offset the C compiler
    gives it in include/lbo.h, and the sizes agree."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = [n for n, _ in pystruct._fields_]
    body = "".join('  printf("%%zu\\n", offsetof(%s, %s));\n' % (cname, n) for n in names)
    src = ("#include <stdio.h>\n#include <stddef.h>\n#include \"lbo.h\"\nint main(void) {\n"
           '  printf("%%zu\\n", sizeof(%s));\n%s  return 0;\n}\n' % (cname, body))
    (tmp_path / "layout.c").write_text(src)
    exe = str(tmp_path / "layout")
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(tmp_path / "layout.c"), "-o", exe])
    got = [int(x) for x in subprocess.check_output([exe]).split()]
    assert got[0] == ctypes.sizeof(pystruct)
    assert got[1:] == [getattr(pystruct, n).offset for n in names]


def test_binding_option_and_precision_codes_match_the_header():
    """The binding's option keys and precision names carry the numbers the
    header's enums give them (LBO_OPT_<NAME> = k; LBO_PREC_<NAME> = k)."""
    hdr = open(os.path.join(ROOT, "include", "lbo.h")).read()
    # enumerator lines only (the comments quote options too)
    opts = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"^\s*LBO_OPT_(\w+)\s*=\s*(\d+)", hdr, re.M)}
    precs = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"^\s*LBO_PREC_(\w+)\s*=\s*(\d+)", hdr, re.M)}
    assert opts and precs
    binding = {k.lower(): v for k, v in lbo.LBO_OPT.items()}
    assert binding == opts
    assert lbo.PRECISION == precs
