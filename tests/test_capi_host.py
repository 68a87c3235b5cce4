"""The C-ABI library loads, exports every entry point declared in include/icon.h and
rejects bad arguments on the host (no GPU needed for any of these calls)."""
import ctypes
import os
import re

from tests.conftest import ROOT


def _declared():
    text = open(os.path.join(ROOT, "include", "icon.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(icon_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(built_lib):
    names = _declared()
    assert len(names) >= 20
    lib = ctypes.CDLL(built_lib)
    for n in names:
        getattr(lib, n)          # dlsym; raises AttributeError if missing


def test_host_argument_checks(built_lib):
    from paper_2511_02021_gb300 import capi as C
    lib = C._lib
    h = ctypes.c_void_p()
    assert lib.icon_grid_build(3, 2, 20, ctypes.byref(h)) == C.ICON_EINVAL
    assert b"root 2" in lib.icon_last_error()
    assert lib.icon_grid_build(2, 11, 20, ctypes.byref(h)) == C.ICON_EINVAL
    assert lib.icon_grid_build(2, 2, 0, ctypes.byref(h)) == C.ICON_EINVAL
    assert lib.icon_grid_build(2, 2, 20, None) == C.ICON_EINVAL
    assert h.value is None                         # out-pointer untouched on error
    f = C.ALLOC_FN(lambda n, c: 0)
    assert lib.icon_set_allocator(ctypes.cast(f, ctypes.c_void_p), None, None) == C.ICON_EINVAL
    assert lib.icon_set_allocator(None, None, None) == C.ICON_OK
    assert lib.icon_state_init(None, 0, 0, ctypes.byref(h)) == C.ICON_EINVAL
    assert lib.icon_dycore_step(None, 1.0, 1) == C.ICON_EINVAL
    assert lib.icon_global_mass(None, None) == C.ICON_EINVAL
    assert lib.icon_ensemble_create(None, 0, ctypes.byref(h)) == C.ICON_EINVAL
    assert lib.icon_ensemble_step_profile(None, None, 5, None, None) == C.ICON_EINVAL
    names = [C.icon_ensemble_phase_name(k) for k in range(C.ICON_ENS_PHASE_COUNT)]
    assert len(set(names)) == C.ICON_ENS_PHASE_COUNT and None not in names
    assert C.icon_ensemble_phase_name(-1) is None and C.icon_ensemble_phase_name(C.ICON_ENS_PHASE_COUNT) is None
    n = ctypes.c_int()
    assert lib.icon_state_add_tracers(None, 1) == C.ICON_EINVAL
    assert lib.icon_state_set_option(None, 1, 0.0) == C.ICON_EINVAL
    assert lib.icon_state_set_option(None, 2, 0.0) == C.ICON_EINVAL
    assert lib.icon_state_set_option(None, 3, 1.0) == C.ICON_EINVAL
    assert lib.icon_state_tracers(None, ctypes.byref(n)) == C.ICON_EINVAL
    assert lib.icon_state_set_tracer(None, 0, None, 0) == C.ICON_EINVAL
    assert lib.icon_state_copy_tracer(None, 0, None, 0) == C.ICON_EINVAL
    lib.icon_grid_free(None)
    lib.icon_state_free(None)
    lib.icon_ensemble_free(None)


def test_case_params_layout_matches_the_header(tmp_path):
    """The Python binding's icon_case_params has the C struct's size and field offsets
    (compiled from include/icon.h with the host C compiler)."""
    import shutil
    import subprocess
    import pytest
    from paper_2511_02021_gb300 import capi as C
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    fields = [f for f, _ in C.CaseParams._fields_]
    src = tmp_path / "layout.c"
    body = "".join('printf("%%zu\\n", offsetof(icon_case_params, %s));\n' % f for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include <stdint.h>\n#include "icon.h"\n'
                   'int main(void) {\nprintf("%zu\\n", sizeof(icon_case_params));\n' + body + 'return 0;\n}\n')
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(C.CaseParams)
    assert out[1:] == [getattr(C.CaseParams, f).offset for f in fields]


def test_binding_constants_match_the_header():
    """Every ICON_* integer constant of the binding equals the header's #define or enum value."""
    import re
    from paper_2511_02021_gb300 import capi as C
    text = open(os.path.join(ROOT, "include", "icon.h")).read()
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define (ICON_\w+) (-?\d+)\b", text, re.M)}
    defs.update({m.group(1): int(m.group(2)) for m in re.finditer(r"^\s+(ICON_\w+) = (-?\d+),", text, re.M)})
    shared = [n for n in defs if hasattr(C, n)]
    assert {"ICON_KIND_COUNT", "ICON_ENS_PHASE_COUNT", "ICON_OK", "ICON_EINVAL"} <= set(shared)
    for n in shared:
        assert getattr(C, n) == defs[n], n


def test_every_environment_switch_is_documented():
    """Each environment variable the library reads is described in the header a user reads."""
    csrc = os.path.join(ROOT, "paper_2511_02021_gb300", "csrc")
    names = set()
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".h")):
            names |= set(re.findall(r'getenv\("([A-Z0-9_]+)"\)', open(os.path.join(csrc, f)).read()))
    assert {"ICON_MIXED_COLUMN", "ICON_TUNE_CACHE", "ICON_STEP_OVERLAP"} <= names
    header = open(os.path.join(ROOT, "include", "icon.h")).read()
    for n in sorted(names):
        assert n in header, n
