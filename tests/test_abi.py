"""The C ABI: liblrvol.so builds, loads without a GPU, and exports every entry
point include/lrvol.h declares; argument checks that precede any CUDA call
return LRVOL_ERR_ARG.  No compute call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1707_01170_gb300 import build as cuda_build
from paper_1707_01170_gb300 import lrvol as lv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lrvol.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lrvol_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return lv.load()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["lrvol_create", "lrvol_build_accel", "lrvol_to_bezier", "lrvol_render", "lrvol_lookup",
              "lrvol_eval", "lrvol_get_bezier", "lrvol_stats", "lrvol_status_string", "lrvol_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(lv.EXPORTED) == sorted(_declared())


def test_status_strings(lib):
    for s in (0, -1, -2, -3, -4, -5, -6, -7):
        assert lib.lrvol_status_string(s)
    assert lib.lrvol_status_string(lv.ERR_STATE).decode() == "call out of order"


def test_argument_errors_before_any_cuda_call(lib):
    vp = ctypes.c_void_p
    h = vp()
    deg = np.array([3, 3, 3], dtype=np.int32)
    box = np.array([[0, 0, 0, 1, 1, 1.0]])
    kn = np.zeros((1, 15))
    one = np.ones(1)
    # null pointers
    assert lib.lrvol_create(None, 1, 1, box.ctypes.data, 1, kn.ctypes.data, one.ctypes.data, one.ctypes.data,
                            ctypes.byref(h)) == lv.ERR_ARG
    # ncomp 2
    assert lib.lrvol_create(deg.ctypes.data, 2, 1, box.ctypes.data, 1, kn.ctypes.data, one.ctypes.data,
                            one.ctypes.data, ctypes.byref(h)) == lv.ERR_ARG
    # degree 5
    d5 = np.array([5, 3, 3], dtype=np.int32)
    assert lib.lrvol_create(d5.ctypes.data, 1, 1, box.ctypes.data, 1, kn.ctypes.data, one.ctypes.data,
                            one.ctypes.data, ctypes.byref(h)) == lv.ERR_ARG
    # box outside [0,1]
    bad = np.array([[0, 0, 0, 1.5, 1, 1.0]])
    assert lib.lrvol_create(deg.ctypes.data, 1, 1, bad.ctypes.data, 1, kn.ctypes.data, one.ctypes.data,
                            one.ctypes.data, ctypes.byref(h)) == lv.ERR_ARG
    # decreasing knots
    kd = np.zeros((1, 15))
    kd[0, :5] = [0, 0.5, 0.25, 1, 1]
    assert lib.lrvol_create(deg.ctypes.data, 1, 1, box.ctypes.data, 1, kd.ctypes.data, one.ctypes.data,
                            one.ctypes.data, ctypes.byref(h)) == lv.ERR_ARG
    assert "non-decreasing" in lv.last_error()
    # null handles
    b = np.array([4, 4, 4], dtype=np.int32)
    assert lib.lrvol_build_accel(None, b.ctypes.data, None) == lv.ERR_ARG
    assert lib.lrvol_to_bezier(None, 0, None) == lv.ERR_ARG
    assert lib.lrvol_render(None, None, None, None, None, None) == lv.ERR_ARG
    assert lib.lrvol_lookup(None, None, 0, None, None) == lv.ERR_ARG
    assert lib.lrvol_get_bezier(None, None) == lv.ERR_ARG
    lib.lrvol_destroy(None)


def test_struct_layouts_match_header(tmp_path):
    """Sizes and field offsets of the ctypes mirrors equal what a C compiler
    makes of include/lrvol.h."""
    fields = {"lrvol_camera": lv.Camera, "lrvol_tf": lv.TF, "lrvol_step": lv.Step, "lrvol_stats_t": lv.Stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lrvol.h"', "int main(void) {"]
    for cname, cls in fields.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for cname, cls in fields.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def test_binding_constants_match_header(tmp_path):
    """Every enum value and size constant the binding mirrors equals what a C
    compiler makes of include/lrvol.h."""
    names = {"OK": "LRVOL_OK", "ERR_ARG": "LRVOL_ERR_ARG", "ERR_OOM": "LRVOL_ERR_OOM", "ERR_CUDA": "LRVOL_ERR_CUDA",
             "ERR_STATE": "LRVOL_ERR_STATE", "ERR_BOUNDS": "LRVOL_ERR_BOUNDS", "ERR_TIMEOUT": "LRVOL_ERR_TIMEOUT",
             "ERR_UNSUPPORTED": "LRVOL_ERR_UNSUPPORTED", "ORTHO": "LRVOL_ORTHO", "PERSP": "LRVOL_PERSP",
             "MLP_IN": "LRVOL_MLP_IN", "MLP_HIDDEN": "LRVOL_MLP_HIDDEN", "MLP_PARAMS": "LRVOL_MLP_PARAMS",
             "MLP_PACKED": "LRVOL_MLP_PACKED", "BAND_ROWS": "LRVOL_BAND_ROWS"}
    for group in ("STEP_FIXED STEP_HEURISTIC STEP_LEARNED", "FIELD_SCALAR FIELD_MAGNITUDE FIELD_COMPONENT",
                  "STORE_F32 STORE_F16 STORE_BF16", "SHADE_NONE SHADE_GRADIENT", "SPLIT_BALANCED SPLIT_MIDPOINT",
                  "REQ_QUEUED REQ_RUNNING REQ_DONE REQ_FAILED"):
        names.update({n: "LRVOL_" + n for n in group.split()})
    methods = {m: "LRVOL_" + m for m in lv.SL_METHODS}
    rules = {r: "LRVOL_SL_" + r.upper() for r in lv.SL_RULES}
    lines = ['#include <stdio.h>', '#include "lrvol.h"', "int main(void) {"]
    for py, c in {**names, **methods, **rules}.items():
        lines.append(f'  printf("{py} %ld\\n", (long)({c}));')
    lines.append("  return 0; }")
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "consts"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for py in names:
        assert int(got[py]) == getattr(lv, py), py
    for i, m in enumerate(lv.SL_METHODS):
        assert int(got[m]) == i, m                   # the binding passes the list index as the method
    for i, r in enumerate(lv.SL_RULES):
        assert int(got[r]) == i, r


def test_missing_library_fails_loudly(tmp_path):
    """Without the compiled library the binding raises on first use; there is
    no CPU fallback (a fresh interpreter, so no library is loaded already)."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1707_01170_gb300 import lrvol as lv\n"
            "try:\n"
            "    lv.load(%r)\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "else:\n"
            "    print('loaded')\n") % (ROOT, str(tmp_path / "no_such" / "liblrvol.so"))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("raised:") and "not built" in out.stdout
