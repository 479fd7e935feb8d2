"""The C-ABI library builds, loads and exports every entry point that
include/dock.h declares; the binding refuses to run without it.  No compute
call is made (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dock.h")).read()
    return sorted(set(re.findall(r"^DOCK_API [^(]*?\b(dock_\w+)\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["dock_object_grid", "dock_sweep_grid", "dock_search_so3", "dock_refine_se3", "dock_register"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2605_21398_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2605_21398_gb300 import dock
    have = {s[0] for s in dock.SIGNATURES}
    assert set(_declared()) <= have | {"dock_version"}


def test_params_default_is_table_I():
    from paper_2605_21398_gb300 import build, dock
    build.build()
    p = dock.default_params()
    assert (p.tau_out1, p.tau_in1, p.deep_value, p.tau_out2, p.tau_in2) == (0.5, 0.2, -50.0, 0.2, 0.03)
    assert p.k_slope == 15.0 and p.iters == 20
    assert p.solver == dock.SOLVER_GAUSS_NEWTON and p.lbfgs_evals == 100 and p.lbfgs_pgtol == 1e-5
    assert ctypes.sizeof(dock.Params) == 128     # 12 doubles, 4 int32, 2 doubles: no padding


def test_binding_fails_loudly_without_the_library(monkeypatch):
    from paper_2605_21398_gb300 import dock
    monkeypatch.setattr(dock, "_lib", None)
    monkeypatch.setattr(dock, "LIB_PATH", os.path.join(ROOT, "does-not-exist", "libdock.so"))
    with pytest.raises(RuntimeError):
        dock.lib()


# ctypes structure of the binding -> the C struct of include/dock.h it mirrors
_STRUCTS = {"Params": "dock_params", "Probe": "dock_probe", "Candidate": "dock_candidate", "Peak": "dock_peak",
            "SearchDesc": "dock_search_desc", "Refined": "dock_refined", "RegisterDesc": "dock_register_desc",
            "Result": "dock_result", "Request": "dock_request", "Tuning": "dock_tuning",
            "KernelStat": "dock_kernel_stat"}


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure has the size and field offsets that a C compiler
    gives the header's struct (a field added to one side only fails here)."""
    import shutil
    import subprocess
    from paper_2605_21398_gb300 import dock
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "dock.h"', 'int main(void) {']
    for py, c in _STRUCTS.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (py, c))
        for name, _ in getattr(dock, py)._fields_:
            cname = name[:-1] if name.endswith("_") else name   # lambda_ (a Python keyword) is lambda in C
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (py, name, c, cname))
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for py in _STRUCTS:
        cls = getattr(dock, py)
        assert int(got["%s size" % py]) == ctypes.sizeof(cls), py
        for name, _ in cls._fields_:
            assert int(got["%s.%s" % (py, name)]) == getattr(cls, name).offset, (py, name)
