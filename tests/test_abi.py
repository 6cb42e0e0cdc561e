"""CPU checks of the C ABI: the library loads, exports every declared symbol,
and the ctypes structures match the C layout of include/lp_sketch_ipm.h.
No CUDA call is made (there may be no GPU)."""

import ctypes
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lp_sketch_ipm.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(lp_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2209_08722_gb300 import _native, build_native
    if not os.path.exists(build_native.lib_path()):
        build_native.build()
    return _native.load()


def test_header_declares_the_solver_entry_points():
    names = _declared_functions()
    for required in ("lp_create", "lp_solve", "lp_normal_solve", "lp_destroy", "lp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_ctypes_signatures_cover_the_header():
    from paper_2209_08722_gb300 import _native
    assert sorted(_native.SIGNATURES) == _declared_functions()


def test_struct_layouts_match_c():
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    from paper_2209_08722_gb300 import _native as nat
    structs = {"lp_matrix": nat.LpMatrix, "lp_options": nat.LpOptions, "lp_result": nat.LpResult,
               "lp_nsolve_info": nat.LpNsolveInfo, "lp_kernel_stats": nat.LpKernelStats,
               "lp_iter_record": nat.LpIterRecord, "lp_phase1_info": nat.LpPhase1Info,
               "lp_state": nat.LpState}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "abi.c")
        exe = os.path.join(td, "abi")
        open(c, "w").write("\n".join(lines))
        subprocess.run([gcc, c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        parts = line.split()
        got[(parts[0], parts[1])] = int(parts[2])
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert got[(cname, field)] == getattr(cls, field).offset, (cname, field)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2209_08722_gb300 import _native
    with pytest.raises(ImportError):
        _native.load(str(tmp_path / "nope.so"))


def test_status_codes_match_the_header():
    """Every status and error code of the header has the same value in the
    Python binding, and a name in its status table."""
    from paper_2209_08722_gb300 import _native as nat
    src = open(HEADER).read()
    codes = dict((name, int(val)) for name, val in
                 re.findall(r"^#define\s+(LP_(?:OK|ERR_\w+|STATUS_\w+|WARN_\w+))\s+(-?\d+)", src, flags=re.M))
    assert "LP_OK" in codes and "LP_ERR_ARG" in codes and "LP_STATUS_STALLED" in codes
    for name, val in codes.items():
        assert getattr(nat, name) == val, name
        assert nat.STATUS_NAMES[val] == name, name
    assert set(nat.STATUS_NAMES) == set(codes.values())
