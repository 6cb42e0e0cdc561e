"""The oracle and the CUDA path stay apart (CPU checks).

The product (the package and its CUDA sources) never imports or includes the
oracle; the oracle never imports the product; the shared input generators
(lpgen) import neither.  Importing the product does not load any oracle
module, and nothing committed outside the working folder reads that folder.
"""

import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2209_08722_gb300")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d or os.sep + "_lib" in d:
            continue
        for f in names:
            if f.endswith(exts):
                yield os.path.join(d, f)


def _imports(path):
    src = open(path, encoding="utf-8").read()
    if path.endswith(".py"):
        return re.findall(r"^\s*(?:from|import)\s+([\w.]+)", src, flags=re.M)
    return re.findall(r'^\s*#\s*include\s+[<"]([^>"]+)[>"]', src, flags=re.M)


def test_product_does_not_import_the_oracle():
    for path in _files(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")):
        for name in _imports(path):
            assert not re.match(r"(\.\./)*oracle\b", name), (path, name)
    for path in _files(os.path.join(ROOT, "include"), (".h",)):
        assert "oracle" not in " ".join(_imports(path)), path


def test_oracle_and_generators_do_not_import_the_product():
    for top in ("oracle", "lpgen"):
        for path in _files(os.path.join(ROOT, top), (".py",)):
            for name in _imports(path):
                assert not name.startswith("paper_2209_08722_gb300"), (path, name)
                if top == "lpgen":
                    assert not name.startswith("oracle"), (path, name)


def test_importing_the_product_loads_no_oracle_module():
    code = ("import sys, paper_2209_08722_gb300, paper_2209_08722_gb300.solver, "
            "paper_2209_08722_gb300._native; "
            "print(sorted(m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, check=True)
    assert out.stdout.strip() == "[]", out.stdout


def test_committed_code_does_not_read_the_working_folder():
    tops = [PKG, os.path.join(ROOT, "tests"), os.path.join(ROOT, "oracle"), os.path.join(ROOT, "lpgen"),
            os.path.join(ROOT, "include")]
    files = [p for t in tops for p in _files(t, (".py", ".cu", ".cuh", ".h", ".cpp"))]
    files += [os.path.join(ROOT, f) for f in ("bench.py", "__graft_entry__.py")]
    work = re.compile(r"""["'/]_work\b""")
    for path in files:
        if os.path.abspath(path) == os.path.abspath(__file__):
            continue
        src = open(path, encoding="utf-8").read()
        assert not work.search(src), path


def test_smoke_refuses_to_run_without_a_gpu():
    # no CPU fallback anywhere: without a CUDA device smoke() stops at once
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: smoke() runs for real there")
    import __graft_entry__
    with pytest.raises(AssertionError, match="cuda"):
        __graft_entry__.smoke()
