"""The oracle and the CUDA path share nothing: neither imports or includes the
other, importing the product does not load the oracle, and the product fails
loudly instead of falling back when its library is missing."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1506_08620_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d or "_build" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def test_product_never_imports_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b)", re.M)
    for f in _files(PKG, (".py",)):
        assert not pat.search(open(f).read()), f


def test_oracle_never_imports_the_product():
    pat = re.compile(r"^\s*(import|from)\s+paper_1506_08620_gb300\b", re.M)
    for f in _files(ORACLE, (".py",)):
        assert not pat.search(open(f).read()), f


def test_no_shared_sources_between_cuda_and_oracle():
    inc = re.compile(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', re.M)
    cuda = {os.path.basename(f) for f in _files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h"))}
    for f in _files(ORACLE, (".c", ".h")):
        for h in inc.findall(open(f).read()):
            assert os.path.basename(h) not in cuda and "csrc" not in h and "ds.h" != os.path.basename(h), (f, h)
    oracle_c = {os.path.basename(f) for f in _files(ORACLE, (".c", ".h"))}
    for f in _files(os.path.join(PKG, "csrc"), (".cu", ".cuh")):
        for h in inc.findall(open(f).read()):
            assert os.path.basename(h) not in oracle_c and "oracle" not in h, (f, h)


def test_importing_the_product_leaves_the_oracle_unloaded():
    code = ("import sys; import paper_1506_08620_gb300 as ds; "
            "assert 'oracle' not in sys.modules, sorted(m for m in sys.modules if 'oracle' in m)")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]


def test_missing_library_fails_loudly():
    code = ("import paper_1506_08620_gb300._abi as a; a.LIB_PATH = '/nonexistent/libds.so'\n"
            "try:\n    a.lib()\nexcept ImportError as e:\n    print('refused:', e)\nelse:\n    raise SystemExit(3)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "refused" in r.stdout, (r.stdout, r.stderr[-2000:])
