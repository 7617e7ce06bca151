"""The range-checking build of the library (libds_bounds.so, -DDS_DEBUG_BOUNDS):
every table and knot gather of the search kernels checks its index against
the extent it reads.  On valid inputs of every search form (single array in
both precisions and every table form, batched, learned with and without
stored values and with escaped cell blocks, the logarithmic searches) the
results equal the oracle's and no check fires: the indices are in range by
construction.  A table entry moved one knot past the end, inside the padding
of the table's own allocation, makes the knot-gather check fire."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def child_result():
    from paper_1506_08620_gb300 import build
    build.build(bounds=True)
    env = dict(os.environ, DS_LIBRARY="bounds")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_child.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_every_search_form_is_exact_with_no_index_out_of_range(child_result):
    valid = {k: v for k, v in child_result.items() if not k.startswith("moved_entry")}
    assert len(valid) >= 60
    bad = {k: v for k, v in valid.items() if v != [0, 0]}
    assert not bad, bad


@pytest.mark.parametrize("path", ["smem", "global"])
def test_a_moved_table_entry_is_caught(child_result, path):
    from paper_1506_08620_gb300 import _abi
    assert child_result["moved_entry_%s" % path][1] == _abi.DS_DEVERR_BOUNDS | (_abi.DS_BS_X << 8)
