"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/ds.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ds.h")).read()
    return sorted(set(re.findall(r"^DS_API\s+[\w\s\*]*?\b(ds_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libds():
    from paper_1506_08620_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("ds_build", "ds_search", "ds_batch_build", "ds_batch_search", "ds_learned_build",
              "ds_learned_search", "ds_info", "ds_free"):
        assert n in names


def test_library_exports_every_declared_symbol(libds):
    missing = [n for n in _declared() if not hasattr(libds, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libds):
    from paper_1506_08620_gb300 import _abi
    assert sorted(_declared()) == _abi.EXPORTED


def test_status_strings_and_version(libds):
    from paper_1506_08620_gb300 import _abi
    L = _abi.lib()
    assert L.ds_abi_version() == 1
    assert L.ds_status_str(_abi.DS_E_OVERFLOW) == b"DS_E_OVERFLOW"
    assert L.ds_status_str(_abi.DS_OK) == b"DS_OK"


def test_argument_errors_need_no_gpu(libds):
    from paper_1506_08620_gb300 import _abi
    L = _abi.lib()
    out = ctypes.c_void_p()
    # null knots and too few knots are rejected before any CUDA call
    assert L.ds_build(None, 10, _abi.DS_F32, 0, None, ctypes.byref(out)) == _abi.DS_E_ARG
    assert L.ds_build(ctypes.c_void_p(16), 1, _abi.DS_F32, 0, None, ctypes.byref(out)) == _abi.DS_E_ARG
    assert L.ds_build(ctypes.c_void_p(16), 10, 7, 0, None, ctypes.byref(out)) == _abi.DS_E_ARG
    assert L.ds_build(ctypes.c_void_p(16), 10, _abi.DS_F32, 1 << 20, None, ctypes.byref(out)) == _abi.DS_E_ARG
    assert b"bad argument" in L.ds_last_error()
    assert L.ds_search(None, None, 0, None, None) == _abi.DS_E_ARG
    L.ds_free(None)


def test_cuda_sources_target_sm103a_only():
    from paper_1506_08620_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_static_build_source_allocates_nothing():
    """The allocation-free build's translation unit names no allocating call:
    its scratch is the file-scope __device__ array, looked up by address."""
    src = open(os.path.join(ROOT, "paper_1506_08620_gb300", "csrc", "ds_static.cu")).read()
    code = "\n".join(l.split("//")[0] for l in src.splitlines())
    for call in ("cudaMalloc", "cudaFree", "cudaMallocAsync", "cudaFreeAsync", "cudaMallocHost", "cudaHostAlloc",
                 "cudaMallocManaged", "cudaMallocPitch", "malloc(", "new ", "std::vector"):
        assert call not in code, call
    assert "__device__ __align__(256)" in code and "cudaGetSymbolAddress" in code


def test_every_device_allocation_goes_through_the_tracked_wrapper():
    # the allocation-failure hook and the live-allocation count see every
    # device allocation only if no source calls the runtime's allocator itself
    import re
    csrc = os.path.join(ROOT, "paper_1506_08620_gb300", "csrc")
    raw = re.compile(r"\bcuda(Malloc|MallocAsync|Free|FreeAsync|MallocManaged|MallocPitch)\s*\(")
    for f in sorted(os.listdir(csrc)):
        if not f.endswith((".cu", ".cuh")):
            continue
        for n, line in enumerate(open(os.path.join(csrc, f)), 1):
            code = line.split("//")[0]
            if raw.search(code):
                # only the wrapper itself may call the runtime
                assert f == "ds_core.cu", "%s:%d calls the CUDA allocator directly: %s" % (f, n, line.strip())


def test_allocation_hook_needs_no_device(libds):
    n, b = ctypes.c_int64(-1), ctypes.c_int64(-1)
    assert libds.ds_debug_fail_alloc(ctypes.c_int64(3)) == 0
    assert libds.ds_debug_alloc_stats(ctypes.byref(n), ctypes.byref(b)) == 0
    assert (n.value, b.value) == (0, 0)
    assert libds.ds_debug_fail_alloc(ctypes.c_int64(-1)) == 0
