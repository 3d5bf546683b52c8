"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every function include/ccl.h declares, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re
import subprocess

import pytest
import torch

from tests.conftest import ROOT

HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ccl_[a-z_0-9]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2006_09299_gb300 import ccl
    return ccl


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "ccl_analyze" in names and "ccl_fill_holes" in names and "ccl_analyze_batched" in names
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = names - exported
    assert not missing, missing
    # and the Python binding binds every one of them under the same name
    assert names <= set(lib.SIGNATURES), names - set(lib.SIGNATURES)


def test_header_compiles_as_c():
    src = '#include "ccl.h"\nint main(void){ return (int)ccl_node_capacity(3, 3) < 0; }\n'
    r = subprocess.run(["gcc", "-std=c99", "-fsyntax-only", "-I", HEADER_DIR, "-x", "c", "-"],
                       input=src, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_node_capacity(lib):
    from oracle import reference
    for w, h in [(1, 1), (2, 3), (15, 7), (512, 512), (8192, 8192), (4097, 33)]:
        assert lib.node_capacity(w, h) == reference.capacity(w, h)
    assert lib.node_capacity(0, 5) == -1 and lib.node_capacity(5, -1) == -1


def test_status_strings(lib):
    for st in (lib.OK, lib.ERR_ARG, lib.ERR_ALIGN, lib.ERR_CAPACITY, lib.ERR_OOM, lib.ERR_CUDA,
               lib.ERR_ITER_LIMIT, lib.ERR_STATE):
        assert isinstance(lib.status_string(st), str) and lib.status_string(st)


def test_bad_arguments_rejected_before_device(lib):
    c = lib._lib
    h = ctypes.c_void_p()
    assert c.ccl_create(ctypes.byref(h), 0, 5, 16) == lib.ERR_ARG
    assert c.ccl_create(ctypes.byref(h), 5, 0, 16) == lib.ERR_ARG
    assert c.ccl_create(ctypes.byref(h), 20, 5, 16) == lib.ERR_ARG      # pitch < w
    assert c.ccl_create(ctypes.byref(h), 20, 5, 24) == lib.ERR_ALIGN    # pitch % 16
    assert c.ccl_create(ctypes.byref(h), 65536, 65536, 65536) == lib.ERR_ARG  # w*h >= 2^31
    assert c.ccl_create(None, 16, 16, 16) == lib.ERR_ARG
    assert not h.value
    assert c.ccl_create_batched(ctypes.byref(h), 0, 100, 10) == lib.ERR_ARG
    assert c.ccl_analyze(None, None, None, None, None, None, None, None) == lib.ERR_ARG
    assert c.ccl_fill_holes(None, 5, None, None, None, None) == lib.ERR_ARG
    assert c.ccl_set_connectivity(None, 0) == lib.ERR_ARG
    c.ccl_destroy(None)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device path")
def test_no_device_is_an_error_not_a_fallback(lib):
    h = ctypes.c_void_p()
    st = lib._lib.ccl_create(ctypes.byref(h), 64, 64, 64)
    assert st == lib.ERR_CUDA and not h.value


C_DEMO = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c", "abi_demo.c")


def build_c_demo(tmpdir):
    """Compile the plain C caller and link it against libccl.so."""
    import paper_2006_09299_gb300.build as b
    cuda = os.path.dirname(os.path.dirname(b.nvcc())) if os.path.sep in b.nvcc() else "/usr/local/cuda"
    exe = os.path.join(str(tmpdir), "abi_demo")
    lib_dir = os.path.dirname(b.OUT)
    cmd = ["gcc", "-std=c99", "-O1", "-I", HEADER_DIR, "-I", os.path.join(cuda, "include"), C_DEMO, "-o", exe,
           "-L", lib_dir, "-lccl", "-Wl,-rpath," + lib_dir, "-L", os.path.join(cuda, "lib64"), "-lcudart",
           "-Wl,-rpath," + os.path.join(cuda, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_plain_c_caller_links_and_reports_no_device(lib, tmp_path):
    """A C program uses the ABI without Python; here (no GPU) ccl_create
    answers CCL_ERR_CUDA and the program says so."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present: the GPU test runs the program")
    exe = build_c_demo(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 2, r.stdout + r.stderr
    assert "no device" in r.stdout


@pytest.mark.gpu
def test_plain_c_caller_on_gpu(lib, tmp_path):
    exe = build_c_demo(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
