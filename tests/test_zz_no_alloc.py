"""ccl_analyze_static: the analysis for callers that cannot allocate device
memory (their memory belongs to another allocator, or they run loops that
must not call cudaMalloc after start-up). Its scratch is a fixed per-device
array inside the library; these tests check, through the C ABI, that two
calls in a row give exactly what the allocating entry point gives and what
the CPU oracle gives (also at the documented size limits), and that
oversized images are refused before anything is enqueued.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import reference as orc
from paper_2006_09299_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccl():
    import __graft_entry__ as g
    g.build()
    from paper_2006_09299_gb300 import ccl as m
    return m


def reference_outputs(ccl, padded, w):
    """The same image through ccl_create + ccl_analyze."""
    h, pitch = padded.shape
    ctx = ccl.Context(w, h, pitch)
    out = ctx.analyze(torch.from_numpy(padded).cuda())
    n, _, _, st = ctx.get_counts()
    assert st == 0
    res = (out.fg.cpu(), out.bg.cpu(), out.parent[:n].cpu(), out.features[:, :n].cpu(), out.counts[:3].cpu())
    ctx.close()
    return res


def test_static_matches_allocating_entry_point_twice(ccl):
    cases = [(inputs.granular(700, 1400, 0.5, 1, 11), 1400, 1408),
             (inputs.granular(513, 2000, 0.35, 3, 12), 2000, 2000)]
    for padded_img, w, pitch in cases:
        padded = inputs.pitched(padded_img, pitch)
        ref = reference_outputs(ccl, padded, w)
        h = padded.shape[0]
        d = torch.from_numpy(padded).cuda()
        out = ccl.Analysis(w, h, ccl.node_capacity(w, h), True, "cuda")
        for call in range(2):
            out.fg.fill_(-7)
            out.bg.fill_(-7)
            ccl.analyze_static(d, w, out)
            torch.cuda.synchronize()
            n = out.n
            assert out.status() == 0, call
            assert torch.equal(out.counts[:3].cpu(), ref[4]), call
            assert torch.equal(out.fg.cpu(), ref[0]), call
            assert torch.equal(out.bg.cpu(), ref[1]), call
            assert torch.equal(out.parent[:n].cpu(), ref[2]), call
            assert torch.equal(out.features[:, :n].cpu(), ref[3]), call


@pytest.mark.parametrize("w,h,d,g", [
    (1024, 1024, 0.5, 1),    # exactly 2^20 pixels
    (4096, 256, 0.45, 2),    # the widest side allowed, four tile columns
    (256, 4096, 0.5, 3),     # the tallest side allowed
    (1, 4096, 0.5, 1),       # one pixel wide
    (1023, 1025, 0.4, 1),    # w not a multiple of 4: scalar label stores
])
def test_static_at_its_limits_matches_the_oracle_twice(ccl, w, h, d, g):
    """Images at the documented size limits, against the CPU oracle itself
    (labels, tree, features, counts), on two calls in a row."""
    img = inputs.granular(h, w, d, g, 1000 + w + h)
    pitch = -(-w // 16) * 16
    padded = inputs.pitched(img, pitch)
    ref = orc.analyze(padded, w=w)
    dev = torch.from_numpy(padded).cuda()
    out = ccl.Analysis(w, h, ccl.node_capacity(w, h), True, "cuda")
    for call in range(2):
        out.fg.fill_(-7)
        out.bg.fill_(-7)
        ccl.analyze_static(dev, w, out)
        torch.cuda.synchronize()
        n = out.n
        assert out.status() == 0, call
        assert n == ref["n"], call
        assert out.counts[:3].cpu().tolist() == ref["counts"][:3].tolist(), call
        np.testing.assert_array_equal(out.fg.cpu().numpy(), ref["fg"])
        np.testing.assert_array_equal(out.bg.cpu().numpy(), ref["bg"])
        np.testing.assert_array_equal(out.parent[:n].cpu().numpy(), ref["parent"])
        np.testing.assert_array_equal(out.features[:, :n].cpu().numpy(), ref["feat"])


def test_static_refuses_oversized_images(ccl):
    lib = ccl._lib
    w, h = 2048, 1024   # 2 Mpx > the 1 Mpx limit
    buf = torch.zeros((h, w), dtype=torch.uint8, device="cuda")
    counts = torch.zeros(4, dtype=torch.int32, device="cuda")
    par = torch.zeros(16, dtype=torch.int32, device="cuda")
    feat = torch.zeros((7, 16), dtype=torch.int64, device="cuda")
    st = lib.ccl_analyze_static(ctypes.c_void_p(buf.data_ptr()), w, h, w, None, None,
                                ctypes.c_void_p(par.data_ptr()), ctypes.c_void_p(feat.data_ptr()), 16,
                                ctypes.c_void_p(counts.data_ptr()), None)
    assert st == ccl.ERR_CAPACITY
    st = lib.ccl_analyze_static(ctypes.c_void_p(buf.data_ptr()), 5000, 10, 5008, None, None,
                                ctypes.c_void_p(par.data_ptr()), ctypes.c_void_p(feat.data_ptr()), 16,
                                ctypes.c_void_p(counts.data_ptr()), None)
    assert st == ccl.ERR_CAPACITY
    torch.cuda.synchronize()
    assert int(counts.abs().sum()) == 0   # nothing was enqueued
