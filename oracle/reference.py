"""ctypes front end of the C flood-fill oracle (ccl_oracle.c).

TEST INFRASTRUCTURE ONLY (see the package docstring). `build()` compiles the C
file with gcc into oracle/liboracle.so; `analyze` and `fill` return numpy
arrays laid out exactly like the library's outputs so that tests compare them
element by element.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccl_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

NF = 7  # AREA, XMIN, YMIN, XMAX, YMAX, SX, SY
AREA, XMIN, YMIN, XMAX, YMAX, SX, SY = range(NF)
INT64_MAX = np.iinfo(np.int64).max

_lib = None


def build(force=False):
    """Compile ccl_oracle.c into liboracle.so (plain C, -O2, no SIMD flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        p = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        lib.oracle_analyze.argtypes = [p, i32, i32, i32, i32, p, p, p, p, p, i64, p, p]
        lib.oracle_analyze.restype = ctypes.c_int
        lib.oracle_fill.argtypes = [i32, p, p, i64, p, i64, p, p, i64, p]
        lib.oracle_fill.restype = ctypes.c_int
        lib.oracle_filter.argtypes = [i32, p, p, i64, p, i32, i64, p, p, i64, p]
        lib.oracle_filter.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def capacity(w, h):
    """Upper bound on the number of nodes of a w x h image: foreground
    components (at most one per 2x2 block) + background components (at most
    one per pixel of a checkerboard colour) + the exterior."""
    return ((h + 1) // 2) * ((w + 1) // 2) + (w * h + 1) // 2 + 1


def analyze(img, w=None, conn=0, cap=None):
    """Label img ([h][pitch] uint8, nonzero = foreground, columns >= w ignored).

    Returns a dict with node [h][w], fg [h][w], bg [h][w], parent [N],
    feat [7][N], node_fg [N] (uint8), counts [4] and n (= N).
    """
    lib = _load()
    img = np.ascontiguousarray(img, dtype=np.uint8)
    h, pitch = img.shape
    w = pitch if w is None else int(w)
    if cap is None:
        cap = capacity(w, h)
    node = np.empty((h, w), np.int32)
    fg = np.empty((h, w), np.int32)
    bg = np.empty((h, w), np.int32)
    parent = np.empty(cap, np.int32)
    feat = np.empty((NF, cap), np.int64)
    node_fg = np.zeros(cap, np.uint8)
    counts = np.zeros(4, np.int32)
    rc = lib.oracle_analyze(_ptr(img), w, h, pitch, conn, _ptr(node), _ptr(fg), _ptr(bg),
                            _ptr(parent), _ptr(feat), cap, _ptr(node_fg), _ptr(counts))
    if rc != 0:
        raise RuntimeError("oracle_analyze failed with status %d" % rc)
    n = int(counts[0])
    return dict(node=node, fg=fg, bg=bg, parent=parent[:n].copy(), feat=feat[:, :n].copy(),
                node_fg=node_fg[:n].copy(), counts=counts, n=n, w=w, h=h)


def fill(res, T, target_fg=0):
    """Area filter on an analyze() result: target_fg = 0 fills holes with
    area <= T, target_fg = 1 removes foreground objects with area <= T.

    Returns (map [N], filtered_feat [7][N], filtered_parent [N])."""
    lib = _load()
    n = res["n"]
    parent = np.ascontiguousarray(res["parent"], np.int32)
    feat = np.ascontiguousarray(res["feat"], np.int64)
    node_fg = np.ascontiguousarray(res["node_fg"], np.uint8)
    fmap = np.empty(n, np.int32)
    ffeat = np.empty((NF, n), np.int64)
    fpar = np.empty(n, np.int32)
    rc = lib.oracle_filter(n, _ptr(parent), _ptr(feat), n, _ptr(node_fg), int(target_fg), int(T), _ptr(fmap),
                           _ptr(ffeat), n, _ptr(fpar))
    if rc != 0:
        raise RuntimeError("oracle_filter failed with status %d" % rc)
    return fmap, ffeat, fpar


def relabel(res, fmap):
    """Label images after filtering: every pixel takes the survivor of its
    node, in the label image of the survivor's colour (-1 in the other)."""
    s = fmap[res["node"]]
    col = res["node_fg"][s].astype(bool)
    return np.where(col, s, -1).astype(np.int32), np.where(col, -1, s).astype(np.int32)


def euler(res):
    """Euler number with 8-foreground / 4-background: foreground components
    minus holes (every background component other than the exterior)."""
    return int(res["counts"][1]) - (int(res["counts"][2]) - 1)
