"""Python binding of libccl.so (include/ccl.h), argument marshalling only.

Every step of the analysis runs in the library's CUDA kernels; this module
allocates output tensors with PyTorch, passes raw device pointers and the
current CUDA stream through ctypes, and turns status codes into exceptions.
Importing it raises ImportError when the library has not been built; there is
no fallback implementation.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libccl.so")
if not os.path.exists(LIB_PATH):
    raise ImportError("libccl.so is not built; run paper_2006_09299_gb300.build.build() "
                      "(or __graft_entry__.build()) first")
_lib = ctypes.CDLL(LIB_PATH)

OK, ERR_ARG, ERR_ALIGN, ERR_CAPACITY, ERR_OOM, ERR_CUDA, ERR_ITER_LIMIT, ERR_STATE = 0, 1, 2, 4, 8, 16, 32, 64
F_AREA, F_XMIN, F_YMIN, F_XMAX, F_YMAX, F_SX, F_SY, F_COUNT = range(8)
CONN_8FG_4BG, CONN_4FG_8BG = 0, 1
TARGET_HOLES, TARGET_OBJECTS = 0, 1
INT64_MAX = (1 << 63) - 1

_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


class ImageDesc(ctypes.Structure):
    """Mirror of ccl_image_desc."""
    _fields_ = [("img", _p), ("w", _i32), ("h", _i32), ("pitch", _i32),
                ("fg_labels", _p), ("bg_labels", _p), ("tree_parent", _p), ("features", _p),
                ("counts", _p), ("capacity", _i64), ("fill_map", _p), ("filled_features", _p),
                ("filled_parent", _p)]


# name -> (restype, argtypes); the names are exactly the C ABI's
SIGNATURES = {
    "ccl_node_capacity": (_i64, [_i32, _i32]),
    "ccl_create": (ctypes.c_int, [ctypes.POINTER(_p), _i32, _i32, _i32]),
    "ccl_set_connectivity": (ctypes.c_int, [_p, _i32]),
    "ccl_analyze": (ctypes.c_int, [_p, _p, _p, _p, _p, _p, _p, _p]),
    "ccl_fill_holes": (ctypes.c_int, [_p, _i64, _p, _p, _p, _p]),
    "ccl_filter_components": (ctypes.c_int, [_p, _i32, _i64, _p, _p, _p, _p]),
    "ccl_relabel_filtered": (ctypes.c_int, [_p, _p, _p, _p]),
    "ccl_get_euler": (ctypes.c_int, [_p, ctypes.POINTER(_i64)]),
    "ccl_filter_components_batched": (ctypes.c_int, [_p, _i32, _i64, _p]),
    "ccl_relabel_filtered_batched": (ctypes.c_int, [_p, _p, _p, _p]),
    "ccl_get_counts": (ctypes.c_int, [_p, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "ccl_create_batched": (ctypes.c_int, [ctypes.POINTER(_p), _i32, _i64, _i32]),
    "ccl_analyze_batched": (ctypes.c_int, [_p, ctypes.POINTER(ImageDesc), _i32, _p]),
    "ccl_analyze_batched_from_host": (ctypes.c_int, [_p, ctypes.POINTER(ImageDesc), ctypes.POINTER(_p),
                                                     ctypes.POINTER(_i64), _i32, _p]),
    "ccl_fill_holes_batched": (ctypes.c_int, [_p, _i64, _p]),
    "ccl_set_graph_cache": (ctypes.c_int, [_p, _i32]),
    "ccl_set_tile_rows": (ctypes.c_int, [_p, _i32]),
    "ccl_set_merge_split": (ctypes.c_int, [_p, _i32]),
    "ccl_set_tile_cols": (ctypes.c_int, [_p, _i32]),
    "ccl_enable_phase_timing": (ctypes.c_int, [_p, _i32]),
    "ccl_read_phase_timing": (ctypes.c_int, [_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64)]),
    "ccl_get_launch_count": (ctypes.c_int, [_p, ctypes.POINTER(_i64)]),
    "ccl_analyze_static": (ctypes.c_int, [_p, _i32, _i32, _i32, _p, _p, _p, _p, _i64, _p, _p]),
    "ccl_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ccl_destroy": (None, [_p]),
}
for _name, (_res, _args) in SIGNATURES.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class CCLError(RuntimeError):
    def __init__(self, status, what):
        self.status = int(status)
        super().__init__("%s: %s (status %d)" % (what, status_string(status), self.status))


def status_string(status):
    return _lib.ccl_status_string(int(status)).decode()


def node_capacity(w, h):
    return int(_lib.ccl_node_capacity(int(w), int(h)))


def _check(status, what):
    if status != OK:
        raise CCLError(status, what)


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


PHASES = ("prologue", "label", "merge", "resolve", "scan", "canon", "write", "fill_map", "fill_merge")


class _Instrumented:
    """Phase timing and launch counting shared by both context kinds."""

    def enable_phase_timing(self, max_calls):
        _check(_lib.ccl_enable_phase_timing(self._h, int(max_calls)), "ccl_enable_phase_timing")

    def read_phase_timing(self):
        """{phase: (total_ms, launches)} of the recorded calls (waits)."""
        ms = (ctypes.c_double * len(PHASES))()
        cnt = (_i64 * len(PHASES))()
        _check(_lib.ccl_read_phase_timing(self._h, ms, cnt), "ccl_read_phase_timing")
        return {p: (ms[i], cnt[i]) for i, p in enumerate(PHASES)}

    def launch_count(self):
        n = _i64()
        _check(_lib.ccl_get_launch_count(self._h, ctypes.byref(n)), "ccl_get_launch_count")
        return n.value

    def set_graph_cache(self, enable):
        _check(_lib.ccl_set_graph_cache(self._h, 1 if enable else 0), "ccl_set_graph_cache")

    def set_tile_rows(self, rows):
        _check(_lib.ccl_set_tile_rows(self._h, int(rows)), "ccl_set_tile_rows")
        self.tile_rows = int(rows)

    def set_tile_cols(self, cols):
        _check(_lib.ccl_set_tile_cols(self._h, int(cols)), "ccl_set_tile_cols")
        self.tile_cols = int(cols)

    def set_merge_split(self, items_per_word):
        _check(_lib.ccl_set_merge_split(self._h, int(items_per_word)), "ccl_set_merge_split")
        self.merge_split = int(items_per_word)


class Analysis:
    """Outputs of one analysed image (device tensors). Node arrays have the
    full capacity; `n` (which waits for the stream) gives the node count."""

    def __init__(self, w, h, cap, labels, device):
        self.w, self.h, self.cap = w, h, cap
        self.fg = torch.empty((h, w), dtype=torch.int32, device=device) if labels else None
        self.bg = torch.empty((h, w), dtype=torch.int32, device=device) if labels else None
        self.parent = torch.empty(cap, dtype=torch.int32, device=device)
        self.features = torch.empty((F_COUNT, cap), dtype=torch.int64, device=device)
        self.counts = torch.zeros(4, dtype=torch.int32, device=device)
        self.fill_map = self.filled_features = self.filled_parent = None

    def alloc_fill(self):
        dev = self.parent.device
        self.fill_map = torch.empty(self.cap, dtype=torch.int32, device=dev)
        self.filled_features = torch.empty((F_COUNT, self.cap), dtype=torch.int64, device=dev)
        self.filled_parent = torch.empty(self.cap, dtype=torch.int32, device=dev)
        return self

    @property
    def n(self):
        return int(self.counts[0].item())

    def status(self):
        return int(self.counts[3].item())


class Context(_Instrumented):
    """ccl_create / ccl_analyze / ccl_fill_holes for images of one shape."""

    def __init__(self, w, h, pitch=None, conn=CONN_8FG_4BG):
        self.w, self.h = int(w), int(h)
        self.pitch = int(pitch if pitch is not None else -(-self.w // 16) * 16)
        self._h = _p()
        _check(_lib.ccl_create(ctypes.byref(self._h), self.w, self.h, self.pitch), "ccl_create")
        self.cap = node_capacity(self.w, self.h)
        if conn != CONN_8FG_4BG:
            self.set_connectivity(conn)
        self.last = None

    def set_connectivity(self, conn):
        _check(_lib.ccl_set_connectivity(self._h, int(conn)), "ccl_set_connectivity")

    def new_outputs(self, labels=True, device="cuda"):
        return Analysis(self.w, self.h, self.cap, labels, device)

    def analyze(self, img, out=None, labels=True, stream=None):
        """img: uint8 CUDA tensor [h][pitch] (nonzero = foreground)."""
        if out is None:
            out = self.new_outputs(labels, img.device)
        _check(_lib.ccl_analyze(self._h, _ptr(img), _ptr(out.fg), _ptr(out.bg), _ptr(out.parent),
                                _ptr(out.features), _ptr(out.counts), _stream(stream)), "ccl_analyze")
        self.last = out
        return out

    def fill_holes(self, area_threshold, out=None, stream=None):
        """Hole filling on the node tables of the last analyze."""
        if out is None:
            out = self.last.alloc_fill() if self.last.fill_map is None else self.last
        _check(_lib.ccl_fill_holes(self._h, int(area_threshold), _ptr(out.fill_map),
                                   _ptr(out.filled_features), _ptr(out.filled_parent), _stream(stream)),
               "ccl_fill_holes")
        return out

    def filter_components(self, target, area_threshold, out=None, stream=None):
        """Area filter on the last analyze (TARGET_HOLES or TARGET_OBJECTS)."""
        if out is None:
            out = self.last.alloc_fill() if self.last.fill_map is None else self.last
        _check(_lib.ccl_filter_components(self._h, int(target), int(area_threshold), _ptr(out.fill_map),
                                          _ptr(out.filled_features), _ptr(out.filled_parent), _stream(stream)),
               "ccl_filter_components")
        return out

    def relabel_filtered(self, fg_out, bg_out, stream=None):
        """Label images through the map of the last fill / filter."""
        _check(_lib.ccl_relabel_filtered(self._h, _ptr(fg_out), _ptr(bg_out), _stream(stream)),
               "ccl_relabel_filtered")

    def euler(self):
        e = _i64()
        st = _lib.ccl_get_euler(self._h, ctypes.byref(e))
        if st not in (OK, ERR_CAPACITY):
            raise CCLError(st, "ccl_get_euler")
        return e.value

    def get_counts(self):
        n, nf, nb = _i32(), _i32(), _i32()
        st = _lib.ccl_get_counts(self._h, ctypes.byref(n), ctypes.byref(nf), ctypes.byref(nb))
        return n.value, nf.value, nb.value, int(st)

    def close(self):
        if self._h:
            _lib.ccl_destroy(self._h)
            self._h = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchContext(_Instrumented):
    """ccl_create_batched / ccl_analyze_batched / ccl_fill_holes_batched."""

    def __init__(self, max_images, max_total_pixels, max_side, conn=CONN_8FG_4BG, graph_cache=True):
        self._h = _p()
        _check(_lib.ccl_create_batched(ctypes.byref(self._h), int(max_images), int(max_total_pixels),
                                       int(max_side)), "ccl_create_batched")
        if conn != CONN_8FG_4BG:
            _check(_lib.ccl_set_connectivity(self._h, int(conn)), "ccl_set_connectivity")
        _check(_lib.ccl_set_graph_cache(self._h, 1 if graph_cache else 0), "ccl_set_graph_cache")

    def new_outputs(self, shapes, labels=True, fill=False, device="cuda"):
        outs = []
        for (w, h) in shapes:
            a = Analysis(w, h, node_capacity(w, h), labels, device)
            outs.append(a.alloc_fill() if fill else a)
        return outs

    def analyze(self, images, outs=None, labels=True, fill=False, stream=None):
        """images: list of (uint8 CUDA tensor [h][pitch], w)."""
        if outs is None:
            outs = self.new_outputs([(w, t.shape[0]) for t, w in images], labels, fill, images[0][0].device)
        descs = (ImageDesc * len(images))()
        for i, ((t, w), o) in enumerate(zip(images, outs)):
            descs[i] = self.image_desc(t, w, o)
        _check(_lib.ccl_analyze_batched(self._h, descs, len(images), _stream(stream)), "ccl_analyze_batched")
        return outs

    @staticmethod
    def image_desc(img, w, out):
        """The descriptor of one image of a batch (device image buffer img,
        uint8 [h][pitch], and its outputs); callers that reuse buffers keep it."""
        return ImageDesc(img.data_ptr(), int(w), int(img.shape[0]), int(img.stride(0)), _ptr(out.fg), _ptr(out.bg),
                         _ptr(out.parent), _ptr(out.features), _ptr(out.counts), out.cap, _ptr(out.fill_map),
                         _ptr(out.filled_features), _ptr(out.filled_parent))

    def analyze_from_host(self, descs, frames, pitches, stream=None):
        """descs: ImageDesc array (device buffers); frames: host addresses of
        the frames (ints), pitches: their row strides in bytes."""
        n = len(frames)
        fr = (_p * n)(*frames)
        pt = (_i64 * n)(*pitches)
        _check(_lib.ccl_analyze_batched_from_host(self._h, descs, fr, pt, n, _stream(stream)),
               "ccl_analyze_batched_from_host")

    def fill_holes(self, area_threshold, stream=None):
        _check(_lib.ccl_fill_holes_batched(self._h, int(area_threshold), _stream(stream)),
               "ccl_fill_holes_batched")

    def filter_components(self, target, area_threshold, stream=None):
        _check(_lib.ccl_filter_components_batched(self._h, int(target), int(area_threshold), _stream(stream)),
               "ccl_filter_components_batched")

    def relabel_filtered(self, fg_outs, bg_outs, stream=None):
        """Label images through the fill / filter map, one (fg, bg) pair of
        int32 tensors per image of the last batch (None skips an image)."""
        n = len(fg_outs)
        fa = (_p * n)(*[_ptr(t) for t in fg_outs])
        ba = (_p * n)(*[_ptr(t) for t in bg_outs])
        _check(_lib.ccl_relabel_filtered_batched(self._h, fa, ba, _stream(stream)), "ccl_relabel_filtered_batched")

    def close(self):
        if self._h:
            _lib.ccl_destroy(self._h)
            self._h = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


STATIC_MAX_PIXELS = 1 << 20
STATIC_MAX_SIDE = 4096


def analyze_static(img, w, out, stream=None):
    """ccl_analyze_static: one analysis without any device allocation by the
    library (scratch in a fixed per-device array; images up to
    STATIC_MAX_PIXELS pixels). `out` is an Analysis with preallocated
    tensors; img is a uint8 CUDA tensor [h][pitch]."""
    _check(_lib.ccl_analyze_static(_ptr(img), int(w), int(img.shape[0]), int(img.stride(0)), _ptr(out.fg),
                                   _ptr(out.bg), _ptr(out.parent), _ptr(out.features), int(out.cap),
                                   _ptr(out.counts), _stream(stream)), "ccl_analyze_static")
    return out
