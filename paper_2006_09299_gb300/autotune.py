"""Autotuner for the tile shape of the CUDA path.

The tile is 1024 columns wide (one 32-bit word per lane); its height is 32
or 16 rows (ccl_set_tile_rows). Taller tiles have fewer tile edges to merge
across; shorter tiles let more CTAs share an SM and hide more latency. Which
wins depends on the images, so the tuner times the caller's own work under
each height with CUDA events and keeps the fastest, per size class, in a
small JSON cache.
"""
import json
import os

TILE_ROWS = (32, 16)


def size_class(shapes, n_images=None):
    """Cache key: bucketed largest side, total pixels and image count."""
    max_side = max(max(w, h) for w, h in shapes)
    px = sum(w * h for w, h in shapes)
    n = len(shapes) if n_images is None else n_images

    def bucket(v):
        b = 1
        while b < v:
            b *= 2
        return b
    return "side%d_px%d_n%d" % (bucket(max_side), bucket(px), bucket(n))


def default_cache_path():
    return os.environ.get("CCL_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ccl_gb300",
                                                         "tile_rows.json"))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(ctx, run, key, cache_path=None, reps=5, warmup=2, timer=None, force=False):
    """Pick the tile height for `run` (a callable that enqueues the work to
    tune, e.g. one batched analysis) on context `ctx`, set it on ctx and
    return (rows, {rows: ms}).

    timer(fn, reps) -> ms per call; defaults to CUDA events on the current
    stream. A cached choice for `key` is reused unless force is set."""
    path = cache_path or default_cache_path()
    data = _load(path)
    if not force and key in data:
        rows = int(data[key]["tile_rows"])
        ctx.set_tile_rows(rows)
        return rows, data[key].get("ms", {})
    if timer is None:
        timer = cuda_timer
    times = {}
    for rows in TILE_ROWS:
        ctx.set_tile_rows(rows)
        for _ in range(warmup):
            run()
        times[rows] = timer(run, reps)
    best = min(times, key=times.get)
    ctx.set_tile_rows(best)
    data[key] = {"tile_rows": best, "ms": {str(k): round(v, 4) for k, v in times.items()}}
    _store(path, data)
    return best, times


def cuda_timer(fn, reps):
    import torch
    s = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(s)
    for _ in range(reps):
        fn()
    b.record(s)
    b.synchronize()
    return a.elapsed_time(b) / reps
