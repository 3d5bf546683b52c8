"""Autotuner for the tile shape and merge schedule of the CUDA path.

Three launch choices change the speed but never the results:
  - the tile height, 32 or 16 rows (ccl_set_tile_rows): taller tiles have
    fewer tile edges to merge across, shorter tiles let more CTAs share an
    SM and hide more latency;
  - the tile width, 1024 or 512 columns (ccl_set_tile_cols): narrower tiles
    give small or narrow images more tiles to spread over the SMs, wider
    tiles fewer vertical tile edges;
  - the merge schedule, 1, 2, 4 or 8 work items per 32-pixel word of a
    boundary between bands of tiles (ccl_set_merge_split): more items spread
    a dense boundary's unions over more threads, fewer cost less on sparse
    boundaries.
Which wins depends on the images, so the tuner times the caller's own work
with CUDA events: first every tile shape (height x width) at the default
merge schedule, then every merge schedule at the best shape, and keeps the
fastest choice per size class in a small JSON cache.
"""
import json
import os

TILE_ROWS = (32, 16)
TILE_COLS = (1024, 512)
MERGE_SPLITS = (4, 1, 2, 8)      # the first is the default


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
                                                         "tile_shape.json"))


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


def choice_name(rows, cols, split):
    return "rows%d_cols%d_split%d" % (rows, cols, split)


def apply(ctx, choice):
    ctx.set_tile_rows(choice["rows"])
    if hasattr(ctx, "set_tile_cols"):
        ctx.set_tile_cols(choice["cols"])
    if hasattr(ctx, "set_merge_split"):
        ctx.set_merge_split(choice["merge_split"])


def tune(ctx, run, key, cache_path=None, reps=5, warmup=2, timer=None, force=False):
    """Pick the tile shape and merge schedule for `run` (a callable that
    enqueues the work to tune, e.g. one batched analysis) on context `ctx`,
    set them on ctx and return (choice, {choice_name: ms}) where choice =
    {"rows", "cols", "merge_split"}.

    timer(fn, reps) -> ms per call; defaults to CUDA events on the current
    stream. A cached choice for `key` is reused unless force is set."""
    path = cache_path or default_cache_path()
    data = _load(path)
    if not force and key in data and "merge_split" in data[key] and "cols" in data[key]:
        choice = {k: int(data[key][k]) for k in ("rows", "cols", "merge_split")}
        apply(ctx, choice)
        return choice, data[key].get("ms", {})
    if timer is None:
        timer = cuda_timer
    times = {}

    def measure(rows, cols, split):
        name = choice_name(rows, cols, split)
        if name not in times:
            apply(ctx, {"rows": rows, "cols": cols, "merge_split": split})
            for _ in range(warmup):
                run()
            times[name] = timer(run, reps)
        return times[name]

    split0 = MERGE_SPLITS[0]
    cols_choices = TILE_COLS if hasattr(ctx, "set_tile_cols") else TILE_COLS[:1]
    shapes = [(r, c) for c in cols_choices for r in TILE_ROWS]
    best_rows, best_cols = min(shapes, key=lambda rc: measure(rc[0], rc[1], split0))
    splits = MERGE_SPLITS if hasattr(ctx, "set_merge_split") else MERGE_SPLITS[:1]
    best_split = min(splits, key=lambda sp: measure(best_rows, best_cols, sp))
    choice = {"rows": best_rows, "cols": best_cols, "merge_split": best_split}
    apply(ctx, choice)
    data[key] = dict(choice, ms={k: round(v, 4) for k, v in times.items()})
    _store(path, data)
    return choice, times


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
