"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws images; it holds none of the labelling arithmetic.
Both the CUDA path's tests and the oracle's tests take their images from here.
All images are uint8 arrays of 0/1 (foreground = 1) unless noted.

Recipes (the paper measures on random images of varying density and
granularity, Section 4; the exact generator is not given):
  bernoulli(h, w, d, seed)    i.i.d. pixels, foreground with probability d.
  granular(h, w, d, g, seed)  a ceil(h/g) x ceil(w/g) grid of Bernoulli(d)
                              blocks anchored at (0, 0), each block g x g
                              pixels, cropped to h x w.
  rings(h, w, seed)           5% salt noise, then 2000 sets of concentric rings
                              (1-12 rings, outer radius 4-400, thickness 1-3,
                              spacing >= thickness + 2) OR'd in; gives deep
                              inclusion trees.
  paper_sweep_image(i_d, i_g, k)
                              2048 x 2048 granular images on the Section 4
                              grid: d in {0, 0.05, .., 1} x g in {1..16}.
  uneven_batch(seed, n)       n images with sides drawn log-uniform in
                              [64, 2048], density U(0.2, 0.8), granularity
                              U{1..8}, row pitch rounded up to 128 bytes with
                              0xA5 in the padding.
  blob_frame(h, w, seed)      filled random ellipses (semi-axes 5-200, any
                              rotation), each with 0-3 elliptical background
                              holes, added until the foreground density reaches
                              a target drawn from U(0.3, 0.6).
"""
import math

import numpy as np

SWEEP_DENSITIES = (0.1, 0.3, 0.5, 0.7, 0.9)
SWEEP_GRANULARITIES = (1, 2, 4, 8, 16)
FRAME_SIZES = ((480, 640), (1080, 1920), (2160, 3840))


def bernoulli(h, w, d, seed):
    rng = np.random.default_rng(seed)
    return (rng.random((h, w)) < d).astype(np.uint8)


def granular(h, w, d, g, seed):
    rng = np.random.default_rng(seed)
    bh, bw = -(-h // g), -(-w // g)
    blocks = (rng.random((bh, bw)) < d).astype(np.uint8)
    return np.ascontiguousarray(np.repeat(np.repeat(blocks, g, axis=0), g, axis=1)[:h, :w])


def sweep_seed(i_d, i_g):
    return 2000 + 10 * i_d + i_g


def sweep_image(i_d, i_g, h=4096, w=4096):
    """One image of the density x granularity sweep."""
    return granular(h, w, SWEEP_DENSITIES[i_d], SWEEP_GRANULARITIES[i_g], sweep_seed(i_d, i_g))


PAPER_DENSITIES = tuple(round(0.05 * i, 2) for i in range(21))
PAPER_GRANULARITIES = tuple(range(1, 17))


def paper_sweep_image(i_d, i_g, k=0, side=2048):
    """Image k of cell (density i_d, granularity i_g) of the Section 4 protocol:
    side x side random images, densities 0..1 in steps of 0.05, granularities
    1..16 (the paper sweeps the same two parameters on 2048 x 2048 images)."""
    seed = 30000 + 1000 * k + 32 * i_d + i_g
    return granular(side, side, PAPER_DENSITIES[i_d], PAPER_GRANULARITIES[i_g], seed)


def rings(h=8192, w=8192, seed=3, n_sets=2000, salt=0.05):
    rng = np.random.default_rng(seed)
    img = (rng.random((h, w)) < salt).astype(np.uint8)
    for _ in range(n_sets):
        cy = int(rng.integers(0, h))
        cx = int(rng.integers(0, w))
        n = int(rng.integers(1, 13))
        outer = int(rng.integers(4, 401))
        step = max(5, outer // n)
        radii = []
        r = outer
        while len(radii) < n and r >= 4:
            t = int(rng.integers(1, min(3, step - 2) + 1))
            radii.append((r, t))
            r -= step
        y0, y1 = max(0, cy - outer), min(h, cy + outer + 1)
        x0, x1 = max(0, cx - outer), min(w, cx + outer + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        dy = (np.arange(y0, y1, dtype=np.int64) - cy)[:, None]
        dx = (np.arange(x0, x1, dtype=np.int64) - cx)[None, :]
        d2 = dy * dy + dx * dx
        on = np.zeros(d2.shape, bool)
        for r, t in radii:
            on |= ((r - t) * (r - t) < d2) & (d2 <= r * r)
        img[y0:y1, x0:x1] |= on.astype(np.uint8)
    return img


def pitched(img, pitch, pad_value=0xA5):
    """Copy img ([h][w]) into a [h][pitch] buffer whose padding holds pad_value."""
    h, w = img.shape
    out = np.full((h, pitch), pad_value, np.uint8)
    out[:, :w] = img
    return out


def uneven_batch(seed=4, n=256, lo=64, hi=2048, pitch_align=128):
    """Returns a list of (padded image [h][pitch], w)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        w = int(math.floor(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        h = int(math.floor(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        d = float(rng.uniform(0.2, 0.8))
        g = int(rng.integers(1, 9))
        img = granular(h, w, d, g, int(rng.integers(0, 2**31)))
        pitch = -(-w // pitch_align) * pitch_align
        out.append((pitched(img, pitch), w))
    return out


def _ellipse_mask(h, w, cy, cx, a, b, theta):
    """Pixels inside the ellipse with semi-axes a, b rotated by theta."""
    r = int(math.ceil(max(a, b))) + 1
    y0, y1 = max(0, int(cy) - r), min(h, int(cy) + r + 1)
    x0, x1 = max(0, int(cx) - r), min(w, int(cx) + r + 1)
    if y0 >= y1 or x0 >= x1:
        return None
    yy = (np.arange(y0, y1, dtype=np.float64) - cy)[:, None]
    xx = (np.arange(x0, x1, dtype=np.float64) - cx)[None, :]
    c, s = math.cos(theta), math.sin(theta)
    u = xx * c + yy * s
    v = -xx * s + yy * c
    return (y0, y1, x0, x1, (u * u) / (a * a) + (v * v) / (b * b) <= 1.0)


def blob_frame(h, w, seed):
    rng = np.random.default_rng(seed)
    target = float(rng.uniform(0.3, 0.6))
    img = np.zeros((h, w), np.uint8)
    fg = 0
    tries = 0
    while fg < target * h * w and tries < 100000:
        tries += 1
        cy, cx = rng.uniform(0, h), rng.uniform(0, w)
        a, b = rng.uniform(5, 200), rng.uniform(5, 200)
        th = rng.uniform(0, math.pi)
        m = _ellipse_mask(h, w, cy, cx, a, b, th)
        if m is None:
            continue
        y0, y1, x0, x1, inside = m
        patch = img[y0:y1, x0:x1]
        fg -= int(patch.sum())
        patch[inside] = 1
        for _ in range(int(rng.integers(0, 4))):
            ha, hb = a * rng.uniform(0.1, 0.5), b * rng.uniform(0.1, 0.5)
            hy = cy + rng.uniform(-0.4, 0.4) * a
            hx = cx + rng.uniform(-0.4, 0.4) * b
            hm = _ellipse_mask(h, w, hy, hx, max(ha, 1.5), max(hb, 1.5), rng.uniform(0, math.pi))
            if hm is None:
                continue
            hy0, hy1, hx0, hx1, hin = hm
            img[hy0:hy1, hx0:hx1][hin] = 0
        fg += int(img[y0:y1, x0:x1].sum())
    return img


def frame_stream(seed=5, n=64):
    """n frames with sizes drawn uniformly from FRAME_SIZES."""
    rng = np.random.default_rng(seed)
    frames = []
    for _ in range(n):
        h, w = FRAME_SIZES[int(rng.integers(0, len(FRAME_SIZES)))]
        frames.append(blob_frame(h, w, int(rng.integers(0, 2**31))))
    return frames


def adversarial(h, w, kind, seed=0):
    """Structured images that stress connectivity across tiles."""
    yy, xx = np.mgrid[0:h, 0:w]
    if kind == "zeros":
        return np.zeros((h, w), np.uint8)
    if kind == "ones":
        return np.ones((h, w), np.uint8)
    if kind == "checker0":
        return ((yy + xx) % 2 == 0).astype(np.uint8)
    if kind == "checker1":
        return ((yy + xx) % 2 == 1).astype(np.uint8)
    if kind == "vstripes":
        return (xx % 2 == 0).astype(np.uint8)
    if kind == "hstripes":
        return (yy % 2 == 0).astype(np.uint8)
    if kind == "diag":
        # 1-pixel diagonal lines: 8-connected foreground, background cut 4-wise
        return ((xx - yy) % 7 == 0).astype(np.uint8)
    if kind == "antidiag":
        return ((xx + yy) % 5 == 0).astype(np.uint8)
    if kind == "spiral":
        img = np.zeros((h, w), np.uint8)
        top, left, bottom, right = 0, 0, h - 1, w - 1
        while top <= bottom and left <= right:
            img[top, left:right + 1] = 1
            img[top:bottom + 1, right] = 1
            if bottom > top:
                img[bottom, left:right + 1] = 1
            if right > left + 2:
                img[top + 2:bottom + 1, left] = 1
            top += 2
            left += 2
            bottom -= 2
            right -= 2
        return img
    if kind == "rings":
        img = np.zeros((h, w), np.uint8)
        c = min(h, w) // 2
        for k in range(0, c, 3):
            img[k, k:w - k] = 1
            img[h - 1 - k, k:w - k] = 1
            img[k:h - k, k] = 1
            img[k:h - k, w - 1 - k] = 1
        return img
    if kind == "comb":
        img = np.zeros((h, w), np.uint8)
        img[:, ::2] = 1
        img[h - 1, :] = 1
        return img
    raise ValueError(kind)


ADVERSARIAL_KINDS = ("zeros", "ones", "checker0", "checker1", "vstripes", "hstripes",
                     "diag", "antidiag", "spiral", "rings", "comb")
