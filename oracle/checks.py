"""Independent properties used to pin the oracle.

TEST INFRASTRUCTURE ONLY. Nothing here reuses the oracle's traversal:
  euler_bitquad    Gray's bit-quad count over the zero-padded image (the
                   Euler-number method the paper cites as prior art).
  surrounds        the surround relation of Section 3.1 tested directly: a
                   barrier search from C that may not step on P must not
                   reach the image border.
  brute_fill       hole filling done on pixels: holes up to the threshold
                   are painted foreground and the image is labelled again.
"""
from collections import deque

import numpy as np


def euler_bitquad(img01, conn=0):
    """Euler number by bit-quads over the image padded with one background
    pixel on every side. With 8-foreground adjacency:
    E = (n(Q1) - n(Q3) - 2 n(QD)) / 4; with 4-foreground adjacency the
    diagonal term changes sign."""
    a = np.pad(np.asarray(img01, dtype=np.int64) != 0, 1).astype(np.int64)
    tl, tr, bl, br = a[:-1, :-1], a[:-1, 1:], a[1:, :-1], a[1:, 1:]
    s = tl + tr + bl + br
    q1 = int((s == 1).sum())
    q3 = int((s == 3).sum())
    qd = int(((s == 2) & (tl == br)).sum())
    num = q1 - q3 - 2 * qd if conn == 0 else q1 - q3 + 2 * qd
    assert num % 4 == 0
    return num // 4


def surrounds(node, colour_of, c, p, conn=0):
    """True if every path from component c to the outside of the image meets
    component p. Paths use the adjacency dual to p's: 4-paths when p is an
    8-connected colour, 8-paths when p is 4-connected."""
    node = np.asarray(node)
    h, w = node.shape
    p_is_fg = bool(colour_of[p])
    p_eight = p_is_fg if conn == 0 else (not p_is_fg)
    path_eight = not p_eight
    seen = np.zeros((h, w), bool)
    q = deque()
    ys, xs = np.nonzero(node == c)
    for y, x in zip(ys.tolist(), xs.tolist()):
        seen[y, x] = True
        q.append((y, x))
    while q:
        y, x = q.popleft()
        if y == 0 or x == 0 or y == h - 1 or x == w - 1:
            return False
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dy == 0 and dx == 0) or (not path_eight and dy != 0 and dx != 0):
                    continue
                ny, nx = y + dy, x + dx
                if not seen[ny, nx] and node[ny, nx] != p:
                    seen[ny, nx] = True
                    q.append((ny, nx))
    return True


def brute_fill_image(img01, node, colour_of, area, T):
    """Paint every hole (background node other than 0 with area <= T)
    foreground; return the new 0/1 image."""
    img = (np.asarray(img01) != 0).astype(np.uint8)
    node = np.asarray(node)
    if T < 0:
        return img
    holes = [k for k in range(1, len(colour_of)) if not colour_of[k] and area[k] <= T]
    if holes:
        mask = np.isin(node, np.asarray(holes))
        img[mask] = 1
    return img


def brute_remove_objects(img01, node, colour_of, area, T):
    """Paint every foreground node with area <= T background; return the new
    0/1 image."""
    img = (np.asarray(img01) != 0).astype(np.uint8)
    node = np.asarray(node)
    if T < 0:
        return img
    objs = [k for k in range(1, len(colour_of)) if colour_of[k] and area[k] <= T]
    if objs:
        img[np.isin(node, np.asarray(objs))] = 0
    return img
