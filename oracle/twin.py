"""Second, independent statement of the oracle's definition, in pure Python.

TEST INFRASTRUCTURE ONLY. Where ccl_oracle.c floods components breadth first,
this module joins pixels with a union-find over the pixel grid plus one
virtual exterior node, then numbers the classes by their first pixel. It is
slow (pure Python loops) and meant for images of a few hundred pixels.

Definitions followed (the paper, Section 3.1 and Algorithms 2-3):
  - foreground pixels join through 8-adjacency and background pixels through
    4-adjacency (swapped when conn = 1);
  - background pixels on the image border belong to the exterior, node 0;
  - nodes other than 0 are numbered 1.. in raster order of their first pixel;
  - parent(C) = node of the pixel directly above the first pixel of C, or 0
    when that pixel lies on row 0;
  - features: area, inclusive bounding box, Sx = sum of x, Sy = sum of y.
"""

INT64_MAX = (1 << 63) - 1


def _find(par, a):
    while par[a] != a:
        par[a] = par[par[a]]
        a = par[a]
    return a


def _join(par, a, b):
    a = _find(par, a)
    b = _find(par, b)
    if a != b:
        if a < b:
            a, b = b, a
        par[a] = b


def analyze(rows, conn=0):
    """rows: list of lists (h x w) of ints, nonzero = foreground."""
    h = len(rows)
    w = len(rows[0])
    fgpx = [[1 if rows[y][x] else 0 for x in range(w)] for y in range(h)]
    ext = w * h  # virtual exterior node
    par = list(range(w * h + 1))
    fg8 = conn == 0
    bg8 = conn == 1
    for y in range(h):
        for x in range(w):
            c = fgpx[y][x]
            eight = fg8 if c else bg8
            nbrs = [(x - 1, y), (x, y - 1)]
            if eight:
                nbrs += [(x - 1, y - 1), (x + 1, y - 1)]
            for nx, ny in nbrs:
                if 0 <= nx < w and 0 <= ny < h and fgpx[ny][nx] == c:
                    _join(par, y * w + x, ny * w + nx)
            if not c and (x == 0 or y == 0 or x == w - 1 or y == h - 1):
                _join(par, y * w + x, ext)
    root_ext = _find(par, ext)
    ident = {root_ext: 0}
    first = {0: None}
    node = [[0] * w for _ in range(h)]
    for y in range(h):
        for x in range(w):
            r = _find(par, y * w + x)
            if r not in ident:
                ident[r] = len(ident)
                first[ident[r]] = (x, y)
            node[y][x] = ident[r]
    n = len(ident)
    feat = [[0, INT64_MAX, INT64_MAX, -1, -1, 0, 0] for _ in range(n)]
    colour = [0] * n
    for y in range(h):
        for x in range(w):
            f = feat[node[y][x]]
            f[0] += 1
            f[1] = min(f[1], x)
            f[2] = min(f[2], y)
            f[3] = max(f[3], x)
            f[4] = max(f[4], y)
            f[5] += x
            f[6] += y
            colour[node[y][x]] = fgpx[y][x]
    parent = [-1] * n
    for k in range(1, n):
        x, y = first[k]
        parent[k] = 0 if y == 0 else node[y - 1][x]
    fg = [[node[y][x] if fgpx[y][x] else -1 for x in range(w)] for y in range(h)]
    bg = [[-1 if fgpx[y][x] else node[y][x] for x in range(w)] for y in range(h)]
    n_fg = sum(colour[1:])
    return dict(node=node, fg=fg, bg=bg, parent=parent, feat=feat, colour=colour,
                first=first, n=n, counts=[n, n_fg, n - n_fg, 0])


def fill(res, T, target_fg=0):
    """Area filter, stated as: a node is absorbed when it is a target (colour
    target_fg, not node 0, area <= T: a hole when target_fg = 0, an object
    when 1) or a child of a target; every node maps to its nearest
    ancestor-or-self that is not absorbed. Returns (map, features, parent)."""
    n = res["n"]
    parent = res["parent"]
    colour = res["colour"]
    feat = res["feat"]

    def is_target(k):
        return T >= 0 and k != 0 and colour[k] == target_fg and feat[k][0] <= T

    absorbed = [is_target(k) or (k != 0 and colour[k] != target_fg and is_target(parent[k])) for k in range(n)]
    fmap = []
    for k in range(n):
        s = k
        while absorbed[s]:
            s = parent[s]
        fmap.append(s)
    ff = [[0, INT64_MAX, INT64_MAX, -1, -1, 0, 0] for _ in range(n)]
    for k in range(n):
        s = fmap[k]
        a, b = ff[s], feat[k]
        a[0] += b[0]
        a[1] = min(a[1], b[1])
        a[2] = min(a[2], b[2])
        a[3] = max(a[3], b[3])
        a[4] = max(a[4], b[4])
        a[5] += b[5]
        a[6] += b[6]
    fpar = [(-1 if (fmap[k] != k or parent[k] < 0) else fmap[parent[k]]) for k in range(n)]
    return fmap, ff, fpar
