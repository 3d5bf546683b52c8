"""The paper's own method, restated step by step: LSL B&W.

TEST INFRASTRUCTURE ONLY. This is written from the paper's description of
  Algorithm 1  segment detection (step 1a),
  Algorithm 2  B&W unification (step 1b), with the initial adjacency table I,
  Algorithm 3  B&W transitive closure (step 2), with optional hole filling,
  Algorithm 4  B&W relabeling (step 3),
and is used only to pin the flood-fill oracle to the paper: on small images
both must give the same partition, the same tree and the same features.

Readings where the paper is silent or its boxes leave a case open:
  - Row -1 is a virtual background row whose only run carries label 0, the
    exterior (the worked example labels the background pixels of row 0 with
    0).
  - Row h is a virtual background row with no features: the printed epilog
    links to 0 only the first run and the last background run of each row, so
    a background run touching only the bottom border would otherwise be
    taken for a hole; the paper defines surrounding through paths to the
    exterior of the image, and the virtual row supplies that link.
  - A new label created for the first run of a row (er = 0) records I = 0.
  - Node 0 keeps I[0] = -1 through the closure.
  - Pixels are foreground when nonzero.
Labels are then renumbered densely by increasing final root, which is the
raster order of each component's first pixel.
"""

INT64_MAX = (1 << 63) - 1
EMPTY = (0, INT64_MAX, INT64_MAX, -1, -1, 0, 0)  # S, xmin, ymin, xmax, ymax, Sx, Sy


def segments(line):
    """Algorithm 1: relative label per pixel (ER), run bounds (RLC), run count.
    Run er covers [RLC[er], RLC[er+1]); even runs are background, odd runs
    foreground; run 0 is background and may be empty."""
    w = len(line)
    rlc = [0] * (w + 2)
    er_tab = [0] * w
    er = 0
    prev = 0
    for j in range(w):
        cur = 1 if line[j] else 0
        rlc[er + 1] = j
        er += cur ^ prev
        er_tab[j] = er
        prev = cur
    rlc[er + 1] = w
    return er_tab, rlc[: er + 2], er + 1


def run_features(i, j0, j1):
    """Features of the run [j0, j1) on row i (x = column, y = row, box inclusive)."""
    if j1 <= j0:
        return EMPTY
    n = j1 - j0
    return (n, j0, i, j1 - 1, i, (j0 + j1 - 1) * n // 2, i * n)


def merge(a, b):
    return (a[0] + b[0], min(a[1], b[1]), min(a[2], b[2]), max(a[3], b[3]),
            max(a[4], b[4]), a[5] + b[5], a[6] + b[6])


def analyze(rows, conn=0, fill=False):
    """Run LSL B&W on rows (h x w, nonzero = foreground).

    Returns (label image [h][w] of canonical ids, parent list, feature list,
    number of nodes). With fill=True the hole-filling branch of Algorithm 3 is
    taken, and the returned partition is the filled one."""
    h = len(rows)
    w = len(rows[0])
    T = [0]
    F = [EMPTY]
    I = [-1]

    def find(e):
        while T[e] != e:
            e = T[e]
        return e

    er_prev = [0] * w
    era_prev = [0]
    era_rows = []
    rlc_rows = []
    for i in range(h + 1):
        line = rows[i] if i < h else [0] * w
        er_cur, rlc, ner = segments(line)
        era = [0] * ner
        ers = 0
        if rlc[1] == 0:  # empty first background run
            era[0] = 0
            ers = 1
        for er in range(ers, ner):
            j0, j1 = rlc[er], rlc[er + 1]
            p = er % 2
            c8 = p if conn == 0 else p ^ 1
            f = run_features(i, j0, j1) if i < h else EMPTY
            j0 = max(j0 - c8, 0)
            j1 = min(j1 + c8, w)
            er0 = er_prev[j0]
            er1 = er_prev[j1 - 1]
            er0 += (er0 % 2) ^ p
            er1 -= (er1 % 2) ^ p
            if er1 >= er0:
                a = find(era_prev[er0])
                for erk in range(er0 + 2, er1 + 1, 2):
                    ak = find(era_prev[erk])
                    if a < ak:
                        T[ak] = a
                    if a > ak:
                        T[a] = ak
                        a = ak
                era[er] = a
                F[a] = merge(F[a], f)
            else:
                ne = len(T)
                era[er] = ne
                T.append(ne)
                F.append(f)
                I.append(era[er - 1] if er >= 1 else 0)
        a = find(era[0])
        T[a] = 0
        if ner % 2 == 1:
            a = find(era[ner - 1])
            T[a] = 0
        er_prev, era_prev = er_cur, era
        if i < h:
            era_rows.append(era)
            rlc_rows.append((rlc, ner))

    # Algorithm 3: transitive closure, feature merge, adjacency to roots.
    ne = len(T)
    for e in range(ne):
        a = T[e]
        if fill and e == a and e != 0:
            s = I[e]
            if T[s] > 0:
                T[e] = s
                a = s
        if a < e:
            r = T[a]
            T[e] = r
            F[r] = merge(F[r], F[e])
        elif e != 0:
            I[e] = T[I[e]]

    roots = sorted({T[e] for e in range(ne)})
    ident = {r: k for k, r in enumerate(roots)}
    # Algorithm 4: relabel every run with its final root.
    label = [[0] * w for _ in range(h)]
    for i in range(h):
        rlc, ner = rlc_rows[i]
        for er in range(ner):
            r = T[era_rows[i][er]]
            for j in range(rlc[er], rlc[er + 1]):
                label[i][j] = ident[r]
    parent = [-1] * len(roots)
    feats = [None] * len(roots)
    for r in roots:
        k = ident[r]
        feats[k] = F[r]
        if r != 0:
            parent[k] = ident[I[r]]
    return label, parent, feats, len(roots)
