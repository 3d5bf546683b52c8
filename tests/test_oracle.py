"""Pins for the CPU oracle: the oracle is checked against things other than
itself (the paper's worked example, the paper's own algorithm restated,
brute force, closed forms, an independent library labeller, the Euler number
by bit-quads and the surround relation tested directly)."""
import itertools

import numpy as np
import pytest

from oracle import checks, paper_lsl, twin
from oracle import reference as orc
from paper_2006_09299_gb300 import inputs

INT64_MAX = np.iinfo(np.int64).max


def grid(lines):
    return np.array([[1 if c == "#" else 0 for c in row] for row in lines], np.uint8)


def first_pixels(node):
    """Raster index of the first pixel of every node present in the grid."""
    flat = np.asarray(node).ravel()
    ids, idx = np.unique(flat, return_index=True)
    return dict(zip(ids.tolist(), idx.tolist()))


def assert_same_as_twin(res, tw):
    assert res["n"] == tw["n"]
    np.testing.assert_array_equal(res["node"], np.array(tw["node"]))
    np.testing.assert_array_equal(res["fg"], np.array(tw["fg"]))
    np.testing.assert_array_equal(res["bg"], np.array(tw["bg"]))
    np.testing.assert_array_equal(res["parent"], np.array(tw["parent"]))
    np.testing.assert_array_equal(res["feat"].T, np.array(tw["feat"], dtype=np.int64))
    np.testing.assert_array_equal(res["node_fg"], np.array(tw["colour"], np.uint8))
    assert list(res["counts"]) == tw["counts"]


# ---------------------------------------------------------------- Figure 3


def test_fig3_nodes_tree_features(fig3):
    img = grid(fig3["grid"])
    res = orc.analyze(img)
    rows = [r.split() for r in fig3["nodes"]]
    assert res["n"] == len(rows)
    for r in rows:
        n = int(r[0])
        assert res["node_fg"][n] == (r[1] == "fg")
        assert list(res["feat"][:, n]) == [int(v) for v in r[2:9]]
        assert res["parent"][n] == int(r[9])
    assert orc.euler(res) == fig3["euler"]
    assert checks.euler_bitquad(img) == fig3["euler"]


def test_fig3_paper_labels_and_classes(fig3):
    """The figure's provisional labels fall into the narrated classes, and
    the narrated surroundings are the tree edges."""
    img = grid(fig3["grid"])
    res = orc.analyze(img)
    where = {}
    for line in fig3["labels"]:
        lab, x, y = map(int, line.split())
        where.setdefault(lab, []).append(res["node"][y, x])
    node_of = {lab: v[0] for lab, v in where.items()}
    for lab, v in where.items():
        assert len(set(v)) == 1
    classes = [list(map(int, c.split())) for c in fig3["classes"]]
    seen = set()
    for cls in classes:
        ids = {node_of[lab] for lab in cls}
        assert len(ids) == 1
        seen |= ids
    assert len(seen) == len(classes)
    for line in fig3["surround"]:
        child, par = map(int, line.split())
        assert res["parent"][node_of[child]] == node_of[par]


def test_fig3_fill(fig3):
    img = grid(fig3["grid"])
    res = orc.analyze(img)
    want = [r.split() for r in fig3["filled"]]
    for T in (11, 12, 10**6, INT64_MAX):
        fmap, ff, fpar = orc.fill(res, T)
        for r in want:
            n = int(r[0])
            vals = [INT64_MAX if v == "EMPTY" else int(v) for v in r[1:8]]
            assert list(ff[:, n]) == vals
            assert fpar[n] == int(r[8])
            assert fmap[n] == int(r[9])
    for T in (10, 0, -1):
        fmap, ff, fpar = orc.fill(res, T)
        np.testing.assert_array_equal(fmap, np.arange(res["n"]))
        np.testing.assert_array_equal(ff, res["feat"])
        np.testing.assert_array_equal(fpar, res["parent"])


def test_fig3_paper_algorithm(fig3):
    """Algorithms 1-4 restated give the same labels, tree and features, and
    with hole filling merge the hole as the paper narrates."""
    img = grid(fig3["grid"])
    res = orc.analyze(img)
    lab, par, feats, n = paper_lsl.analyze(img.tolist())
    assert n == res["n"]
    np.testing.assert_array_equal(np.array(lab), res["node"])
    assert par == list(res["parent"])
    assert [list(f) for f in feats] == res["feat"].T.tolist()
    lab, par, feats, n = paper_lsl.analyze(img.tolist(), fill=True)
    assert n == 2
    assert feats[1][0] == 67 and feats[1][5] == 463 and feats[1][6] == 217


# ------------------------------------------------------ brute force (tiny)


def all_images(h, w):
    for bits in range(1 << (h * w)):
        yield np.array([(bits >> k) & 1 for k in range(h * w)], np.uint8).reshape(h, w)


@pytest.mark.parametrize("h,w", [(1, 1), (1, 5), (5, 1), (2, 2), (2, 3), (3, 2), (3, 3),
                                 (1, 12), (12, 1), (2, 6), (3, 4), (4, 3)])
def test_exhaustive_small_vs_twin(h, w):
    for img in all_images(h, w):
        res = orc.analyze(img)
        assert_same_as_twin(res, twin.analyze(img.tolist()))


def test_exhaustive_4x4_vs_twin():
    for img in all_images(4, 4):
        res = orc.analyze(img)
        assert_same_as_twin(res, twin.analyze(img.tolist()))


@pytest.mark.parametrize("h,w", [(3, 3), (3, 4), (4, 3), (2, 5)])
def test_exhaustive_vs_paper_algorithm(h, w):
    for img in all_images(h, w):
        res = orc.analyze(img)
        lab, par, feats, n = paper_lsl.analyze(img.tolist())
        assert n == res["n"]
        np.testing.assert_array_equal(np.array(lab), res["node"])
        assert par == list(res["parent"])
        assert [list(f) for f in feats] == res["feat"].T.tolist()


def test_random_vs_twin_and_paper_algorithm():
    rng = np.random.default_rng(7)
    for it in range(300):
        h, w = int(rng.integers(1, 13)), int(rng.integers(1, 13))
        img = (rng.random((h, w)) < rng.uniform(0.1, 0.9)).astype(np.uint8)
        for conn in (0, 1):
            res = orc.analyze(img, conn=conn)
            assert_same_as_twin(res, twin.analyze(img.tolist(), conn=conn))
            lab, par, feats, n = paper_lsl.analyze(img.tolist(), conn=conn)
            assert n == res["n"]
            np.testing.assert_array_equal(np.array(lab), res["node"])
            assert par == list(res["parent"])
            assert [list(f) for f in feats] == res["feat"].T.tolist()


def test_paper_algorithm_unconditional_fill_matches_oracle_fill():
    """Algorithm 3's hole filling equals the oracle's fill with T = infinity."""
    rng = np.random.default_rng(11)
    for it in range(300):
        h, w = int(rng.integers(1, 13)), int(rng.integers(1, 13))
        img = (rng.random((h, w)) < rng.uniform(0.2, 0.8)).astype(np.uint8)
        res = orc.analyze(img)
        fmap, ff, fpar = orc.fill(res, INT64_MAX)
        lab, par, feats, n = paper_lsl.analyze(img.tolist(), fill=True)
        surv = np.unique(fmap)
        assert n == len(surv)
        dense = {int(s): k for k, s in enumerate(surv)}
        np.testing.assert_array_equal(np.vectorize(lambda v: dense[int(fmap[v])])(res["node"]),
                                      np.array(lab))
        for s, k in dense.items():
            assert list(ff[:, s]) == list(feats[k])
            assert (fpar[s] == -1 and par[k] == -1) or dense[int(fpar[s])] == par[k]


# ------------------------------------------------------------- library


@pytest.mark.parametrize("seed", range(6))
def test_partition_matches_scipy(seed):
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(100 + seed)
    h, w = int(rng.integers(20, 90)), int(rng.integers(20, 90))
    g = int(rng.integers(1, 4))
    img = inputs.granular(h, w, float(rng.uniform(0.2, 0.8)), g, seed)
    res = orc.analyze(img)
    lf, nf = ndi.label(img, structure=np.ones((3, 3)))
    lb, nb = ndi.label(1 - img)
    # same partition: the map between ids is a bijection on each colour
    fgm = img != 0
    pairs_f = set(zip(lf[fgm].tolist(), res["node"][fgm].tolist()))
    assert len(pairs_f) == nf == len({b for _, b in pairs_f})
    pairs_b = set(zip(lb[~fgm].tolist(), res["node"][~fgm].tolist()))
    assert len({a for a, _ in pairs_b}) == nb == len(pairs_b)
    # background library components touching the border are all node 0
    border = np.zeros_like(fgm)
    border[0, :] = border[-1, :] = border[:, 0] = border[:, -1] = True
    ext = set(lb[border & ~fgm].tolist())
    for a, b in pairs_b:
        assert (b == 0) == (a in ext)


# ------------------------------------------- closed forms and invariants


def check_invariants(img, res, conn=0):
    h, w = img.shape
    n = res["n"]
    feat = res["feat"]
    par = res["parent"]
    assert n <= orc.capacity(w, h)
    assert feat[orc.AREA].sum() == w * h
    assert feat[orc.SX].sum() == h * w * (w - 1) // 2
    assert feat[orc.SY].sum() == w * h * (h - 1) // 2
    assert par[0] == -1 and res["node_fg"][0] == 0
    if n > 1:
        assert np.all(par[1:] < np.arange(1, n)) and np.all(par[1:] >= 0)
        assert np.all(res["node_fg"][1:] != res["node_fg"][par[1:]])
    fp = first_pixels(res["node"])
    order = [fp[k] for k in range(1, n)]
    assert order == sorted(order)
    for k in range(1, n):
        y, x = divmod(fp[k], w)
        assert feat[orc.XMIN, k] <= x <= feat[orc.XMAX, k]
        assert feat[orc.YMIN, k] == y <= feat[orc.YMAX, k]
    assert orc.euler(res) == checks.euler_bitquad(img, conn)


@pytest.mark.parametrize("case", range(10))
def test_invariants_random(case):
    rng = np.random.default_rng(500 + case)
    h, w = int(rng.integers(1, 200)), int(rng.integers(1, 200))
    img = inputs.granular(h, w, float(rng.uniform(0.05, 0.95)), int(rng.integers(1, 6)), case)
    for conn in (0, 1):
        check_invariants(img, orc.analyze(img, conn=conn), conn)


def test_invariants_config_512():
    img = inputs.bernoulli(512, 512, 0.5, 1)
    check_invariants(img, orc.analyze(img))


def test_surround_by_barrier_search():
    rng = np.random.default_rng(21)
    for it in range(60):
        h, w = int(rng.integers(3, 16)), int(rng.integers(3, 16))
        img = inputs.granular(h, w, float(rng.uniform(0.3, 0.7)), int(rng.integers(1, 3)), it)
        for conn in (0, 1):
            res = orc.analyze(img, conn=conn)
            for k in range(1, res["n"]):
                p = int(res["parent"][k])
                if p == 0:
                    continue
                assert checks.surrounds(res["node"], res["node_fg"], k, p, conn)


@pytest.mark.parametrize("T", [-1, 0, 1, 2, 3, 5, 10, 40, INT64_MAX])
def test_fill_matches_brute_force(T):
    rng = np.random.default_rng(31)
    for it in range(40):
        h, w = int(rng.integers(2, 40)), int(rng.integers(2, 40))
        img = inputs.granular(h, w, float(rng.uniform(0.3, 0.8)), int(rng.integers(1, 3)), it)
        res = orc.analyze(img)
        fmap, ff, fpar = orc.fill(res, T)
        filled = checks.brute_fill_image(img, res["node"], res["node_fg"], res["feat"][orc.AREA], T)
        res2 = orc.analyze(filled)
        # every pixel's survivor corresponds one-to-one to its node after repainting
        pairs = set(zip(fmap[res["node"]].ravel().tolist(), res2["node"].ravel().tolist()))
        assert len(pairs) == len({a for a, _ in pairs}) == len({b for _, b in pairs})
        for a, b in pairs:
            assert list(ff[:, a]) == list(res2["feat"][:, b])
        surv = sorted({a for a, _ in pairs} | {0})
        assert all(fmap[s] == s for s in surv)
        for k in range(res["n"]):
            if fmap[k] != k:
                assert fpar[k] == -1 and ff[orc.AREA, k] == 0


# ---------------------------------------------------------- special cases


def test_all_background():
    res = orc.analyze(np.zeros((7, 9), np.uint8))
    assert res["n"] == 1 and res["parent"][0] == -1
    assert list(res["feat"][:, 0]) == [63, 0, 0, 8, 6, 9 * 8 // 2 * 7, 7 * 6 // 2 * 9]


def test_all_foreground():
    res = orc.analyze(np.ones((5, 6), np.uint8))
    assert res["n"] == 2 and list(res["parent"]) == [-1, 0]
    assert list(res["feat"][:, 0]) == [0, INT64_MAX, INT64_MAX, -1, -1, 0, 0]
    assert res["feat"][orc.AREA, 1] == 30
    assert np.all(res["bg"] == -1) and np.all(res["fg"] == 1)


def test_checkerboard():
    h, w = 9, 12
    img = inputs.adversarial(h, w, "checker0")
    res = orc.analyze(img)
    n_fg = 1
    interior_bg = int(((img[1:-1, 1:-1]) == 0).sum())
    assert res["counts"][1] == n_fg
    assert res["n"] == 1 + n_fg + interior_bg
    assert np.all(res["parent"][2:] == 1)
    border = np.zeros_like(img, bool)
    border[0, :] = border[-1, :] = border[:, 0] = border[:, -1] = True
    assert np.all(res["node"][border & (img == 0)] == 0)


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_nested_square_rings(k):
    """k nested 1-pixel square rings with 1-pixel gaps: a chain of depth 2k,
    ring j (0-based from outside) of side s_j = 4k - 1 - 4j has area 4(s_j - 1)."""
    s = 4 * k + 1
    img = np.zeros((s + 2, s + 2), np.uint8)
    for j in range(k):
        a, b = 1 + 2 * j, s - 2 * j
        img[a, a:b + 1] = img[b, a:b + 1] = 1
        img[a:b + 1, a] = img[a:b + 1, b] = 1
    res = orc.analyze(img)
    assert res["n"] == 2 * k + 1
    assert list(res["parent"]) == [-1] + list(range(2 * k))
    for j in range(k):
        side = s - 4 * j
        assert res["feat"][orc.AREA, 1 + 2 * j] == 4 * (side - 1)
        inner = side - 2
        assert res["feat"][orc.AREA, 2 + 2 * j] == inner * inner - (0 if j == k - 1 else (inner - 2) ** 2)
    fmap, ff, fpar = orc.fill(res, INT64_MAX)
    assert np.all(fmap[1:] == 1) and ff[orc.AREA, 1] == s * s


def test_padding_bytes_ignored():
    img = inputs.bernoulli(13, 17, 0.5, 3)
    a = orc.analyze(img)
    b = orc.analyze(inputs.pitched(img, 32), w=17)
    c = orc.analyze(inputs.pitched(img * 255, 48, pad_value=0x5A), w=17)
    for key in ("node", "fg", "bg", "parent", "feat", "counts"):
        np.testing.assert_array_equal(a[key], b[key])
        np.testing.assert_array_equal(a[key], c[key])


def test_capacity_bound_reached():
    """The node bound is tight on a checkerboard with odd sides."""
    for h, w in [(1, 1), (3, 3), (5, 7), (7, 5)]:
        img = inputs.adversarial(h, w, "checker1")
        img[0, :] = img[-1, :] = 1
        img[:, 0] = img[:, -1] = 1
        res = orc.analyze(img)
        assert res["n"] <= orc.capacity(w, h)


# --------------------------------------------------- object removal (dual)


@pytest.mark.parametrize("T", [-1, 0, 1, 2, 4, 9, 30, INT64_MAX])
def test_object_removal_matches_brute_force(T):
    """Removing foreground objects with area <= T from the node table equals
    painting them background and labelling again."""
    rng = np.random.default_rng(41)
    for it in range(40):
        h, w = int(rng.integers(2, 40)), int(rng.integers(2, 40))
        img = inputs.granular(h, w, float(rng.uniform(0.2, 0.7)), int(rng.integers(1, 3)), it + 100)
        res = orc.analyze(img)
        fmap, ff, fpar = orc.fill(res, T, target_fg=1)
        painted = checks.brute_remove_objects(img, res["node"], res["node_fg"], res["feat"][orc.AREA], T)
        res2 = orc.analyze(painted)
        pairs = set(zip(fmap[res["node"]].ravel().tolist(), res2["node"].ravel().tolist()))
        assert len(pairs) == len({a for a, _ in pairs}) == len({b for _, b in pairs})
        for a, b in pairs:
            assert list(ff[:, a]) == list(res2["feat"][:, b])
        # the relabelled images equal the repainted image's labels up to
        # renumbering: colours agree pixel by pixel, and the survivor ids
        # written in them partition the image exactly as the repainted
        # image's own labelling does (a bijection between the two id sets)
        fg2, bg2 = orc.relabel(res, fmap)
        assert np.array_equal(fg2 >= 0, painted != 0) and np.array_equal(bg2 >= 0, painted == 0)
        ids = np.where(fg2 >= 0, fg2, bg2)
        assert ids.min() >= 0
        idpairs = set(zip(ids.ravel().tolist(), res2["node"].ravel().tolist()))
        assert len(idpairs) == len({a for a, _ in idpairs}) == len({b for _, b in idpairs})
        for k in range(res["n"]):
            if fmap[k] != k:
                assert fpar[k] == -1 and ff[orc.AREA, k] == 0


def test_filters_match_twin():
    rng = np.random.default_rng(43)
    for it in range(150):
        h, w = int(rng.integers(1, 11)), int(rng.integers(1, 11))
        img = (rng.random((h, w)) < rng.uniform(0.2, 0.8)).astype(np.uint8)
        res = orc.analyze(img)
        tw = twin.analyze(img.tolist())
        for tgt in (0, 1):
            for T in (-1, 0, 1, 3, INT64_MAX):
                fmap, ff, fpar = orc.fill(res, T, target_fg=tgt)
                m2, f2, p2 = twin.fill(tw, T, target_fg=tgt)
                assert list(fmap) == m2 and list(fpar) == p2
                assert ff.T.tolist() == f2
