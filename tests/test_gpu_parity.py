"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Everything is integer and the result is unique (canonical node ids), so the
bar is bit-exact equality of the label images, the tree, the int64 features,
the counts and the hole-filling outputs."""
import numpy as np
import pytest
import torch

from oracle import reference as orc
from paper_2006_09299_gb300 import inputs

pytestmark = pytest.mark.gpu

INT64_MAX = np.iinfo(np.int64).max


@pytest.fixture(scope="module")
def ccl():
    import __graft_entry__ as g
    g.build()
    from paper_2006_09299_gb300 import ccl as m
    return m


def to_dev(padded):
    return torch.from_numpy(np.ascontiguousarray(padded)).cuda()


def run_single(ccl, padded, w, conn=0, labels=True, fills=()):
    h, pitch = padded.shape
    ctx = ccl.Context(w, h, pitch, conn=conn)
    out = ctx.analyze(to_dev(padded), labels=labels)
    res = {}
    n, nfg, nbg, st = ctx.get_counts()
    res.update(n=n, counts=(n, nfg, nbg), status=st,
               parent=out.parent[:n].cpu().numpy(), feat=out.features[:, :n].cpu().numpy())
    if labels:
        res["fg"] = out.fg.cpu().numpy()
        res["bg"] = out.bg.cpu().numpy()
    res["fills"] = {}
    for T in fills:
        ctx.fill_holes(T)
        torch.cuda.synchronize()
        res["fills"][T] = (out.fill_map[:n].cpu().numpy(), out.filled_features[:, :n].cpu().numpy(),
                           out.filled_parent[:n].cpu().numpy())
    st2 = ctx.get_counts()[3]
    res["status"] |= st2
    ctx.close()
    return res


def oracle_cap(w, h):
    return min(orc.capacity(w, h), max(4096, (w * h) // 4))


def run_oracle(padded, w, conn=0):
    h = padded.shape[0]
    try:
        return orc.analyze(padded, w=w, conn=conn, cap=oracle_cap(w, h))
    except RuntimeError:
        return orc.analyze(padded, w=w, conn=conn)


def assert_parity(g, r, labels=True, fills=()):
    assert g["status"] == 0, g["status"]
    assert g["n"] == r["n"]
    assert g["counts"] == (int(r["counts"][0]), int(r["counts"][1]), int(r["counts"][2]))
    if labels:
        np.testing.assert_array_equal(g["fg"], r["fg"])
        np.testing.assert_array_equal(g["bg"], r["bg"])
    np.testing.assert_array_equal(g["parent"], r["parent"])
    np.testing.assert_array_equal(g["feat"], r["feat"])
    for T in fills:
        fmap, ff, fpar = orc.fill(r, T)
        gm, gf, gp = g["fills"][T]
        np.testing.assert_array_equal(gm, fmap)
        np.testing.assert_array_equal(gf, ff)
        np.testing.assert_array_equal(gp, fpar)


SIZES = [(1, 1), (1, 2), (2, 1), (3, 40), (15, 17), (31, 33), (32, 32), (33, 1023), (64, 1024),
         (65, 1025), (70, 2049), (100, 3000), (257, 1100), (40, 4100), (2100, 7), (1000, 1)]


@pytest.mark.parametrize("conn", [0, 1])
@pytest.mark.parametrize("kind", inputs.ADVERSARIAL_KINDS)
def test_adversarial_shapes(ccl, kind, conn):
    for h, w in SIZES:
        img = inputs.adversarial(h, w, kind)
        pitch = -(-w // 16) * 16
        padded = inputs.pitched(img, pitch)
        g = run_single(ccl, padded, w, conn=conn, fills=(0, 3, INT64_MAX))
        assert_parity(g, run_oracle(padded, w, conn), fills=(0, 3, INT64_MAX))


@pytest.mark.parametrize("conn", [0, 1])
@pytest.mark.parametrize("case", range(8))
def test_random_multi_tile(ccl, conn, case):
    rng = np.random.default_rng(900 + case)
    h = int(rng.integers(30, 200))
    w = int(rng.integers(900, 3300))
    d = [0.1, 0.3, 0.5, 0.7, 0.9, 0.45, 0.55, 0.62][case]
    g = [1, 1, 1, 1, 1, 2, 3, 4][case]
    img = inputs.granular(h, w, d, g, case)
    pitch = -(-w // 16) * 16 + 16 * int(rng.integers(0, 3))
    padded = inputs.pitched(img * np.uint8(1 + 254 * (case % 2)), pitch)
    res = run_single(ccl, padded, w, conn=conn, fills=(-1, 2, 64, INT64_MAX))
    assert_parity(res, run_oracle(padded, w, conn), fills=(-1, 2, 64, INT64_MAX))


def test_config1_512(ccl):
    img = inputs.bernoulli(512, 512, 0.5, 1)
    g = run_single(ccl, img, 512, fills=(64, INT64_MAX))
    assert_parity(g, run_oracle(img, 512), fills=(64, INT64_MAX))


def test_labels_off(ccl):
    img = inputs.granular(300, 2500, 0.5, 2, 5)
    padded = inputs.pitched(img, 2512)
    g = run_single(ccl, padded, 2500, labels=False, fills=(10,))
    assert_parity(g, run_oracle(padded, 2500), labels=False, fills=(10,))


def test_context_reuse_and_graph_replay(ccl):
    h, w = 130, 2000
    ctx = ccl.Context(w, h, 2000)
    out = ctx.new_outputs()
    for seed in range(4):
        img = inputs.granular(h, w, 0.3 + 0.1 * seed, 1 + seed, seed)
        ctx.analyze(to_dev(img), out=out)
        n, nfg, nbg, st = ctx.get_counts()
        r = run_oracle(img, w)
        assert st == 0 and n == r["n"]
        np.testing.assert_array_equal(out.fg.cpu().numpy(), r["fg"])
        np.testing.assert_array_equal(out.features[:, :n].cpu().numpy(), r["feat"])
        np.testing.assert_array_equal(out.parent[:n].cpu().numpy(), r["parent"])
    ctx.close()


def test_batched_equals_oracle_and_single(ccl):
    batch = inputs.uneven_batch(seed=4, n=24, lo=16, hi=1500)
    imgs = [(to_dev(p), w) for p, w in batch]
    tot = sum(p.shape[0] * w for p, w in batch)
    bctx = ccl.BatchContext(len(batch), tot, 1500)
    outs = bctx.analyze(imgs, fill=True)
    bctx.fill_holes(20)
    torch.cuda.synchronize()
    for (p, w), o in zip(batch, outs):
        r = run_oracle(p, w)
        n = o.n
        assert o.status() == 0
        assert n == r["n"]
        np.testing.assert_array_equal(o.fg.cpu().numpy(), r["fg"])
        np.testing.assert_array_equal(o.bg.cpu().numpy(), r["bg"])
        np.testing.assert_array_equal(o.parent[:n].cpu().numpy(), r["parent"])
        np.testing.assert_array_equal(o.features[:, :n].cpu().numpy(), r["feat"])
        fmap, ff, fpar = orc.fill(r, 20)
        np.testing.assert_array_equal(o.fill_map[:n].cpu().numpy(), fmap)
        np.testing.assert_array_equal(o.filled_features[:, :n].cpu().numpy(), ff)
        np.testing.assert_array_equal(o.filled_parent[:n].cpu().numpy(), fpar)
    # the same batch again (graph replay) gives the same result
    outs2 = bctx.analyze(imgs)
    torch.cuda.synchronize()
    for o, o2 in zip(outs, outs2):
        assert torch.equal(o.fg, o2.fg) and torch.equal(o.counts[:3], o2.counts[:3])
    bctx.close()


def test_batched_from_host_frames_equals_device_inputs(ccl):
    """ccl_analyze_batched_from_host: frames in host memory, pinned or
    pageable, with row strides of w (any w), the device buffer's or wider,
    are copied into device image buffers and analysed; the results equal those of the same images
    analysed from device memory. A host pitch below w is refused."""
    batch = inputs.uneven_batch(seed=9, n=12, lo=16, hi=1300)
    tot = sum(p.shape[0] * w for p, w in batch)
    ref_ctx = ccl.BatchContext(len(batch), tot, 1300)
    ref = ref_ctx.analyze([(to_dev(p), w) for p, w in batch], fill=True)
    ref_ctx.fill_holes(20)
    ctx = ccl.BatchContext(len(batch), tot, 1300, graph_cache=False)
    outs = ctx.new_outputs([(w, p.shape[0]) for p, w in batch], fill=True)
    frames, pitches, keep = [], [], []
    descs = (ccl.ImageDesc * len(batch))()
    for i, ((p, w), o) in enumerate(zip(batch, outs)):
        h = p.shape[0]
        dev_img = torch.full((h, -(-w // 16) * 16), 77, dtype=torch.uint8, device="cuda")
        dpitch = dev_img.shape[1]
        if i % 4 == 0:      # pinned, rows w bytes apart
            f = torch.empty((h, w), dtype=torch.uint8).pin_memory()
            f.numpy()[:] = p[:, :w]
            addr, pitch = f.data_ptr(), w
        elif i % 4 == 1:    # pageable, rows w bytes apart
            f = np.ascontiguousarray(p[:, :w])
            addr, pitch = f.__array_interface__["data"][0], w
        elif i % 4 == 2:    # pinned, rows laid out as on the device (one linear copy)
            f = torch.zeros((h, dpitch), dtype=torch.uint8).pin_memory()
            f.numpy()[:, :w] = p[:, :w]
            addr, pitch = f.data_ptr(), dpitch
        else:               # pageable, the padded rows (pitch wider than the device's)
            f = np.ascontiguousarray(p)
            addr, pitch = f.__array_interface__["data"][0], p.shape[1]
        keep += [f, dev_img]
        descs[i] = ccl.BatchContext.image_desc(dev_img, w, o)
        frames.append(addr)
        pitches.append(pitch)
    for call in range(2):
        for o in outs:
            o.fg.fill_(-7)
        ctx.analyze_from_host(descs, frames, pitches)
        ctx.fill_holes(20)
        torch.cuda.synchronize()
        for o, r in zip(outs, ref):
            n = r.n
            assert o.status() == 0 and o.n == n, call
            assert torch.equal(o.fg, r.fg) and torch.equal(o.bg, r.bg), call
            assert torch.equal(o.parent[:n], r.parent[:n]), call
            assert torch.equal(o.features[:, :n], r.features[:, :n]), call
            assert torch.equal(o.fill_map[:n], r.fill_map[:n]), call
            assert torch.equal(o.filled_features[:, :n], r.filled_features[:, :n]), call
    bad = list(pitches)
    bad[1] = batch[1][1] - 1
    with pytest.raises(RuntimeError):
        ctx.analyze_from_host(descs, frames, bad)
    ctx.close()
    ref_ctx.close()


def test_capacity_error_reported_on_device(ccl):
    img = inputs.adversarial(64, 64, "checker0")
    d = to_dev(img)
    bctx = ccl.BatchContext(1, 64 * 64, 64)
    o = ccl.Analysis(64, 64, 100, True, "cuda")   # far fewer slots than nodes
    bctx.analyze([(d, 64)], outs=[o])
    torch.cuda.synchronize()
    assert o.status() & ccl.ERR_CAPACITY
    r = run_oracle(img, 64)
    assert o.n == r["n"]
    np.testing.assert_array_equal(o.fg.cpu().numpy(), r["fg"])   # labels are still right
    bctx.close()


def test_bad_alignment_is_rejected(ccl):
    buf = torch.zeros(64 * 64 + 16, dtype=torch.uint8, device="cuda")
    bctx = ccl.BatchContext(1, 64 * 64, 64)
    o = ccl.Analysis(64, 64, ccl.node_capacity(64, 64), True, "cuda")
    with pytest.raises(ccl.CCLError) as e:
        bctx.analyze([(buf[1:1 + 64 * 64].view(64, 64), 64)], outs=[o])
    assert e.value.status == ccl.ERR_ALIGN
    bctx.close()


# ------------------------------------------------------------ full sizes


def test_sweep_4096_selected(ccl):
    """Density x granularity sweep at full size: g = 1 (the worst case) and
    two coarser images, compared element by element."""
    for i_d, i_g in [(2, 0), (3, 0), (4, 2), (0, 4)]:
        img = inputs.sweep_image(i_d, i_g)
        g = run_single(ccl, img, 4096, fills=(64,))
        assert_parity(g, run_oracle(img, 4096), fills=(64,))


def test_rings_8192_full(ccl):
    img = inputs.rings()
    g = run_single(ccl, img, 8192, fills=(64,))
    assert_parity(g, run_oracle(img, 8192), fills=(64,))


@pytest.mark.parametrize("conn", [0, 1])
def test_filter_objects_relabel_euler(ccl, conn):
    """Small-object removal (the dual filter), the label images rewritten
    through the filter map, and the Euler number, each against the oracle and
    against the pixel-level brute force of the oracle's checks."""
    from oracle import checks
    for seed, (h, w) in enumerate([(1, 1), (33, 1023), (70, 2049), (257, 1100)]):
        img = inputs.granular(h, w, 0.45, 1 + seed % 3, 11 + seed)
        pitch = -(-w // 16) * 16
        padded = np.zeros((h, pitch), np.uint8)
        padded[:, :w] = img
        r = run_oracle(padded, w, conn)
        ctx = ccl.Context(w, h, pitch, conn=conn)
        out = ctx.analyze(to_dev(padded))
        n = ctx.get_counts()[0]
        assert ctx.euler() == orc.euler(r) == checks.euler_bitquad(padded[:, :w], conn)
        for target, T in ((ccl.TARGET_OBJECTS, 3), (ccl.TARGET_OBJECTS, 40), (ccl.TARGET_HOLES, 5)):
            ctx.filter_components(target, T)
            fg_out = torch.empty_like(out.fg)
            bg_out = torch.empty_like(out.bg)
            ctx.relabel_filtered(fg_out, bg_out)
            torch.cuda.synchronize()
            assert ctx.get_counts()[3] == 0
            fmap, ff, fpar = orc.fill(r, T, target_fg=target)
            np.testing.assert_array_equal(out.fill_map[:n].cpu().numpy(), fmap)
            np.testing.assert_array_equal(out.filled_features[:, :n].cpu().numpy(), ff)
            np.testing.assert_array_equal(out.filled_parent[:n].cpu().numpy(), fpar)
            efg, ebg = orc.relabel(r, fmap)
            np.testing.assert_array_equal(fg_out.cpu().numpy(), efg)
            np.testing.assert_array_equal(bg_out.cpu().numpy(), ebg)
        # in place: the outputs may be the analysis label images themselves
        ctx.filter_components(ccl.TARGET_OBJECTS, 3)
        ctx.relabel_filtered(out.fg, out.bg)
        torch.cuda.synchronize()
        efg, ebg = orc.relabel(r, orc.fill(r, 3, target_fg=1)[0])
        np.testing.assert_array_equal(out.fg.cpu().numpy(), efg)
        np.testing.assert_array_equal(out.bg.cpu().numpy(), ebg)
        ctx.close()


def test_filter_batched_objects(ccl):
    batch = inputs.uneven_batch(seed=9, n=12, lo=16, hi=1200)
    imgs = [(to_dev(p), w) for p, w in batch]
    tot = sum(p.shape[0] * w for p, w in batch)
    bctx = ccl.BatchContext(len(batch), tot, 1200)
    outs = bctx.analyze(imgs, fill=True)
    bctx.filter_components(ccl.TARGET_OBJECTS, 12)
    fg_outs = [torch.empty_like(o.fg) for o in outs]
    bg_outs = [torch.empty_like(o.bg) for o in outs]
    fg_outs[3] = bg_outs[3] = None   # an image may be skipped
    bctx.relabel_filtered(fg_outs, bg_outs)
    torch.cuda.synchronize()
    for i, ((p, w), o) in enumerate(zip(batch, outs)):
        if fg_outs[i] is None:
            continue
        r = run_oracle(p, w)
        efg, ebg = orc.relabel(r, orc.fill(r, 12, target_fg=1)[0])
        np.testing.assert_array_equal(fg_outs[i].cpu().numpy(), efg)
        np.testing.assert_array_equal(bg_outs[i].cpu().numpy(), ebg)
    for (p, w), o in zip(batch, outs):
        r = run_oracle(p, w)
        n = o.n
        assert o.status() == 0 and n == r["n"]
        fmap, ff, fpar = orc.fill(r, 12, target_fg=1)
        np.testing.assert_array_equal(o.fill_map[:n].cpu().numpy(), fmap)
        np.testing.assert_array_equal(o.filled_features[:, :n].cpu().numpy(), ff)
        np.testing.assert_array_equal(o.filled_parent[:n].cpu().numpy(), fpar)
    bctx.close()


def test_uneven256_full_batch_as_benched(ccl):
    """The full 256-image uneven batch (about 99 Mpx) in one batched call,
    the launch configuration the bench times (CUDA graph replay), under every
    tile height and merge schedule the autotuner can pick, every image
    against the oracle."""
    batch = inputs.uneven_batch(seed=4, n=256)
    imgs = [(to_dev(p), w) for p, w in batch]
    shapes = [(w, p.shape[0]) for p, w in batch]
    tot = sum(p.shape[0] * w for p, w in batch)
    refs = []
    for p, w in batch:
        r = run_oracle(p, w)
        f = orc.fill(r, 64)
        r.pop("node")   # not compared; keeps the host copy of 256 results smaller
        refs.append((r, f))
    bctx = ccl.BatchContext(len(batch), tot, 2048)
    outs = bctx.new_outputs(shapes, labels=True, fill=True)
    # every tile shape and merge schedule the autotuner can choose
    for rows, cols, split in [(32, 1024, 4), (16, 1024, 4), (32, 512, 4), (16, 512, 4), (32, 1024, 1),
                              (32, 1024, 2), (32, 1024, 8), (16, 512, 1), (32, 512, 2), (16, 1024, 8)]:
        bctx.set_tile_rows(rows)
        bctx.set_tile_cols(cols)
        bctx.set_merge_split(split)
        for _ in range(2):   # the second call replays the cached graph
            bctx.analyze(imgs, outs=outs)
            bctx.fill_holes(64)
        torch.cuda.synchronize()
        for o, (r, (fmap, ff, fpar)) in zip(outs, refs):
            n = o.n
            assert o.status() == 0 and n == r["n"], (rows, cols, split)
            np.testing.assert_array_equal(o.fg.cpu().numpy(), r["fg"])
            np.testing.assert_array_equal(o.bg.cpu().numpy(), r["bg"])
            np.testing.assert_array_equal(o.parent[:n].cpu().numpy(), r["parent"])
            np.testing.assert_array_equal(o.features[:, :n].cpu().numpy(), r["feat"])
            np.testing.assert_array_equal(o.fill_map[:n].cpu().numpy(), fmap)
            np.testing.assert_array_equal(o.filled_features[:, :n].cpu().numpy(), ff)
            np.testing.assert_array_equal(o.filled_parent[:n].cpu().numpy(), fpar)
    bctx.close()


def test_sweep4096_full_batch_as_benched(ccl):
    """All 25 images of the default bench workload (4096 x 4096, d in
    {0.1..0.9} x g in {1..16}) in one batched call with hole filling 64, as
    the bench times it, every image against the oracle."""
    batch = [(inputs.sweep_image(i, j), 4096) for i in range(5) for j in range(5)]
    imgs = [(to_dev(p), w) for p, w in batch]
    bctx = ccl.BatchContext(len(batch), 25 * 4096 * 4096, 4096)
    outs = bctx.new_outputs([(4096, 4096)] * len(batch), labels=True, fill=True)
    for _ in range(2):
        bctx.analyze(imgs, outs=outs)
        bctx.fill_holes(64)
    torch.cuda.synchronize()
    for (p, w), o in zip(batch, outs):
        r = run_oracle(p, w)
        n = o.n
        assert o.status() == 0 and n == r["n"]
        np.testing.assert_array_equal(o.fg.cpu().numpy(), r["fg"])
        np.testing.assert_array_equal(o.bg.cpu().numpy(), r["bg"])
        np.testing.assert_array_equal(o.parent[:n].cpu().numpy(), r["parent"])
        np.testing.assert_array_equal(o.features[:, :n].cpu().numpy(), r["feat"])
        fmap, ff, fpar = orc.fill(r, 64)
        np.testing.assert_array_equal(o.fill_map[:n].cpu().numpy(), fmap)
        np.testing.assert_array_equal(o.filled_features[:, :n].cpu().numpy(), ff)
        np.testing.assert_array_equal(o.filled_parent[:n].cpu().numpy(), fpar)
    bctx.close()
