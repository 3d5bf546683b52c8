"""Autotuner logic (CPU, fake timer) and tile-height parity (GPU)."""
import numpy as np
import pytest

from paper_2006_09299_gb300 import autotune, inputs


class FakeCtx:
    def __init__(self):
        self.rows = self.cols = self.split = None

    def set_tile_rows(self, rows):
        self.rows = rows

    def set_tile_cols(self, cols):
        self.cols = cols

    def set_merge_split(self, split):
        self.split = split


def test_tune_picks_fastest_shape_and_schedule_and_caches(tmp_path):
    ctx = FakeCtx()
    cost = {(32, 1024, 4): 2.0, (16, 1024, 4): 1.5, (32, 512, 4): 1.7, (16, 512, 4): 1.6,
            (16, 1024, 1): 1.6, (16, 1024, 2): 1.4, (16, 1024, 8): 1.45}
    timer = lambda fn, reps: cost[(ctx.rows, ctx.cols, ctx.split)]
    path = str(tmp_path / "t.json")
    choice, times = autotune.tune(ctx, lambda: None, "k1", cache_path=path, timer=timer)
    # shapes first at the default schedule, then schedules at the best shape
    assert choice == {"rows": 16, "cols": 1024, "merge_split": 2}
    assert (ctx.rows, ctx.cols, ctx.split) == (16, 1024, 2)
    assert set(times) == {autotune.choice_name(*k) for k in cost}
    # cached: the timer is not consulted again
    ctx2 = FakeCtx()
    choice2, _ = autotune.tune(ctx2, lambda: None, "k1", cache_path=path,
                               timer=lambda fn, reps: pytest.fail("re-timed"))
    assert choice2 == choice and (ctx2.rows, ctx2.cols, ctx2.split) == (16, 1024, 2)
    # a narrower tile wins after a forced re-tune
    cost.update({(32, 512, 4): 1.0, (32, 512, 1): 1.1, (32, 512, 2): 0.9, (32, 512, 8): 1.2})
    choice3, _ = autotune.tune(ctx, lambda: None, "k1", cache_path=path, timer=timer, force=True)
    assert choice3 == {"rows": 32, "cols": 512, "merge_split": 2}


def test_size_class_buckets():
    a = autotune.size_class([(4096, 4096)] * 25)
    b = autotune.size_class([(4000, 4090)] * 25)
    c = autotune.size_class([(512, 512)])
    assert a == b and a != c


@pytest.mark.gpu
@pytest.mark.parametrize("rows,cols,split", [(16, 1024, 4), (32, 1024, 4), (32, 1024, 1), (32, 1024, 2),
                                             (32, 1024, 8), (16, 1024, 1), (16, 1024, 8), (32, 512, 4),
                                             (16, 512, 4), (32, 512, 1), (16, 512, 8)])
def test_tile_shapes_agree_with_oracle(rows, cols, split):
    import torch

    import __graft_entry__ as g
    g.build()
    from oracle import reference as orc
    from paper_2006_09299_gb300 import ccl

    cases = [inputs.granular(70, 2100, 0.5, 1, 1), inputs.granular(40, 1030, 0.6, 2, 2),
             inputs.adversarial(33, 1025, "diag"), inputs.adversarial(47, 1100, "spiral"),
             inputs.adversarial(17, 3000, "checker0"), inputs.rings(300, 2500, seed=9, n_sets=40)]
    for img in cases:
        h, w = img.shape
        pitch = -(-w // 16) * 16
        padded = inputs.pitched(img, pitch)
        for conn in (0, 1):
            ctx = ccl.Context(w, h, pitch, conn=conn)
            ctx.set_tile_rows(rows)
            ctx.set_tile_cols(cols)
            ctx.set_merge_split(split)
            out = ctx.analyze(torch.from_numpy(padded).cuda())
            ctx.fill_holes(8)
            n, nf, nb, st = ctx.get_counts()
            ref = orc.analyze(padded, w=w, conn=conn)
            fm, ff, fp = orc.fill(ref, 8)
            assert st == 0 and n == ref["n"]
            np.testing.assert_array_equal(out.fg.cpu().numpy(), ref["fg"])
            np.testing.assert_array_equal(out.bg.cpu().numpy(), ref["bg"])
            np.testing.assert_array_equal(out.parent[:n].cpu().numpy(), ref["parent"])
            np.testing.assert_array_equal(out.features[:, :n].cpu().numpy(), ref["feat"])
            np.testing.assert_array_equal(out.fill_map[:n].cpu().numpy(), fm)
            np.testing.assert_array_equal(out.filled_features[:, :n].cpu().numpy(), ff)
            ctx.close()


@pytest.mark.gpu
def test_batched_tile_height_16_matches_32():
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2006_09299_gb300 import ccl

    batch = inputs.uneven_batch(seed=8, n=12, lo=20, hi=1500)
    imgs = [(torch.from_numpy(p).cuda(), w) for p, w in batch]
    tot = sum(p.shape[0] * w for p, w in batch)
    res = {}
    for rows in (32, 16):
        bctx = ccl.BatchContext(len(batch), tot, 1500)
        bctx.set_tile_rows(rows)
        res[rows] = bctx.analyze(imgs)
        torch.cuda.synchronize()
        bctx.close()
    for a, b in zip(res[32], res[16]):
        n = a.n
        assert n == b.n and a.status() == 0 and b.status() == 0
        assert torch.equal(a.fg, b.fg) and torch.equal(a.bg, b.bg)
        assert torch.equal(a.parent[:n], b.parent[:n]) and torch.equal(a.features[:, :n], b.features[:, :n])
