"""Serving loop: host logic with a fake backend (CPU), and results alone vs
in a mix on the GPU."""
import time

import numpy as np
import pytest

from paper_2006_09299_gb300 import inputs
from paper_2006_09299_gb300.serve import Server, Slot, latency_stats, poisson_run


class FakeBackend:
    """Completes each batch `delay` seconds after launch; records launches."""

    def __init__(self, delay=0.002, nbytes=100):
        self.delay = delay
        self.nbytes = nbytes
        self.launches = []
        self.alloc = 0
        self.freed = 0

    def size_key(self, frame):
        return frame.shape

    def slot_bytes(self, key):
        return self.nbytes * key[0] * key[1]

    def alloc_slot(self, key):
        self.alloc += 1
        return Slot(key, self.slot_bytes(key), object())

    def free_slot(self, slot):
        self.freed += 1

    def launch(self, k, batch, T):
        self.launches.append((k, [r.rid for r in batch]))
        return time.perf_counter() + self.delay

    def done(self, handle):
        return time.perf_counter() >= handle

    def results(self, handle, batch):
        return [("res%d" % r.rid, 0) for r in batch]

    def retire(self, handle):
        pass


def drain(s, limit=5.0):
    t = time.perf_counter()
    while s.step() and time.perf_counter() - t < limit:
        time.sleep(0.0005)


def test_batches_respect_max_batch_and_streams():
    be = FakeBackend(delay=0.01)
    s = Server(be, memory_budget=10**9, max_batch=4, n_streams=2)
    reqs = [s.submit(np.zeros((2, 3), np.uint8)) for _ in range(10)]
    s.step()
    # two streams busy, 4 + 4 launched, 2 still admitted
    assert [len(b) for _, b in be.launches] == [4, 4]
    assert {k for k, _ in be.launches} == {0, 1}
    drain(s)
    assert all(r.done.is_set() and r.result == "res%d" % r.rid for r in reqs)
    assert sorted(rid for _, b in be.launches for rid in b) == list(range(10))


def test_a_burst_admits_at_most_one_batch_beyond_the_streams():
    """Frames beyond what the streams can take plus one batch wait
    unadmitted: a burst does not allocate a slot for every waiting frame."""
    be = FakeBackend(delay=0.05)
    s = Server(be, memory_budget=10**9, max_batch=2, n_streams=1)
    reqs = [s.submit(np.zeros((2, 3), np.uint8)) for _ in range(20)]
    s.step()
    assert len(be.launches) == 1 and len(be.launches[0][1]) == 2
    assert len(s.admitted) == 2 and len(s.waiting) == 16
    assert be.alloc == 4          # slots for the launched batch and the next one only
    released = set()
    t = time.perf_counter()
    while time.perf_counter() - t < 5.0:
        busy = s.step()
        for r in reqs:
            if r.done.is_set() and r.rid not in released:
                s.release(r)      # the client is done with the results: the slot goes back
                released.add(r.rid)
        if not busy and len(released) == len(reqs):
            break
        time.sleep(0.0005)
    assert all(r.done.is_set() for r in reqs)
    assert sorted(rid for _, b in be.launches for rid in b) == list(range(20))
    assert be.alloc <= 6          # released slots are reused, not allocated per frame


def test_continuous_batching_admits_while_in_flight():
    be = FakeBackend(delay=0.02)
    s = Server(be, memory_budget=10**9, max_batch=8, n_streams=2)
    a = [s.submit(np.zeros((4, 4), np.uint8)) for _ in range(3)]
    s.step()
    b = [s.submit(np.zeros((4, 4), np.uint8)) for _ in range(3)]
    s.step()   # second stream takes the new arrivals while the first batch runs
    assert len(be.launches) == 2 and be.launches[1][1] == [r.rid for r in b]
    drain(s)
    assert all(r.done.is_set() for r in a + b)
    assert max(r.t_launch for r in b) < min(r.t_done for r in a)   # overlapped


def test_memory_budget_admission_and_slot_reuse():
    be = FakeBackend(delay=0.001, nbytes=1)
    s = Server(be, memory_budget=2 * 100, max_batch=8, n_streams=1)   # room for two 10x10 slots
    reqs = [s.submit(np.zeros((10, 10), np.uint8)) for _ in range(6)]
    s.step()
    assert len(s.admitted) + sum(len(b) for _, _, b in s.inflight) == 2
    assert s.used <= s.budget
    for _ in range(200):
        s.step()
        for r in reqs:
            if r.done.is_set() and r.slot is not None:
                s.release(r)
        if all(r.done.is_set() for r in reqs):
            break
        time.sleep(0.001)
    assert all(r.done.is_set() for r in reqs)
    assert be.alloc == 2          # slots reused, never more than the budget allows
    # a larger size class evicts idle slots to fit
    big = s.submit(np.zeros((14, 14), np.uint8))
    drain(s)
    assert big.done.is_set() and be.freed >= 1 and s.used <= s.budget


def test_cancel_before_launch():
    be = FakeBackend(delay=0.05)
    s = Server(be, memory_budget=10**9, max_batch=1, n_streams=1)
    r1 = s.submit(np.zeros((2, 2), np.uint8))
    s.step()
    r2 = s.submit(np.zeros((2, 2), np.uint8))
    assert s.cancel(r2) and r2.cancelled and r2.done.is_set()
    assert not s.cancel(r1)       # already launched
    drain(s)
    assert [rid for _, b in be.launches for rid in b] == [r1.rid]


def test_poisson_driver_samples_the_queue_depth():
    be = FakeBackend(delay=0.001)
    s = Server(be, memory_budget=10**9, max_batch=8, n_streams=2)
    s.start()
    try:
        reqs, depth, samples = poisson_run(s, [np.zeros((3, 3), np.uint8)], rate_hz=1000, duration_s=0.2,
                                           depth_samples=True)
    finally:
        s.stop()
    assert len(samples) == len(reqs) > 50 and min(samples) >= 0 and depth >= 0
    assert sorted(samples)[int(0.95 * (len(samples) - 1))] <= 4 * 8   # a fast backend keeps the queue short


def test_poisson_driver_and_latency_stats():
    be = FakeBackend(delay=0.001)
    s = Server(be, memory_budget=10**9, max_batch=8, n_streams=2)
    s.start()
    try:
        reqs, depth = poisson_run(s, [np.zeros((3, 3), np.uint8)], rate_hz=2000, duration_s=0.2)
    finally:
        s.stop()
    st = latency_stats(reqs)
    assert st["n"] == len(reqs) > 100
    assert 0 < st["p50_ms"] <= st["p99_ms"]


@pytest.mark.gpu
def test_results_alone_and_in_the_mix_are_identical():
    import torch

    import __graft_entry__ as g
    g.build()
    from paper_2006_09299_gb300 import ccl
    from paper_2006_09299_gb300.serve import GpuBackend

    frames = inputs.frame_stream(seed=5, n=12)
    be = GpuBackend(n_streams=2, max_batch=4)
    s = Server(be, memory_budget=8 << 30, max_batch=4, n_streams=2)
    s.start()
    try:
        reqs = [s.submit(f) for f in frames]
        for r in reqs:
            assert r.done.wait(60)
    finally:
        s.stop()
    torch.cuda.synchronize()
    for f, r in zip(frames, reqs):
        h, w = f.shape
        pitch = -(-w // 16) * 16
        ctx = ccl.Context(w, h, pitch)
        alone = ctx.analyze(torch.from_numpy(inputs.pitched(f, pitch, 0)).cuda())
        n, _, _, st = ctx.get_counts()
        mix = r.result
        assert st == 0 and mix.status() == 0
        assert mix.n == n
        assert torch.equal(mix.fg, alone.fg) and torch.equal(mix.bg, alone.bg)
        assert torch.equal(mix.parent[:n], alone.parent[:n])
        assert torch.equal(mix.features[:, :n], alone.features[:, :n])
        ctx.close()
    # and the mix is the oracle's result, hole filling included
    from oracle import reference as orc
    for f, r in list(zip(frames, reqs))[:4]:
        ref = orc.analyze(f, w=f.shape[1])
        mix = r.result
        n = mix.n
        assert n == ref["n"]
        np.testing.assert_array_equal(mix.fg.cpu().numpy(), ref["fg"])
        np.testing.assert_array_equal(mix.bg.cpu().numpy(), ref["bg"])
        np.testing.assert_array_equal(mix.parent[:n].cpu().numpy(), ref["parent"])
        np.testing.assert_array_equal(mix.features[:, :n].cpu().numpy(), ref["feat"])
        fmap, ff, fpar = orc.fill(ref, s.fill_threshold)
        np.testing.assert_array_equal(mix.fill_map[:n].cpu().numpy(), fmap)
        np.testing.assert_array_equal(mix.filled_features[:, :n].cpu().numpy(), ff)
        np.testing.assert_array_equal(mix.filled_parent[:n].cpu().numpy(), fpar)


def test_preallocate_respects_budget_and_is_reused():
    be = FakeBackend(nbytes=100)
    s = Server(be, memory_budget=100 * 10 * 10 * 5, max_batch=4, n_streams=2)
    s.preallocate([(10, 10), (20, 20)], per_key=3)
    # 3 slots of 10x10 (10000 bytes each) fit; a 20x20 slot (40000) does not
    # fit in the 20000 bytes left of the 50000 budget
    assert len(s.free_slots[(10, 10)]) == 3
    assert len(s.free_slots[(20, 20)]) == 0
    assert s.used == 30000 <= s.budget
    allocated = be.alloc
    r = s.submit(np.zeros((10, 10), np.uint8))
    s.step()
    assert r.slot is not None and be.alloc == allocated   # an idle slot was reused


def test_release_drops_the_result_so_evicted_slots_are_freed():
    be = FakeBackend(delay=0.0)
    s = Server(be, memory_budget=10**9, max_batch=4, n_streams=1)
    r = s.submit(np.zeros((2, 2), np.uint8))
    drain(s)
    assert r.done.is_set() and r.result == "res%d" % r.rid
    s.release(r)
    # the slot's tensors are reused from here on: the request holds none of them
    assert r.slot is None and r.result is None
    assert len(s.free_slots[(2, 2)]) == 1


def test_the_server_keeps_no_host_frame_alive():
    import gc
    import weakref
    be = FakeBackend(delay=0.0)
    s = Server(be, memory_budget=10**9, max_batch=4, n_streams=2)
    refs, reqs = [], []
    for k in range(64):
        f = np.full((8, 8 + k % 3), k, np.uint8)   # a fresh host array per request
        refs.append(weakref.ref(f))
        reqs.append(s.submit(f))
        del f
        s.step()
    drain(s)
    for r in reqs:
        assert r.done.is_set() and r.pixels == 8 * r.slot.key[1]
        s.release(r)
    gc.collect()
    assert all(ref() is None for ref in refs)        # every frame was freed


class SlowFailingBackend(FakeBackend):
    """Launches two batches that stay on the device, then fails."""

    def launch(self, k, batch, T):
        if len(self.launches) >= 2:
            raise MemoryError("device allocation failed")
        return super().launch(k, batch, T)


def test_a_failure_never_returns_slots_of_batches_still_on_the_device():
    be = SlowFailingBackend(delay=10.0)
    s = Server(be, memory_budget=10**9, max_batch=1, n_streams=3)
    reqs = [s.submit(np.zeros((2, 2), np.uint8)) for _ in range(4)]
    with pytest.raises(MemoryError):
        s.step()
    s._fail(MemoryError("device allocation failed"))
    assert len(be.launches) == 2 and sum(r.t_launch is not None for r in reqs) == 3
    for r in reqs:
        assert r.done.is_set() and r.status == "failed"
        s.release(r)
    # the slots of the two running batches and of the launch that raised
    # (its copies may be queued) are not in the pool; the admitted one is
    assert len(s.free_slots[(2, 2)]) == be.alloc - 3


class FailingBackend(FakeBackend):
    """Raises on its n-th launch, as an out-of-memory allocation would."""

    def __init__(self, fail_at, **kw):
        super().__init__(**kw)
        self.fail_at = fail_at

    def launch(self, k, batch, T):
        if len(self.launches) + 1 >= self.fail_at:
            raise MemoryError("device allocation failed")
        return super().launch(k, batch, T)


def test_a_failed_scheduler_pass_fails_pending_requests_and_the_driver():
    be = FailingBackend(fail_at=3, delay=0.001)
    s = Server(be, memory_budget=10**9, max_batch=2, n_streams=2)
    s.start()
    t0 = time.perf_counter()
    try:
        with pytest.raises(RuntimeError):
            poisson_run(s, [np.zeros((3, 3), np.uint8)], rate_hz=2000, duration_s=0.3, drain_s=5.0)
    finally:
        s.stop()
    assert time.perf_counter() - t0 < 5.0            # no request is waited on after the failure
    assert isinstance(s.error, MemoryError)
    with pytest.raises(RuntimeError):
        s.submit(np.zeros((3, 3), np.uint8))


def test_the_driver_waits_a_bounded_time_for_unfinished_work():
    be = FakeBackend(delay=10.0)                      # batches that never finish in time
    s = Server(be, memory_budget=10**9, max_batch=4, n_streams=1)
    s.start()
    t0 = time.perf_counter()
    try:
        reqs, _ = poisson_run(s, [np.zeros((3, 3), np.uint8)], rate_hz=500, duration_s=0.1, drain_s=0.5)
    finally:
        s.stop()
    assert time.perf_counter() - t0 < 3.0
    assert any(not r.done.is_set() for r in reqs)
