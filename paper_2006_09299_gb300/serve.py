"""Continuous-batching serving loop for connected component analysis.

Frames (uint8 host arrays of mixed sizes) arrive one by one. The server
  - admits a waiting frame when a resident slot of its size class is free,
    or when the device-memory budget allows a new one (label images, tree,
    features and the image buffer stay resident per slot and are reused),
    while fewer than max_batch x (n_streams + 1) frames are admitted and
    not yet launched;
  - every tick launches the admitted frames as ONE batched analysis
    (ccl_analyze_batched + ccl_fill_holes_batched) on the next free CUDA
    stream; each stream has its own batched context, so a new tick runs on
    the device while earlier ticks are still in flight;
  - completes a request when its batch's CUDA event has fired: its results
    are the slot's device tensors, and latency = completion - arrival. They
    stay valid until the client releases the request: the slot is then
    reused (or freed when memory is needed for another size class), and the
    request drops its reference to them;
  - if a scheduler pass fails (an allocation or a launch raises), every
    request not yet completed is completed with status "failed", the error
    is kept in Server.error, and later submissions raise.

The scheduling logic (admission, batching, stream rotation, completion) is
plain Python over a backend object; GpuBackend drives the CUDA library, and
tests substitute a fake backend to check the host logic without a GPU.
"""
import collections
import math
import threading
import time

import numpy as np


class Request:
    __slots__ = ("rid", "frame", "pixels", "t_arrive", "t_admit", "t_launch", "t_done", "slot", "done",
                 "cancelled", "result", "status")

    def __init__(self, rid, frame, t_arrive):
        self.rid = rid
        self.frame = frame              # dropped once the frame is staged into its slot
        self.pixels = int(frame.size)
        self.t_arrive = t_arrive
        self.t_admit = self.t_launch = self.t_done = None
        self.slot = None
        self.done = threading.Event()
        self.cancelled = False
        self.result = None
        self.status = None

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_arrive


class Slot:
    """Resident buffers for one frame of a size class (allocated by the backend)."""

    def __init__(self, key, nbytes, handle):
        self.key = key
        self.nbytes = nbytes
        self.handle = handle


class Server:
    def __init__(self, backend, memory_budget, max_batch=16, n_streams=2, fill_threshold=64):
        self.backend = backend
        self.budget = int(memory_budget)
        self.max_batch = int(max_batch)
        self.n_streams = int(n_streams)
        self.fill_threshold = fill_threshold
        self.used = 0
        self.free_slots = collections.defaultdict(list)   # size key -> [Slot]
        self.waiting = collections.deque()
        self.admitted = collections.deque()
        self.inflight = []                                 # (stream, handle, [Request])
        self.stream_busy = [False] * self.n_streams
        self.next_stream = 0
        self.launch_failed = []                            # requests of a launch that raised
        self.lock = threading.Lock()
        self.wake = threading.Event()
        self._stop = False
        self._thread = None
        self._rid = 0
        self.ticks = 0
        self.error = None

    # ------------------------------------------------------------ clients
    def submit(self, frame, t_arrive=None):
        with self.lock:
            if self.error is not None:
                raise RuntimeError("the serving scheduler failed: %r" % (self.error,))
            r = Request(self._rid, frame, time.perf_counter() if t_arrive is None else t_arrive)
            self._rid += 1
            self.waiting.append(r)
        self.wake.set()
        return r

    def cancel(self, req):
        """Cancel a request that has not been launched yet."""
        with self.lock:
            if req.t_launch is None and not req.done.is_set():
                req.cancelled = True
                try:
                    self.waiting.remove(req)
                except ValueError:
                    try:
                        self.admitted.remove(req)
                    except ValueError:
                        pass
                    self._release(req)
                req.done.set()
                return True
        return False

    # ---------------------------------------------------------- scheduling
    def _release(self, req):
        if req.slot is not None:
            self.free_slots[req.slot.key].append(req.slot)
            req.slot = None

    def _admit(self):
        # no more admitted than the streams can take plus one batch: under a
        # burst the rest waits unadmitted, instead of tying up (or allocating)
        # slots for frames that cannot launch yet
        while self.waiting and len(self.admitted) < self.max_batch * (self.n_streams + 1):
            r = self.waiting[0]
            key = self.backend.size_key(r.frame)
            if self.free_slots[key]:
                r.slot = self.free_slots[key].pop()
            else:
                need = self.backend.slot_bytes(key)
                if self.used + need > self.budget:
                    if self._evict_for(need):
                        continue
                    break            # wait for memory: frames are admitted in arrival order
                r.slot = self.backend.alloc_slot(key)
                self.used += r.slot.nbytes
            r.t_admit = time.perf_counter()
            self.waiting.popleft()
            self.admitted.append(r)

    def preallocate(self, keys, per_key):
        """Allocate up to `per_key` idle slots for each size key (within the
        memory budget), so that bursts are not slowed by allocation."""
        with self.lock:
            for key in keys:
                while len(self.free_slots[key]) < per_key:
                    need = self.backend.slot_bytes(key)
                    if self.used + need > self.budget:
                        break
                    self.free_slots[key].append(self.backend.alloc_slot(key))
                    self.used += need

    def _evict_for(self, need):
        """Free idle slots of other size classes until `need` bytes fit."""
        freed = False
        for key in list(self.free_slots):
            while self.free_slots[key] and self.used + need > self.budget:
                s = self.free_slots[key].pop()
                self.backend.free_slot(s)
                self.used -= s.nbytes
                freed = True
        return freed and self.used + need <= self.budget

    def _launch(self):
        while self.admitted:
            k = None
            for j in range(self.n_streams):
                c = (self.next_stream + j) % self.n_streams
                if not self.stream_busy[c]:
                    k = c
                    break
            if k is None:
                return
            batch = []
            while self.admitted and len(batch) < self.max_batch:
                batch.append(self.admitted.popleft())
            now = time.perf_counter()
            for r in batch:
                r.t_launch = now
            try:
                handle = self.backend.launch(k, batch, self.fill_threshold)
            except Exception:
                # copies of this batch may already be queued on the device:
                # its requests are failed with the in-flight ones
                self.launch_failed.extend(batch)
                raise
            for r in batch:
                r.frame = None      # staged: the server keeps no host frame alive
            self.stream_busy[k] = True
            self.inflight.append((k, handle, batch))
            self.next_stream = (k + 1) % self.n_streams
            self.ticks += 1

    def _complete(self):
        still = []
        for k, handle, batch in self.inflight:
            if self.backend.done(handle):
                now = time.perf_counter()
                results = self.backend.results(handle, batch)
                for r, res in zip(batch, results):
                    r.result, r.status = res
                    r.t_done = now
                    r.done.set()
                self.stream_busy[k] = False
                self.backend.retire(handle)
            else:
                still.append((k, handle, batch))
        self.inflight = still

    def release(self, req):
        """Give a finished request's slot back: its result tensors are reused,
        so the request drops them (an evicted slot's memory is then freed)."""
        with self.lock:
            self._release(req)
            req.result = None
        self.wake.set()

    def _fail(self, err):
        """A scheduler pass raised: complete every pending request as failed.
        Requests whose batch may still run on the device lose their slot
        outright (it is never handed back to the pool, since kernels may
        still write to it); waiting and admitted requests give theirs back."""
        with self.lock:
            self.error = err
            launched = [r for _, _, b in self.inflight for r in b] + self.launch_failed
            self.launch_failed = []
            for r in launched:
                r.slot = None
            pending = list(self.waiting) + list(self.admitted) + launched
            for r in self.admitted:
                self._release(r)
            self.waiting.clear()
            self.admitted.clear()
            self.inflight = []
            for r in pending:
                r.status = "failed"
                r.done.set()

    def step(self):
        """One scheduler pass: completions, admission, launches."""
        with self.lock:
            self._complete()
            self._admit()
            self._launch()
            return bool(self.waiting or self.admitted or self.inflight)

    # --------------------------------------------------------------- loop
    def start(self, poll_s=20e-6, switch_interval=2e-4):
        # the scheduler shares the interpreter with the clients: a short GIL
        # switch interval keeps its reaction time well under a millisecond
        import sys
        self._old_switch = sys.getswitchinterval()
        sys.setswitchinterval(switch_interval)

        def loop():
            try:
                while not self._stop:
                    busy = self.step()
                    if not busy:
                        self.wake.wait(0.002)
                        self.wake.clear()
                    else:
                        time.sleep(poll_s)
            except Exception as e:   # reported through Server.error and the requests
                self._fail(e)
        self._thread = threading.Thread(target=loop, daemon=True)
        self._thread.start()

    def stop(self):
        self._stop = True
        self.wake.set()
        if self._thread is not None:
            self._thread.join()
            import sys
            sys.setswitchinterval(self._old_switch)

    def queue_depth(self):
        with self.lock:
            return len(self.waiting) + len(self.admitted)


# ----------------------------------------------------------------- backend


class GpuBackend:
    """Runs batches through the CUDA library on n_streams streams."""

    def __init__(self, n_streams=2, max_batch=16, max_side=3840, max_frame_px=3840 * 2160, device=0,
                 capacity_fraction=16, stage_threads=4):
        import torch
        from . import ccl
        self.torch = torch
        self.ccl = ccl
        self.dev = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(n_streams)]
        # batch compositions vary from tick to tick: plain launches, no graph cache
        self.ctxs = [ccl.BatchContext(max_batch, max_batch * max_frame_px, max_side, graph_cache=False)
                     for _ in range(n_streams)]
        self.capacity_fraction = capacity_fraction
        # frames are staged into their slots' pinned buffers by a few host
        # threads (numpy copies release the interpreter lock), so the
        # scheduler thread is not limited to one core's copy bandwidth;
        # frames the client registered as pinned are copied to the device
        # directly, without staging. Every launch is one library call that
        # copies the batch's frames and analyses them, from descriptors kept
        # per slot (the scheduler thread does little per frame)
        import concurrent.futures
        self.stager = concurrent.futures.ThreadPoolExecutor(max_workers=stage_threads)
        self.pinned = {}   # data pointer -> (registered host tensor, nbytes)

    def register_frames(self, frames):
        """Pin the memory of the client's frame arrays in place (a frame pool
        that decoders write into); submitted frames that lie in it skip the
        staging copy. Call unregister_frames before the arrays are freed."""
        torch = self.torch
        for f in frames:
            ptr, n = f.__array_interface__["data"][0], f.nbytes
            if ptr in self.pinned or not f.flags["C_CONTIGUOUS"]:
                continue
            err = torch.cuda.cudart().cudaHostRegister(ptr, n, 0)
            if int(err) != 0:
                raise RuntimeError("cudaHostRegister failed (%s)" % (err,))
            self.pinned[ptr] = (f, n)

    def unregister_frames(self):
        torch = self.torch
        torch.cuda.synchronize()
        for ptr in list(self.pinned):
            torch.cuda.cudart().cudaHostUnregister(ptr)
        self.pinned.clear()

    def _direct(self, frame):
        """The frame lies in registered memory (rows w bytes apart)."""
        return frame.__array_interface__["data"][0] in self.pinned and frame.flags["C_CONTIGUOUS"]

    @staticmethod
    def size_key(frame):
        return frame.shape

    def _cap(self, key):
        h, w = key
        return min(self.ccl.node_capacity(w, h), max(4096, (w * h) // self.capacity_fraction))

    def slot_bytes(self, key):
        h, w = key
        pitch = -(-w // 16) * 16
        cap = self._cap(key)
        return h * pitch + 8 * h * w + cap * (4 + 56 + 4 + 56 + 4) + 16

    def alloc_slot(self, key):
        torch = self.torch
        h, w = key
        pitch = -(-w // 16) * 16
        img = torch.empty((h, pitch), dtype=torch.uint8, device=self.dev)
        out = self.ccl.Analysis(w, h, self._cap(key), True, self.dev).alloc_fill()
        desc = self.ccl.BatchContext.image_desc(img, w, out)
        # [device image, outputs, pinned staging buffer (allocated on first
        # use: frames from the registered pool never need it), width, descriptor]
        return Slot(key, self.slot_bytes(key), [img, out, None, w, desc])

    def free_slot(self, slot):
        slot.handle = None

    def launch(self, k, batch, fill_threshold):
        torch = self.torch
        st = self.streams[k]
        direct = [self._direct(r.frame) for r in batch]

        def stage(r):
            hd = r.slot.handle
            if hd[2] is None:
                hd[2] = torch.empty(tuple(hd[0].shape), dtype=torch.uint8).pin_memory()
            hd[2].numpy()[:, :hd[3]] = r.frame
        staged = [r for r, dr in zip(batch, direct) if not dr]
        if len(staged) >= 4:
            list(self.stager.map(stage, staged))
        else:
            for r in staged:
                stage(r)
        n = len(batch)
        descs = (self.ccl.ImageDesc * n)()
        frames, pitches = [0] * n, [0] * n
        for i, (r, dr) in enumerate(zip(batch, direct)):
            img, out, host, w, desc = r.slot.handle
            descs[i] = desc
            if dr:
                frames[i], pitches[i] = r.frame.__array_interface__["data"][0], r.frame.strides[0]
            else:
                frames[i], pitches[i] = host.data_ptr(), host.stride(0)
        self.ctxs[k].analyze_from_host(descs, frames, pitches, stream=st)
        self.ctxs[k].fill_holes(fill_threshold, stream=st)
        ev = torch.cuda.Event()
        ev.record(st)
        return ev

    def done(self, handle):
        return handle.query()

    def results(self, handle, batch):
        return [(r.slot.handle[1], None) for r in batch]

    def retire(self, handle):
        pass


# ----------------------------------------------------------------- driver


def poisson_run(server, frames, rate_hz, duration_s, seed=0, release=True, drain_s=30.0, depth_samples=False):
    """Submit frames (cycled) with Poisson arrivals at rate_hz for duration_s;
    wait (at most drain_s in all) for the admitted work to finish. Returns the
    requests and the queue depth seen at the end of the arrival window (and,
    with depth_samples, the queue depth sampled at every arrival); raises if
    the scheduler failed."""
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    t_next = t0
    reqs = []
    samples = []
    unreleased = collections.deque()
    i = 0
    while True:
        t_next += rng.exponential(1.0 / rate_hz)
        if t_next - t0 > duration_s:
            break
        wait = t_next - time.perf_counter()
        if wait > 0:
            time.sleep(wait)          # releases the interpreter to the scheduler
        if server.error is not None:
            raise RuntimeError("the serving scheduler failed") from server.error
        reqs.append(server.submit(frames[i % len(frames)], t_arrive=t_next))
        unreleased.append(reqs[-1])
        if depth_samples:
            samples.append(len(server.waiting) + len(server.admitted))
        i += 1
        # hand back the slots of finished requests (their results were
        # consumed), oldest first: requests finish roughly in arrival order
        if release:
            while unreleased and unreleased[0].done.is_set():
                r = unreleased.popleft()
                if r.slot is not None:
                    server.release(r)
    depth_end = server.queue_depth()
    deadline = time.perf_counter() + drain_s
    for r in reqs:
        r.done.wait(max(0.0, deadline - time.perf_counter()))
        if release and r.slot is not None and r.done.is_set():
            server.release(r)
    if server.error is not None:
        raise RuntimeError("the serving scheduler failed") from server.error
    return (reqs, depth_end, samples) if depth_samples else (reqs, depth_end)


def latency_stats(reqs):
    lat = sorted(r.latency for r in reqs if r.latency is not None)
    if not lat:
        return {"p50_ms": None, "p99_ms": None, "n": 0}
    def q(p):
        return lat[min(len(lat) - 1, int(math.ceil(p * len(lat))) - 1)] * 1e3
    return {"p50_ms": round(q(0.50), 3), "p99_ms": round(q(0.99), 3), "n": len(lat)}
