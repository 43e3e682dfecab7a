"""Serving loop for encrypted Softmax requests: continuous batching on one GPU.

A request is a client's encrypted Softmax input: n_ct ciphertexts packed for one plan (Softmax
dimension n, range M) as in Sec. 4.2, at the fresh level and scale of that plan.  The server
keeps the evaluation keys resident (they live in the context), admits waiting requests in
arrival order while the HBM budget allows, and runs every admitted request of the same shape
(plan, n_ct, level, scale) as one batched pass (`he_softmax_grouped`: each request is its own
group, so its result is the one it would get alone, bit for bit).  Requests that arrive while
a batch runs are admitted as memory frees up and join the next batch; their uploads (host to
device, on a copy stream) overlap the running batch, and the previous batch's downloads do too.

With several contexts (the same keys in each), every context is a lane with its own worker
thread and streams, and batches of different shapes run concurrently on the device.

`BatchPolicy` is the host-only admission and batching rule (tested without a GPU); `Server`
drives the GPU through the C ABI.
"""
from __future__ import annotations

import collections
import itertools
import threading
import time


class Request:
    """One encrypted Softmax request (host buffers; results are written into host_out)."""

    _ids = itertools.count(1)   # next() on a count is atomic: submit() may run on many threads

    def __init__(self, plan, n_ct, level, scale, host_in, host_out, words):
        self.rid = next(Request._ids)
        self.plan = plan            # plan name
        self.n_ct = n_ct
        self.level = level
        self.scale = scale
        self.host_in = host_in      # pinned int64 tensor [n_ct * 2 * (level + 1) * N]
        self.host_out = host_out    # pinned int64 tensor, same size (the output is at a lower level)
        self.words = words          # device words of the input ciphertexts
        self.t_submit = time.perf_counter()
        self.t_done = None
        self.out_level = None
        self.out_scale = None
        self.error = None
        self.done = threading.Event()

    def key(self):
        return (self.plan, self.n_ct, self.level, self.scale)

    def wait(self, timeout=None):
        if not self.done.wait(timeout):
            raise TimeoutError("request %d not finished" % self.rid)
        if self.error:
            raise RuntimeError(self.error)
        return self

    @property
    def latency_ms(self):
        return None if self.t_done is None else (self.t_done - self.t_submit) * 1e3


class BatchPolicy:
    """Admission by HBM budget and same-shape batching (no GPU needed).

    budget_bytes: device bytes the server may hold for requests (keys are outside it);
    work_factor: device bytes a request holds while its batch runs, per byte of its input
    ciphertexts (inputs, outputs and the circuit's temporaries: key-switch digits, tensors,
    bootstrapping intermediates); max_batch_ct: ciphertexts per batched pass."""

    def __init__(self, budget_bytes, max_batch_ct=64, work_factor=8.0):
        self.budget = float(budget_bytes)
        self.max_batch_ct = int(max_batch_ct)
        self.work_factor = float(work_factor)
        self.in_use = 0.0

    def cost(self, req):
        return req.words * 8.0 * self.work_factor

    def fits_ever(self, req):
        return self.cost(req) <= self.budget and req.n_ct <= self.max_batch_ct

    def admit(self, waiting, admitted):
        """Moves requests from the front of `waiting` (a deque, arrival order) to `admitted` while
        they fit in the budget; a request that can never fit is returned as rejected.  The
        order is kept: a large request at the front is not overtaken."""
        rejected = []
        while waiting:
            r = waiting[0]
            if not self.fits_ever(r):
                rejected.append(waiting.popleft())
                continue
            c = self.cost(r)
            if self.in_use + c > self.budget:
                break
            self.in_use += c
            admitted.append(waiting.popleft())
        return rejected

    def next_batch(self, admitted):
        """The oldest admitted request's shape, and every admitted request of that shape in
        arrival order up to max_batch_ct ciphertexts (removed from `admitted`)."""
        if not admitted:
            return []
        k = admitted[0].key()
        batch, rest, nct = [], [], 0
        for r in admitted:
            if r.key() == k and nct + r.n_ct <= self.max_batch_ct:
                batch.append(r)
                nct += r.n_ct
            else:
                rest.append(r)
        admitted[:] = rest
        return batch

    def release(self, batch):
        for r in batch:
            self.in_use -= self.cost(r)
        if self.in_use < 1e-6:
            self.in_use = 0.0


def percentile(xs, p):
    """Nearest-rank percentile (p in [0, 100]) of a non-empty list."""
    s = sorted(xs)
    k = max(0, min(len(s) - 1, int(-(-p * len(s) // 100)) - 1))
    return s[k]


class _Lane:
    """One context with its upload and download streams, its batches in flight and the worker
    thread that issues them (the only thread that uses this context while the server runs)."""

    def __init__(self, server, ctx):
        torch = server.torch
        self.g = ctx
        # uploads and downloads on separate streams: the next batch's uploads must not queue
        # behind the running batch's downloads
        self.up_stream = torch.cuda.Stream(device=ctx.device)
        self.down_stream = torch.cuda.Stream(device=ctx.device)
        self.inflight = collections.deque()   # (batch, device buffer, done event)
        self.wake = threading.Event()
        self.thread = threading.Thread(target=server._loop, args=(self,), daemon=True)


class Server:
    """Continuous batching over one or more contexts on the device (ctx: a context, or a list of
    contexts with the same keys, e.g. made with the same keygen seed).  Every context has its own
    worker thread and stream, so batches of different shapes -- requests of different
    dimensions -- run concurrently on the GPU: while one lane's one-ciphertext circuit leaves SMs
    idle, another lane's fills them.  A batch's result does not depend on the lane that runs it.
    Do not use the contexts from another thread while the server runs.  plans: {name: plan dict}."""

    def __init__(self, ctx, plans, budget_bytes, max_batch_ct=64, work_factor=8.0, max_inflight=2, start=True):
        import torch

        self.torch = torch
        ctxs = list(ctx) if isinstance(ctx, (list, tuple)) else [ctx]
        self.g = ctxs[0]
        self.plans = plans
        self.policy = BatchPolicy(budget_bytes, max_batch_ct, work_factor)
        self.max_inflight = max_inflight
        self.lock = threading.Lock()   # guards the queues, the policy and the result lists
        self.arrivals = collections.deque()
        self.waiting = collections.deque()
        self.admitted = []
        self.finished = []
        self.batches = []                      # sizes (requests, ciphertexts) of the batches run
        self.running = True
        self.lanes = [_Lane(self, c) for c in ctxs]
        self.started = False
        if start:
            self.start()

    def start(self):
        """Starts the workers (for a server created with start=False: requests submitted before
        are then admitted together)."""
        if not self.started:
            self.started = True
            for ln in self.lanes:
                ln.thread.start()

    def _wake_all(self):
        for ln in self.lanes:
            ln.wake.set()

    # ---- client side
    def submit(self, plan, host_in, n_ct, level, scale):
        """Queues a request; host_in: pinned int64 CPU tensor of the request's ciphertexts
        ([n_ct][2][level+1][N] words, NTT form).  Returns the Request (wait() for it)."""
        torch = self.torch
        words = n_ct * 2 * (level + 1) * self.g.n
        if host_in.numel() != words:
            raise ValueError("host_in holds %d words, the request needs %d" % (host_in.numel(), words))
        host_out = torch.empty(words, dtype=torch.int64).pin_memory()
        r = Request(plan, n_ct, level, scale, host_in, host_out, words)
        with self.lock:
            self.arrivals.append(r)
        self._wake_all()
        return r

    def close(self):
        """Finishes every submitted request, then stops the workers."""
        self.start()
        self.running = False
        self._wake_all()
        for ln in self.lanes:
            ln.thread.join()

    def stats(self):
        lat = [r.latency_ms for r in self.finished if r.error is None]
        if not lat:
            return {"requests": 0}
        span = max(r.t_done for r in self.finished) - min(r.t_submit for r in self.finished)
        return {"requests": len(lat), "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
                "max_ms": max(lat), "span_s": span, "batches": len(self.batches), "lanes": len(self.lanes),
                "mean_batch_requests": sum(b[0] for b in self.batches) / len(self.batches),
                "mean_batch_ct": sum(b[1] for b in self.batches) / len(self.batches)}

    # ---- workers
    def _loop(self, ln):
        while True:
            # cleared before the arrivals are drained: a submit() after this point sets it again,
            # so the wait below returns at once instead of sleeping through its timeout
            ln.wake.clear()
            with self.lock:
                while self.arrivals:
                    self.waiting.append(self.arrivals.popleft())
                for r in self.policy.admit(self.waiting, self.admitted):
                    self._fail(r, "request larger than the server's HBM budget or batch limit")
                freed = self._retire(ln)
                batch = None
                if self.admitted and len(ln.inflight) < self.max_inflight:
                    batch = self.policy.next_batch(self.admitted)
                idle = not (self.waiting or self.admitted or self.arrivals)
            if freed:
                self._wake_all()   # memory was released: the other lanes may admit more
            if batch:
                self._launch(ln, batch)
                continue
            if not self.running and idle and not ln.inflight:
                return
            ln.wake.wait(0.0002 if ln.inflight else 0.01)

    def _launch(self, ln, batch):
        torch, g = self.torch, ln.g
        r0 = batch[0]
        nct = sum(r.n_ct for r in batch)
        try:
            dev = g.alloc(r0.level, nct, r0.scale)
            # uploads on the upload stream, then the batched circuit on the context stream
            with torch.cuda.stream(ln.up_stream):
                off = 0
                for r in batch:
                    dev.tensor[off:off + r.words].copy_(r.host_in, non_blocking=True)
                    off += r.words
                up = torch.cuda.Event()
                up.record(ln.up_stream)
            g.stream.wait_event(up)
            g.softmax_grouped(dev, self.plans[r0.plan], len(batch))
            fin = torch.cuda.Event()
            fin.record(g.stream)
            # each request's part back to its host buffer once the batch is done
            ln.down_stream.wait_event(fin)
            per = 2 * (dev.level + 1) * g.n
            with torch.cuda.stream(ln.down_stream):
                off = 0
                for r in batch:
                    w = r.n_ct * per
                    r.host_out[:w].copy_(dev.tensor[off:off + w], non_blocking=True)
                    r.out_level, r.out_scale = dev.level, dev.scale
                    off += w
                down = torch.cuda.Event()
                down.record(ln.down_stream)
            ln.inflight.append((batch, dev, down))
            with self.lock:
                self.batches.append((len(batch), nct))
        except Exception as e:  # noqa: BLE001 - reported on every request of the batch
            with self.lock:
                for r in batch:
                    self._fail(r, str(e))
                self.policy.release(batch)

    def _retire(self, ln):
        """(lock held) Finishes the lane's batches whose downloads are done; True if any."""
        freed = False
        while ln.inflight and ln.inflight[0][2].query():
            batch, dev, _ = ln.inflight.popleft()
            t = time.perf_counter()
            for r in batch:
                r.t_done = t
                self.finished.append(r)
                r.done.set()
            self.policy.release(batch)
            del dev
            freed = True
        return freed

    def _fail(self, r, msg):
        """(lock held)"""
        r.error = msg
        r.t_done = time.perf_counter()
        self.finished.append(r)
        r.done.set()
