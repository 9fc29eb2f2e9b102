"""Request serving with continuous batching on one GPU.

Requests ask for samples x ~= Q^{-1/2} z (Algorithm 1; Proposition 1 for the
preconditioned 2-D operator), for log det Q (Section 6) or for linear solves
x = Q^{-1} b (Section 5.1) of a lattice GMRF drawn per request: a 2-D
SPDE-type field (Q = tau (K - Lap)^2, zero-Neumann, mirror-preconditioned) or a
3-D 7-point field (Q = tau (K + L), Dirichlet).

Batched mode (the default).  Samples and log dets of one grid and one
coefficient field share an engine: one problem (tau = 1) with the library's
continuous-batching server (gmrf_server_*), a table of vector slots whose
Lanczos state (bases, alpha/beta) stays resident on the device.  The vectors of
every request of that engine share each launch of the step kernels; a
request's vectors enter free slots as soon as slots free up, also while other
vectors are in mid-iteration, and the request's tau is applied when its
vectors finish.  Each engine is driven by its own host thread on its own CUDA
stream, so the engines' kernels overlap on the device.  Engines are created
when their first request arrives, sized by the memory budget (slots x basis
bytes), and an idle engine is released when a new one needs its memory.
Linear solves (which the server does not run) go through the direct mode.

Direct mode: every request is one call of the library on its own problem and
stream, admitted when its memory fits the budget (max_inflight at once); with
max_inflight = 1, block_width = 1 and FP64 this is the one-request,
one-sample-at-a-time baseline.

Every result depends only on its own request (problem, seed, tolerance): the
library's reductions have a fixed order per vector and the server's results
are bitwise those of the synchronous calls, so a request returns the same bits
alone and in any mix (tests/test_gpu_serve.py).
"""
from __future__ import annotations

import heapq
import threading
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import inputs


@dataclass(order=True)
class Request:
    arrival: float
    rid: int = field(compare=False)
    kind: str = field(compare=False)          # "sample", "logdet" or "solve" (x = Q^{-1} b, Section 5.1)
    shape: tuple = field(compare=False)       # (N, N) 2-D SPDE or (N, N, N) 3-D
    tau: float = field(compare=False, default=1.0)
    count: int = field(compare=False, default=1)   # samples, probes or right-hand sides
    seed: int = field(compare=False, default=0)
    field_id: int = field(compare=False, default=0)
    tol: float = field(compare=False, default=1e-6)


@dataclass
class Result:
    rid: int
    kind: str
    shape: tuple
    count: int
    latency_ms: float
    start_ms: float
    end_ms: float
    m_used: list
    status: int
    x: object = None          # device tensor [count][n] for samples and solves
    logdet: float = None
    std_err: float = None


def make_mix(nreq, rate, seed=4, sizes2d=(128, 256, 512, 1024), sizes3d=(64, 96, 128), nfields=4,
             max_samples=64, probes=(16, 64), p_logdet=0.25, p_solve=0.0):
    """A Poisson request stream (rate requests/s) of the serving mix; a
    fraction p_solve are linear solves with 1 .. max_samples seeded
    right-hand sides (the stream is the same as without solves for p_solve = 0)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(nreq):
        t += rng.exponential(1.0 / rate)
        if rng.random() < 0.5:
            shape = (int(rng.choice(sizes2d)),) * 2
        else:
            shape = (int(rng.choice(sizes3d)),) * 3
        u = rng.random()
        kind = "logdet" if u < p_logdet else ("solve" if u < p_logdet + p_solve else "sample")
        count = int(rng.integers(probes[0], probes[1] + 1)) if kind == "logdet" else int(rng.integers(1, max_samples + 1))
        reqs.append(Request(arrival=t, rid=i, kind=kind, shape=shape, tau=float(rng.uniform(0.5, 5.0)),
                            count=count, seed=int(rng.integers(1, 2 ** 31)), field_id=int(rng.integers(0, nfields))))
    return reqs


class FieldPool:
    """Per-request coefficient fields, generated once per (shape, field id)."""

    def __init__(self, torch):
        self.torch = torch
        self.cache = {}
        self.lock = threading.Lock()

    def get(self, shape, fid):
        key = (shape, fid)
        with self.lock:
            if key not in self.cache:
                if len(shape) == 2:
                    k2 = inputs.kappa2_gp_field(shape, seed=100 + fid, ell=64.0 * shape[0] / 1024)
                else:
                    k2 = inputs.kappa2_uniform_field(shape, seed=100 + fid)
                self.cache[key] = self.torch.from_numpy(k2).cuda()
            return self.cache[key]


class Engine:
    """One grid and field: a problem with tau = 1 and its library server
    (gmrf_server_*), driven by its own host thread and CUDA stream."""

    def __init__(self, owner, key, k2, nslots, m_max):
        torch, g = owner.torch, owner.g
        self.owner, self.key, self.nslots, self.m_max = owner, key, nslots, m_max
        shape = key[0]
        self.n = int(np.prod(shape))
        self.stream = torch.cuda.Stream()
        self.prob = owner._problem(shape, k2, 1.0, self.stream)
        self.server = g.Server(self.prob, nslots=nslots, m_max=m_max, tol=owner.tol, check_every=owner.check_every)
        self.lock = threading.Lock()    # guards `incoming` and `active` (the library server is the loop's alone)
        self.wake = threading.Event()
        self.incoming = []     # (Request, x) handed over by the dispatcher, submitted by the loop
        self.active = {}       # library request id -> (Request, x); the loop's alone
        self.inflight = 0      # requests handed over and not yet completed
        self.last_used = time.perf_counter()
        self.stop = False
        self.error = None
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def busy(self):
        with self.lock:
            return self.inflight > 0

    def submit(self, req):
        """Hands a request to the engine; the engine's loop submits it to the
        library server between two steps, so the dispatcher never waits for a
        step in flight."""
        torch = self.owner.torch
        dt = torch.float64 if self.owner.precision == "fp64" else torch.float32
        x = torch.empty(req.count * self.n, dtype=dt, device="cuda") if req.kind == "sample" else None
        with self.lock:
            self.incoming.append((req, x))
            self.inflight += 1
            self.last_used = time.perf_counter()
        self.wake.set()

    def _loop(self):
        torch = self.owner.torch
        with torch.cuda.stream(self.stream):
            while not self.stop:
                self.wake.wait(timeout=0.05)
                with self.lock:
                    incoming, self.incoming = self.incoming, []
                    if not incoming and not self.active:
                        self.wake.clear()
                        continue
                finished = []
                try:
                    for req, x in incoming:
                        if req.kind == "sample":
                            rid = self.server.submit_sample(x, req.count, req.seed, req.tau)
                        else:
                            rid = self.server.submit_logdet(req.count, req.seed, req.tau)
                        self.active[rid] = (req, x)
                    left = self.server.step()
                    for rid, (req, x) in list(self.active.items()):
                        r = self.server.poll(rid)
                        if r is not None:
                            finished.append((rid, req, x, r))
                            del self.active[rid]
                    with self.lock:
                        self.inflight -= len(finished)
                        if left == 0 and not self.active and not self.incoming:
                            self.wake.clear()
                        self.last_used = time.perf_counter()
                except Exception as e:  # surfaced by the dispatcher
                    self.error = e
                    self.stop = True
                for rid, req, x, (rc, infos, ld, se) in finished:
                    self.owner._complete(req, rc, infos, x, ld, se)

    def close(self):
        self.stop = True
        self.wake.set()
        self.thread.join()
        self.server.close()
        self.prob.close()


class Server:
    """Serving over the C-ABI library: batched engines (continuous batching of
    samples and log dets into shared launches) or direct per-request calls."""

    # Lanczos steps a vector may take: the mirror-preconditioned 2-D mix needs
    # 20-80 at tol 1e-6 and the 3-D mix 30-60 (plus the accuracy check's extra
    # steps), so 128 bounds both and keeps the resident bases small
    M_MAX_2D = 128
    M_MAX_3D = 128

    def __init__(self, mem_budget=None, max_inflight=16, precision="fp32", chunk_bytes=8 << 30, block_width=None,
                 mode="batched", nslots_max=64, check_every=8, tol=1e-6, keep_outputs=True):
        import torch
        from . import gmrf
        self.torch = torch
        self.g = gmrf
        free, _ = torch.cuda.mem_get_info()
        self.budget = int(mem_budget if mem_budget is not None else 0.6 * free)
        self.max_inflight = max_inflight
        self.precision = precision
        self.chunk_bytes = chunk_bytes
        self.fields = FieldPool(torch)
        self.tuning = {}   # grid shape -> block width / z chunk from the library's autotuner (direct mode)
        self.block_width = block_width  # fixed vectors per launch (e.g. 1: one sample at a time)
        self.mode = mode
        self.nslots_max = nslots_max
        self.check_every = check_every
        self.tol = tol
        # keep_outputs False: a completed request's device output is released
        # (its result keeps the step counts, statuses and log dets), as when a
        # server hands each result on and keeps no copy
        self.keep_outputs = keep_outputs
        self.used = 0
        self.cv = threading.Condition()
        self.engines = {}  # (shape, field id) -> Engine
        self.engines_created = 0
        self.engines_released = 0
        self.plan = {}     # (shape, field id) -> slots, from prepare(): every engine of the stream fits at once

    def _m_max(self, req_or_shape):
        shape = req_or_shape.shape if hasattr(req_or_shape, "shape") else req_or_shape
        return self.M_MAX_2D if len(shape) == 2 else self.M_MAX_3D

    # ---- memory model
    def vec_bytes(self, req):
        """Device bytes one vector of this request needs inside the library."""
        return self._slot_bytes(req.shape, 2 if req.kind == "logdet" and self.mode == "direct" else None)

    def _slot_bytes(self, shape, slots=None):
        n = int(np.prod(shape))
        es = 8 if self.precision == "fp64" else 4
        m = self._m_max(shape)
        slots = m + 1 if slots is None else slots
        b = (slots + 6) * n * es + 2 * m * 384 * 8 + 64 * m
        if len(shape) == 2:
            b += 3 * n * es + 2 * shape[0] * es   # spectrum, g, w workspaces
        return b

    def chunk(self, req):
        per = self.vec_bytes(req)
        c = max(1, min(req.count, self.chunk_bytes // per))
        return min(c, self.block_width) if self.block_width else c

    def need(self, req):
        """Budget a request takes in direct mode: the library's state for one
        chunk of its vectors (the call is held to that many vectors per
        launch), its output and its coefficient field."""
        n = int(np.prod(req.shape))
        es = 8 if self.precision == "fp64" else 4
        out = req.count * n * es if req.kind in ("sample", "solve") else 0
        return self.chunk(req) * self.vec_bytes(req) + out + (2 * out if req.kind == "solve" else 0) + 8 * n

    def engine_slots(self, shape, key=None):
        """Slots of an engine: the prepared plan's share for its grid and field,
        else as many as a quarter of the budget holds, 8 .. nslots_max."""
        if key is not None and key in self.plan:
            return self.plan[key]
        per = self._slot_bytes(shape)
        return int(max(8, min(self.nslots_max, (self.budget // 4) // per)))

    # ---- results
    def _complete(self, req, rc, infos, x, ld, se):
        end = time.perf_counter()
        res = Result(req.rid, req.kind, req.shape, req.count, (end - self._t0 - req.arrival) * 1e3, 0.0,
                     (end - self._t0) * 1e3, [i.m_used for i in infos], rc, x=x if self.keep_outputs else None,
                     logdet=ld if req.kind == "logdet"
                     else None, std_err=se if req.kind == "logdet" else None)
        with self.cv:
            self._results[req.rid] = res
            self.cv.notify_all()

    # ---- direct mode: one library call per request
    def _run(self, req, t0):
        torch, g = self.torch, self.g
        start = time.perf_counter()
        shape = req.shape
        n = int(np.prod(shape))
        k2 = self.fields.get(shape, req.field_id)
        stream = torch.cuda.Stream()
        prob = self._problem(shape, k2, req.tau, stream)
        # at most chunk(req) vectors per launch: the library's state then stays
        # within what need() reserved for this request
        width = self.chunk(req)
        if shape in self.tuning and not self.block_width:
            t = self.tuning[shape]
            prob.set_tuning(block_width=min(width, t["block_width"]), zchunk=t["zchunk"])
        else:
            prob.set_tuning(block_width=width)
        dt = torch.float64 if self.precision == "fp64" else torch.float32
        res = Result(req.rid, req.kind, shape, req.count, 0.0, 0.0, 0.0, [], 0)
        with prob:
            if req.kind == "sample":
                # one call: the library chunks the vectors by the tuned block width
                x = torch.empty(req.count * n, dtype=dt, device="cuda")
                rc, info = prob.sample(x, nsamples=req.count, tol=req.tol, m_max=self._m_max(req), seed=req.seed,
                                       raise_on_error=False)
                res.m_used = [i.m_used for i in info]
                res.status = rc
                res.x = x
            elif req.kind == "solve":
                # seeded right-hand sides from the library's Philox stream, on the problem's stream
                b = torch.empty(req.count * n, dtype=dt, device="cuda")
                g.rng(0, req.count, n, req.seed, b, precision=self.precision, stream=stream.cuda_stream)
                x = torch.empty_like(b)
                rc, info = prob.solve(b, x, nrhs=req.count, tol=req.tol, m_max=self._m_max(req), raise_on_error=False)
                res.m_used = [i.m_used for i in info]
                res.status = rc
                res.x = x
            else:
                ld, se, q, info, rc = prob.logdet(nprobes=req.count, tol=req.tol, m_max=self._m_max(req),
                                                  seed=req.seed, raise_on_error=False)
                res.logdet, res.std_err = ld, se
                res.m_used = [i.m_used for i in info]
                res.status = rc
            stream.synchronize()
        end = time.perf_counter()
        if not self.keep_outputs:
            res.x = None
        res.start_ms = (start - t0) * 1e3
        res.end_ms = (end - t0) * 1e3
        res.latency_ms = (end - t0 - req.arrival) * 1e3
        return res

    def _problem(self, shape, k2, tau, stream):
        g = self.g
        if len(shape) == 2:
            return g.Problem(shape, "neumann", "spde_squared", kappa2=k2, tau=tau, precond="mirror",
                             precision=self.precision, stream=stream.cuda_stream)
        return g.Problem(shape, "dirichlet", "shifted_laplacian", kappa2=k2, tau=tau,
                         precision=self.precision, stream=stream.cuda_stream)

    def prepare(self, requests, tune=True):
        """Generates the coefficient fields of `requests` (their inputs) and
        the library's per-process state before serving starts; in direct mode
        with `tune`, runs the library's autotuner once per grid shape of the
        stream (block width up to the largest request count of that shape,
        3-D z chunk)."""
        for r in requests:
            self.fields.get(r.shape, r.field_id)
        if self.mode == "batched":
            # One engine per grid and field of the stream, all resident at once,
            # so that no engine is torn down and rebuilt while the stream runs.
            # Slots follow demand: the same number of slots per requested vector
            # for every engine (4 .. nslots_max each), the largest such ratio
            # whose slot tables fit the budget; an engine whose slots are cheap
            # (small grids) gets at least what an eighth of an equal share of
            # the budget holds.
            demand = {}
            for r in requests:
                if r.kind != "solve":
                    k = (r.shape, r.field_id)
                    demand[k] = demand.get(k, 0) + r.count
            keys = sorted(set(demand) - set(self.plan), key=lambda k: (len(k[0]), k))
            if keys:
                fixed = sum(self.plan[k] * self._slot_bytes(k[0]) for k in self.plan)
                floor_bytes = self.budget // (8 * (len(self.plan) + len(keys)))

                def slots(k, ratio):
                    return int(max(4, min(self.nslots_max, max(floor_bytes // self._slot_bytes(k[0]),
                                                               ratio * demand[k]))))

                def mem(ratio):
                    return fixed + sum(slots(k, ratio) * self._slot_bytes(k[0]) for k in keys)

                lo, hi = 0.0, float(self.nslots_max)
                for _ in range(50):
                    mid = 0.5 * (lo + hi)
                    lo, hi = (mid, hi) if mem(mid) <= self.budget else (lo, mid)
                for k in keys:
                    self.plan[k] = slots(k, lo)
                for k in keys:
                    if k not in self.engines:
                        self._engine_for(Request(arrival=0.0, rid=-1, kind="sample", shape=k[0], field_id=k[1]))
        if tune and self.mode == "direct":
            widest = {}
            for r in requests:
                widest[r.shape] = max(widest.get(r.shape, 1), r.count)
            for shape in sorted(widest, key=lambda sh: (len(sh), sh)):
                if shape in self.tuning:
                    continue
                stream = self.torch.cuda.Stream()
                k2 = self.fields.get(shape, 0)
                with self._problem(shape, k2, 1.0, stream) as prob:
                    self.tuning[shape] = prob.autotune(widest[shape])
        self.torch.cuda.synchronize()

    # ---- batched mode: engines
    def _engine_for(self, req):
        """The engine of the request's grid and field, created (and idle
        engines released) within the memory budget; None while it does not fit."""
        key = (req.shape, req.field_id)
        if key in self.engines:
            return self.engines[key]
        ns = self.engine_slots(req.shape, key)
        need = ns * self._slot_bytes(req.shape)
        used = sum(e.nslots * self._slot_bytes(e.key[0]) for e in self.engines.values())
        if used + need > self.budget:
            for k, e in sorted(self.engines.items(), key=lambda kv: kv[1].last_used):
                if used + need <= self.budget:
                    break
                if not e.busy():
                    e.close()
                    del self.engines[k]
                    self.engines_released += 1
                    used -= e.nslots * self._slot_bytes(k[0])
        if used + need > self.budget and self.engines:
            return None
        e = Engine(self, key, self.fields.get(req.shape, req.field_id), ns, self._m_max(req.shape))
        self.engines[key] = e
        self.engines_created += 1
        return e

    def close(self):
        for e in self.engines.values():
            e.close()
        self.engines = {}

    def serve(self, requests, realtime=True):
        """Serves `requests` (arrival times in seconds from now).  Returns the
        results in request order and a metrics dict."""
        reqs = sorted(requests)
        self._results = {}
        created0, released0 = self.engines_created, self.engines_released
        t0 = time.perf_counter()
        self._t0 = t0
        direct = [] if self.mode == "batched" else None
        waiting = []  # batched requests whose engine does not fit yet
        inflight = [0]
        futures = {}

        def done_direct(need):
            with self.cv:
                self.used -= need
                inflight[0] -= 1
                self.cv.notify_all()

        with ThreadPoolExecutor(max_workers=self.max_inflight) as ex:
            i = 0
            pending = []  # direct-mode heap by arrival
            while True:
                now = time.perf_counter() - t0
                while i < len(reqs) and (not realtime or reqs[i].arrival <= now):
                    r = reqs[i]
                    i += 1
                    if self.mode == "batched" and r.kind != "solve":
                        waiting.append(r)
                    else:
                        heapq.heappush(pending, r)
                # batched: hand arrivals to their engines
                still = []
                for r in waiting:
                    e = self._engine_for(r)
                    if e is None:
                        still.append(r)
                    else:
                        e.submit(r)
                waiting = still
                for e in self.engines.values():
                    if e.error is not None:
                        raise e.error
                with self.cv:
                    # direct: admit in arrival order while memory and slots allow
                    while pending:
                        req = pending[0]
                        need = self.need(req)
                        if inflight[0] >= self.max_inflight or (self.used + need > self.budget and inflight[0] > 0):
                            break
                        heapq.heappop(pending)
                        self.used += need
                        inflight[0] += 1
                        fut = ex.submit(self._run, req, t0)
                        fut.add_done_callback(lambda f, nd=need: done_direct(nd))
                        futures[req.rid] = fut
                    for rid, fut in list(futures.items()):
                        if fut.done():
                            self._results[rid] = fut.result()
                            del futures[rid]
                    if i >= len(reqs) and not pending and not waiting and not futures and \
                            len(self._results) == len(reqs):
                        break
                    nxt = reqs[i].arrival - (time.perf_counter() - t0) if i < len(reqs) else None
                    timeout = 0.01 if nxt is None else max(0.0, min(0.01, nxt))
                    self.cv.wait(timeout=timeout)
        wall = time.perf_counter() - t0
        out = [self._results[r.rid] for r in requests]
        lat = np.array([r.latency_ms for r in out])
        nsamp = sum(r.count for r in out if r.kind == "sample")
        nld = sum(1 for r in out if r.kind == "logdet")
        nsol = sum(r.count for r in out if r.kind == "solve")
        metrics = {"requests": len(out), "wall_s": wall, "samples": nsamp, "samples_per_s": nsamp / wall,
                   "logdets": nld, "logdets_per_s": nld / wall, "solves": nsol, "solves_per_s": nsol / wall,
                   "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                   "statuses": {str(c): sum(1 for r in out if r.status == c) for c in sorted({r.status for r in out})},
                   "mode": self.mode}
        if self.mode == "batched":
            metrics["engines"] = {"created": self.engines_created - created0, "released": self.engines_released -
                                  released0, "live": len(self.engines),
                                  "slots": {"%s/%d" % ("x".join(map(str, k[0])), k[1]): e.nslots
                                            for k, e in self.engines.items()}}
        return out, metrics
