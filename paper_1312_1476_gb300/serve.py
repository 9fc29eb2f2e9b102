"""Request serving with continuous admission on one GPU.

Requests ask for samples x ~= Q^{-1/2} z (Algorithm 1; Proposition 1 for the
preconditioned 2-D operator) or for log det Q (Section 6) of a lattice GMRF
drawn per request: a 2-D SPDE-type field (Q = tau (K - Lap)^2, zero-Neumann,
mirror-preconditioned) or a 3-D 7-point field (Q = tau (K + L), Dirichlet).

Scheduling: a request is admitted when its estimated device memory (Lanczos
basis, scalars, workspaces) fits in the remaining budget; admitted requests
run concurrently, each on its own problem and CUDA stream, so their kernels
overlap on the device.  A request's samples are computed in chunks small
enough to stay inside the memory it was admitted with, and its Lanczos state
stays on the device for the whole call.  When a request finishes, its memory
returns to the budget and waiting requests are admitted at once (arrivals are
served while earlier requests are still running).

Every result depends only on its own request (problem, seed, tolerance): the
library's reductions have a fixed order per vector, so a request returns the
same bits alone and in any mix (tests/test_gpu_serve.py).
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


class Server:
    """Continuous-admission server over the C-ABI library."""

    M_MAX_2D = 300
    M_MAX_3D = 300

    def __init__(self, mem_budget=None, max_inflight=16, precision="fp32", chunk_bytes=8 << 30, block_width=None):
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
        self.tuning = {}   # grid shape -> block width / z chunk from the library's autotuner
        self.block_width = block_width  # fixed vectors per launch (e.g. 1: one sample at a time)
        self.used = 0
        self.cv = threading.Condition()

    def _m_max(self, req):
        return self.M_MAX_2D if len(req.shape) == 2 else self.M_MAX_3D

    def vec_bytes(self, req):
        """Device bytes one vector of this request needs inside the library."""
        n = int(np.prod(req.shape))
        es = 8 if self.precision == "fp64" else 4
        m = self._m_max(req)
        slots = 2 if req.kind == "logdet" else m + 1
        b = (slots + 4) * n * es + 2 * m * 384 * 8 + 64 * m
        if len(req.shape) == 2:
            b += 3 * n * es + 2 * req.shape[0] * es   # spectrum, g, w workspaces
        return b

    def chunk(self, req):
        per = self.vec_bytes(req)
        c = max(1, min(req.count, self.chunk_bytes // per))
        return min(c, self.block_width) if self.block_width else c

    def need(self, req):
        return self.chunk(req) * self.vec_bytes(req) + 8 * int(np.prod(req.shape))

    def _run(self, req, t0):
        torch, g = self.torch, self.g
        start = time.perf_counter()
        shape = req.shape
        n = int(np.prod(shape))
        k2 = self.fields.get(shape, req.field_id)
        stream = torch.cuda.Stream()
        prob = self._problem(shape, k2, req.tau, stream)
        if self.block_width:
            prob.set_tuning(block_width=self.block_width)
        elif shape in self.tuning:
            t = self.tuning[shape]
            prob.set_tuning(block_width=t["block_width"], zchunk=t["zchunk"])
        dt = torch.float64 if self.precision == "fp64" else torch.float32
        res = Result(req.rid, req.kind, shape, req.count, 0.0, 0.0, 0.0, [], 0)
        with prob:
            c = self.chunk(req)
            if req.kind == "sample":
                x = torch.empty(req.count * n, dtype=dt, device="cuda")
                for s0 in range(0, req.count, c):
                    cc = min(c, req.count - s0)
                    rc, info = prob.sample(x[s0 * n:(s0 + cc) * n], nsamples=cc, tol=req.tol, m_max=self._m_max(req),
                                           seed=(req.seed + s0) & 0x7FFFFFFF, raise_on_error=False)
                    res.m_used += [i.m_used for i in info]
                    res.status = min(res.status, rc)
                res.x = x
            elif req.kind == "solve":
                # seeded right-hand sides from the library's Philox stream, on the problem's stream
                b = torch.empty(req.count * n, dtype=dt, device="cuda")
                g.rng(0, req.count, n, req.seed, b, precision=self.precision, stream=stream.cuda_stream)
                x = torch.empty_like(b)
                for s0 in range(0, req.count, c):
                    cc = min(c, req.count - s0)
                    rc, info = prob.solve(b[s0 * n:(s0 + cc) * n], x[s0 * n:(s0 + cc) * n], nrhs=cc, tol=req.tol,
                                          m_max=self._m_max(req), raise_on_error=False)
                    res.m_used += [i.m_used for i in info]
                    res.status = min(res.status, rc)
                res.x = x
            else:
                ld, se, q, info, rc = prob.logdet(nprobes=req.count, tol=req.tol, m_max=self._m_max(req),
                                                  seed=req.seed, raise_on_error=False)
                res.logdet, res.std_err = ld, se
                res.m_used = [i.m_used for i in info]
                res.status = rc
            stream.synchronize()
        end = time.perf_counter()
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
        the library's per-process state before serving starts; with `tune`,
        runs the library's autotuner once per grid shape of the stream (block
        width up to the largest request count of that shape, 3-D z chunk)."""
        for r in requests:
            self.fields.get(r.shape, r.field_id)
        if tune:
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

    def serve(self, requests, realtime=True):
        """Serves `requests` (arrival times in seconds from now).  Returns the
        results in request order and a metrics dict."""
        reqs = sorted(requests)
        pending = []  # min-heap by arrival
        results = {}
        t0 = time.perf_counter()
        inflight = [0]

        def done(req, need, fut):
            with self.cv:
                self.used -= need
                inflight[0] -= 1
                self.cv.notify_all()

        with ThreadPoolExecutor(max_workers=self.max_inflight) as ex:
            futures = {}
            i = 0
            while i < len(reqs) or pending:
                now = time.perf_counter() - t0
                while i < len(reqs) and (not realtime or reqs[i].arrival <= now):
                    heapq.heappush(pending, reqs[i])
                    i += 1
                with self.cv:
                    # admit in arrival order while memory and slots allow
                    while pending:
                        req = pending[0]
                        need = self.need(req)
                        if inflight[0] >= self.max_inflight or (self.used + need > self.budget and inflight[0] > 0):
                            break
                        heapq.heappop(pending)
                        self.used += need
                        inflight[0] += 1
                        fut = ex.submit(self._run, req, t0)
                        fut.add_done_callback(lambda f, r=req, nd=need: done(r, nd, f))
                        futures[req.rid] = fut
                    nxt = reqs[i].arrival - (time.perf_counter() - t0) if i < len(reqs) else None
                    if pending or nxt is None or nxt > 0:
                        timeout = 0.05 if nxt is None else max(0.0, min(0.05, nxt))
                        self.cv.wait(timeout=timeout)
            for rid, fut in futures.items():
                results[rid] = fut.result()
        wall = time.perf_counter() - t0
        out = [results[r.rid] for r in requests]
        lat = np.array([r.latency_ms for r in out])
        nsamp = sum(r.count for r in out if r.kind == "sample")
        nld = sum(1 for r in out if r.kind == "logdet")
        nsol = sum(r.count for r in out if r.kind == "solve")
        metrics = {"requests": len(out), "wall_s": wall, "samples": nsamp, "samples_per_s": nsamp / wall,
                   "logdets": nld, "logdets_per_s": nld / wall, "solves": nsol, "solves_per_s": nsol / wall,
                   "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                   "statuses": sorted(set(r.status for r in out))}
        return out, metrics
