#!/usr/bin/env python3
"""Benchmark of the Krylov GMRF sampler (Algorithm 1 + Proposition 1) on GB300.

Workload: 2-D SPDE-type GMRF on a 1024 x 1024 grid with zero-Neumann boundary,
Q = (K - Lap)^2 (13-point), log kappa^2(s) a smooth Gaussian field (mean
log 0.05, sd 0.5, length-scale 64 cells), preconditioned by the constant-kappa
circulant version of Q via 2-D FFT (Section 5.1), FP32 vectors with FP64
recurrence scalars, one sample per step to relative tolerance 1e-6.

One step = one gmrf_sample call: Philox noise z, ||z||, the preconditioned
Lanczos loop with its stopping rule, T_m^{-1/2} e_1, x = ||z|| V_m y and the
final M^{-1/2}.  Inputs are resident in HBM; L2 is flushed (256 MiB write)
before every timed step, and every step is timed with CUDA events on the
problem's stream.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GRID = 1024
TOL = 1e-6
M_MAX = 2000
M_MAX_3D = 100
M_MAX_512 = 200   # 256 bases of m_max + 3 vectors stay resident
KAPPA_SEED = 1


def workload_config(precond):
    return {
        "workload": "2D SPDE GMRF %dx%d zero-Neumann, Q=(K-Lap)^2 13-point, log kappa^2 ~ GP(mean log 0.05, "
                    "sd 0.5, ell 64 cells), %s-preconditioned (2D FFT), FP32 vectors / FP64 scalars, "
                    "1 sample per step, rel tol %g" % (GRID, GRID, precond, TOL),
        "grid": [GRID, GRID], "bc": "neumann", "op": "spde_squared", "precond": precond,
        "samples_per_step": 1, "tol": TOL, "m_max": M_MAX,
        "l2": "flushed before every timed step (256 MiB write)",
    }


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        import tempfile
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="gmrf_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def l2_copy_peak(torch, reps=40, trials=6):
    """L2 bandwidth measured live: the best of device copies between two
    buffers of 16, 24 and 32 MiB (working sets of 32-64 MiB, inside the 129 MB
    L2; read + write bytes) and of sums over 32 and 64 MiB (read bytes), reps
    launches per CUDA-event pair, best of `trials`.  Returns (GB/s, what)."""
    best, what = 0.0, ""

    def timed(fn, nbytes):
        for _ in range(3):
            fn()
        top = 0.0
        for _ in range(trials):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            top = max(top, nbytes * reps / (e0.elapsed_time(e1) / 1e3) / 1e9)
        return top

    for mib in (16, 24, 32):
        a = torch.ones(mib * (1 << 20) // 4, dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        r = timed(lambda: b.copy_(a), 2.0 * a.numel() * 4)
        if r > best:
            best, what = r, "copy %d MiB -> %d MiB" % (mib, mib)
        del a, b
    for mib in (32, 64):
        a = torch.ones(mib * (1 << 20) // 4, dtype=torch.float32, device="cuda")
        out = torch.empty((), dtype=torch.float32, device="cuda")
        r = timed(lambda: torch.sum(a, dim=0, out=out), 1.0 * a.numel() * 4)
        if r > best:
            best, what = r, "sum over %d MiB" % mib
        del a
    return best, what


# ------------------------------------------------------------ roofline bytes
def algorithmic_bytes(kclass, n, nx, ny, kind):
    """Bytes each launch of a kernel class must move for one 1024^2 vector
    (FP32).  Spectral rows: circulant (nx/2+1) complex, mirror nx reals."""
    spec = ny * (nx // 2 + 1) * 8 if kind == "circulant" else n * 4
    return {
        "pre_col": 2 * spec,                       # read + write the spectrum
        "pre_row_fwd": 2 * 4 * n + 4 * n + spec,   # q_{j-1}, v_{j-1} in; v_j, spectrum out
        "pre_row_mid": spec + 3 * 4 * n + spec,    # spectrum, v_j, kappa^2 in; g, spectrum out
        "pre_row_last": spec + 3 * 4 * n + 4 * n,  # spectrum, g, v_j, v_{j-1} in; q_j out
    }.get(kclass)


def stencil_step_bytes(n, vec_steps, launches):
    """Algorithmic bytes of fused stencil steps (FP32): per vector-step read
    q_{j-1}, v_{j-1} and write v_j, q_j (16 n); the coefficient field kappa^2
    (4 n) is shared by the vectors of a launch and counted once per launch."""
    return 16.0 * n * vec_steps + 4.0 * n * launches


KERNEL_SOURCES = ("common.cuh", "fft.cuh", "precond.h", "precond_fast.h", "precond_fast.cuh",
                  "precond_fast_mirror.cu", "precond_fast_circ.cu", "precond.cu")


def kernel_sources_sha1():
    """SHA-1 over the sources of the preconditioned step kernels (the traffic
    figures in profiles/ncu_traffic.json are valid only for this source)."""
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1312_1476_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def traffic_from_profile(kclass, key="bytes_per_launch"):
    """DRAM (key "bytes_per_launch") or L2 ("lts_bytes_per_launch") bytes per
    launch from the committed ncu summary, if it matches the current kernel
    source; else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        if d.get("kernel_sources_sha1") != kernel_sources_sha1():
            return None
        return d.get(key, {}).get(kclass)
    except (OSError, ValueError):
        return None


# ------------------------------------------------------------ CPU baseline
def oracle_headline_setup(precond):
    """The oracle's operator for the headline workload (FP64 sparse Q, the
    preconditioner's FFT maps), built once outside any timed region."""
    from oracle import lanczos as olz, precond as opre, stencil
    from paper_1312_1476_gb300 import inputs
    shape = (GRID, GRID)
    k2 = inputs.kappa2_gp_field(shape, seed=KAPPA_SEED).astype(np.float64)
    kb = opre.kappa2_bar(k2)
    kind = "periodic" if precond == "circulant" else "neumann"
    Q = stencil.precision_matrix(shape, "neumann", "spde_squared", k2, 1.0)
    return {"Q": Q, "shape": shape, "kind": kind, "kb": kb}


def oracle_headline_sample(setup, seed):
    """One complete sample of the headline workload by the oracle: Algorithm 1
    on the preconditioned operator with its own stopping rule (FP64, tol 1e-6,
    checked every step), then x = M^{-1/2} u (Proposition 1).  Returns m."""
    from oracle import lanczos as olz
    from paper_1312_1476_gb300 import inputs
    z = inputs.gaussian_vectors(1, GRID * GRID, seed=seed, dtype=np.float64)[0]
    _, m, _, status = olz.precond_sample(setup["Q"], setup["shape"], setup["kind"], "spde_squared", setup["kb"],
                                         1.0, z, TOL, M_MAX)
    if status not in ("ok", "breakdown"):
        raise RuntimeError("oracle sample did not converge: %s" % status)
    return m


def cpu_baseline(precond, nsamples=1):
    """The oracle (FP64 NumPy/SciPy) timed on the host cores: nsamples
    complete samples of the headline workload (a bounded sample of it)."""
    import scipy.fft
    cores = os.cpu_count() or 1
    with scipy.fft.set_workers(cores):
        t0 = time.perf_counter()
        setup = oracle_headline_setup(precond)
        t1 = time.perf_counter()
        ms = [oracle_headline_sample(setup, seed=2 + i) for i in range(nsamples)]
        t2 = time.perf_counter()
    return {"value": nsamples / (t2 - t1), "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": "%d complete %dx%d sample(s) (oracle Algorithm 1 + Proposition 1, FP64, tol %g, m = %s, "
                      "scipy.fft workers=%d); operator assembly (%.1f s) not counted"
                      % (nsamples, GRID, GRID, TOL, ms, cores, t1 - t0)}


# ------------------------------------------------------------------- ours
def run_ours(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1312_1476_gb300 import _build, inputs, replicas
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        dist.barrier()
    from paper_1312_1476_gb300 import gmrf

    shape = (GRID, GRID)
    n = GRID * GRID
    k2 = torch.from_numpy(inputs.kappa2_gp_field(shape, seed=KAPPA_SEED)).cuda()
    stream = torch.cuda.current_stream()
    prob = gmrf.Problem(shape, "neumann", "spde_squared", kappa2=k2, precond=args.precond, precision="fp32",
                        stream=stream.cuda_stream)
    if args.host_loop:
        prob.set_tuning(host_loop=True)
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    seed0 = replicas.replica_seed(1000, rank)

    def step(i, out=None, z=None):
        rc, info = prob.sample(out if out is not None else x, nsamples=1, tol=TOL, m_max=M_MAX,
                               seed=seed0 + i, z=z, check_every=args.check_every)
        return rc, info[0]

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    gmrf.trace_reset()

    def timed_region(trace):
        """K steps, each bracketed by CUDA events on the problem's stream, L2
        flushed before each; returns (device ms, m per step, err_est per step, wall s)."""
        gmrf.trace_timing(trace)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        ms_used, errs = [], []
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            rc, info = step(args.warmup + i)
            ev[i][1].record(stream)
            ms_used.append(info.m_used)
            errs.append(info.err_est)
            if rc != gmrf.OK:
                raise RuntimeError("sample failed: %s %s" % (gmrf.strerror(rc), info))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        gmrf.trace_timing(False)
        return sum(a.elapsed_time(b) for a, b in ev), ms_used, errs, wall

    # headline: no per-kernel events inside the graphs (they perturb the step)
    dev_ms, ms_used, errs, t_wall = timed_region(False)
    launches = gmrf.trace_query("all")[1]
    clk = clocks.stop()
    t_max = replicas.max_over_ranks(dev_ms, dist if world > 1 else None, device="cuda")
    if world > 1:
        dist.barrier()
    value = world * args.steps / (t_max / 1e3)
    # the host-driven iteration on the same steps, for comparison (not the value)
    if args.host_loop:
        loop = {"used": "host-replayed step graphs", "ms_per_step_host_loop": round(dev_ms / args.steps, 4)}
    else:
        prob.set_tuning(host_loop=True)
        host_ms = timed_region(False)[0]
        prob.set_tuning(host_loop=False)
        loop = {"used": "device-side WHILE node", "ms_per_step_device_loop": round(dev_ms / args.steps, 4),
                "ms_per_step_host_loop": round(host_ms / args.steps, 4)}
    # roofline: the same K steps again with CUDA events around every kernel
    gmrf.trace_reset()
    traced_ms, _, _, _ = timed_region(True)

    # per-kernel times from the live trace over the timed region
    classes = ["pre_row_fwd", "pre_col", "pre_row_mid", "pre_row_last", "stencil_step", "tm", "assemble",
               "pre_apply", "init", "rng", "other"]
    per = {c: gmrf.trace_query(c) for c in classes}
    dom = max((c for c in classes if algorithmic_bytes(c, n, GRID, GRID, args.precond)),
              key=lambda c: per[c][0])
    ms_tot, nl, nt = per[dom]
    traced_kernel_ms = sum(v[0] for v in per.values())
    # the per-launch CUDA events inflate the step (traced_ms vs dev_ms): the
    # dominant class's untraced time is its traced share of the untraced step
    avg_traced_s = ms_tot / max(nt, 1) / 1e3
    avg_s = avg_traced_s * (dev_ms / traced_ms)
    ab = algorithmic_bytes(dom, n, GRID, GRID, args.precond)
    peak, peak_src = load_peaks()
    achieved = ab / avg_s / 1e9
    l2peak, l2how = l2_copy_peak(torch)
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic_from_profile(dom),
            "algorithmic_bytes_per_launch": ab, "avg_launch_us": round(avg_s * 1e6, 3),
            "avg_launch_us_traced": round(avg_traced_s * 1e6, 3),
            "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src,
            "kernel_share": {c: round(per[c][0] / max(traced_kernel_ms, 1e-9), 4) for c in classes if per[c][1]},
            "l2": {"achieved": round(achieved, 1), "peak": round(l2peak, 1), "unit": "GB/s",
                   "frac": round(achieved / l2peak, 4),
                   "peak_source": "measured live: best of in-L2 device copies and sums (%s)" % l2how,
                   "traffic": traffic_from_profile(dom, "lts_bytes_per_launch"),
                   "note": "one 1024^2 vector's working set (about 30 MB) stays in the 129 MB L2, so L2 is the "
                           "ceiling that applies; traffic = ncu lts__t_bytes.sum per launch"},
            "timing": "per-class kernel time from CUDA events around every launch (external event nodes of the "
                      "step graphs) in a second pass of the same %d steps (%.3f ms/step traced vs %.3f untraced); "
                      "avg_launch_us = traced average x untraced/traced step time; value uses the untraced pass"
                      % (args.steps, traced_ms / args.steps, dev_ms / args.steps)}

    # end to end through the C ABI with pinned host buffers (z in, x out)
    zh = torch.from_numpy(inputs.gaussian_vectors(1, n, seed=7, dtype=np.float32)[0]).pin_memory()
    xh = torch.empty(n, dtype=torch.float32).pin_memory()
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        e2e_ev[i][0].record(stream)
        rc, _ = step(i, out=xh, z=zh)
        e2e_ev[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = replicas.max_over_ranks(sum(a.elapsed_time(b) for a, b in e2e_ev), dist if world > 1 else None,
                                     device="cuda")

    if rank == 0:
        out = {
            "metric": "GMRF samples/s at 1e-6 rel err (1024^2 grid), %HBM peak; serve p50/p99 ms",
            "value": round(value, 3), "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(args.precond),
            "m_used": {"mean": float(np.mean(ms_used)), "min": int(min(ms_used)), "max": int(max(ms_used))},
            "err_est_max": float(max(errs)),
            "roofline": roof,
            "e2e": {"value": round(world * args.steps / (e2e_ms / 1e3), 3), "unit": "samples/s",
                    "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n},
            "gpu_launches": int(launches),
            "lanczos_loop": loop,
            "clocks": clk,
            "wall_s_timed_region": round(t_wall, 3),
        }
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.precond)
        if world == 1 and not args.no_variants:
            # the other workloads are single-GPU measurements: under torchrun the
            # line carries the replicated headline only
            out["variants"] = measure_variants(args, gmrf, torch, flush, peak)
        print(json.dumps(out), flush=True)
    prob.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def measure_variants(args, gmrf, torch, flush, peak):
    """Other measured workloads, reported beside the headline."""
    from paper_1312_1476_gb300 import inputs
    out = {}
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        ms = []
        for i in range(reps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = fn(i)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.mean(ms)), r

    # plain-torus circulant preconditioner on the headline input
    shape = (GRID, GRID)
    n = GRID * GRID
    k2 = torch.from_numpy(inputs.kappa2_gp_field(shape, seed=KAPPA_SEED)).cuda()
    with gmrf.Problem(shape, "neumann", "spde_squared", kappa2=k2, precond="circulant",
                      stream=stream.cuda_stream) as p:
        x = torch.empty(n, dtype=torch.float32, device="cuda")
        p.sample(x, nsamples=1, tol=TOL, m_max=M_MAX, seed=1)
        ms, (rc, info) = timed(lambda i: p.sample(x, nsamples=1, tol=TOL, m_max=M_MAX, seed=10 + i), 3)
        out["circulant"] = {"workload": "same input, plain-torus circulant M", "samples_per_s": 1e3 / ms,
                            "ms_per_sample": ms, "m_used": info[0].m_used, "status": rc}

    # Section 5.1: the linear solve x = Q^{-1} b on the headline problem (the
    # sampler's iteration and preconditioner, T_m^{-1} in place of T_m^{-1/2})
    with gmrf.Problem(shape, "neumann", "spde_squared", kappa2=k2, precond="mirror",
                      stream=stream.cuda_stream) as p:
        b = torch.from_numpy(inputs.gaussian_vectors(1, n, seed=7, dtype=np.float32)).cuda()
        x = torch.empty(n, dtype=torch.float32, device="cuda")
        p.solve(b, x, nrhs=1, tol=TOL, m_max=M_MAX)
        ms, (rc, info) = timed(lambda i: p.solve(b, x, nrhs=1, tol=TOL, m_max=M_MAX), 3)
        out["solve_1024"] = {"workload": "headline problem, x = Q^{-1} b (Section 5.1 solve), mirror M, FP32, "
                                         "relative residual of the preconditioned system 1e-6, one right-hand side",
                             "solves_per_s": 1e3 / ms, "ms_per_solve": ms, "m_used": info[0].m_used,
                             "status": rc}
    # the sMMALA proposal of Section 3 at 1024^2 (LGCP recipe of Table 1, FP32,
    # tol 1e-6): one mean solve (Q + H)^{-1} grad and one sample, both with the
    # prior as the preconditioner
    mdl = inputs.lgcp_smmala_model(GRID)
    with gmrf.Problem(shape, "periodic", "spde_plus_diag", kappa2=torch.from_numpy(mdl["d"]).cuda(),
                      kappa2_const=mdl["kappa2_prior"], tau=mdl["tau"], precond="circulant",
                      stream=stream.cuda_stream) as p:
        gb = torch.from_numpy(inputs.lgcp_gradient(GRID).astype(np.float32)).cuda()
        xm = torch.empty(n, dtype=torch.float32, device="cuda")
        xs = torch.empty(n, dtype=torch.float32, device="cuda")
        p.solve(gb, xm, nrhs=1, tol=TOL, m_max=200)
        p.sample(xs, nsamples=1, tol=TOL, m_max=200, seed=1)
        mss, (rcs, infs) = timed(lambda i: p.solve(gb, xm, nrhs=1, tol=TOL, m_max=200), 3)
        msp, (rcp, infp) = timed(lambda i: p.sample(xs, nsamples=1, tol=TOL, m_max=200, seed=50 + i), 3)
        out["smmala_proposal_1024"] = {
            "workload": "LGCP sMMALA proposal on a 1024^2 torus (Table 1 recipe), FP32, tol 1e-6: mean solve "
                        "(Q + H)^{-1} grad log pi(y|x) plus one sample, prior (circulant) preconditioner",
            "proposals_per_s": 1e3 / (mss + msp), "ms_solve": mss, "ms_sample": msp,
            "m_solve": infs[0].m_used, "m_sample": infp[0].m_used, "status": [rcs, rcp]}

    # batched 512^2: 256 samples + log det with 64 Rademacher probes in one call each
    shape = (512, 512)
    n = 512 * 512
    k2 = torch.from_numpy(inputs.kappa2_gp_field(shape, seed=KAPPA_SEED, ell=64.0)).cuda()
    with gmrf.Problem(shape, "neumann", "spde_squared", kappa2=k2, precond="mirror",
                      stream=stream.cuda_stream) as p:
        ns = 256
        tune512 = p.autotune(ns)
        x = torch.empty(ns * n, dtype=torch.float32, device="cuda")
        p.sample(x, nsamples=ns, tol=TOL, m_max=M_MAX_512, seed=1)
        gmrf.trace_reset()
        ms, (rc, info) = timed(lambda i: p.sample(x, nsamples=ns, tol=TOL, m_max=M_MAX_512, seed=20 + i), 3)
        mld, ld = timed(lambda i: p.logdet(nprobes=64, tol=TOL, m_max=M_MAX_512, seed=30 + i), 3)
        # coloured Hutchinson (Section 6.1) at the same number of quadratures
        # (about 64): draws x (p + 1)^2 colour classes
        coloured = {}
        for pd, nd in ((1, 16), (2, 7), (3, 4)):
            mc, lc = timed(lambda i: p.logdet(nprobes=nd, tol=TOL, m_max=M_MAX_512, seed=30 + i, colour_dist=pd), 2)
            coloured["p%d" % pd] = {"draws": nd, "quadratures": nd * (pd + 1) ** 2, "logdet": lc[0],
                                    "std_err": lc[1], "logdets_per_s": 1e3 / mc}
        # the same 256 samples and 64 probes as one block of 320 vectors (one call)
        msc, rsl = timed(lambda i: p.sample_logdet(x, nsamples=ns, nprobes=64, tol=TOL, m_max=M_MAX_512,
                                                   seed=20 + i, probe_seed=30 + i), 3)
        one_block = {"vectors": ns + 64, "ms_per_call": msc, "samples_per_s": ns * 1e3 / msc,
                     "logdets_per_s": 1e3 / msc, "logdet": rsl[2], "logdet_std_err": rsl[3], "status": rsl[0]}
        out["batched_512"] = {
            "workload": "512x512 SPDE (same recipe, ell 64), mirror M, 256 samples per call (m_max %d, one "
                        "batch); log det with 64 Rademacher probes per call" % M_MAX_512,
            "samples_per_s": ns * 1e3 / ms, "ms_per_call": ms,
            "m_mean": float(np.mean([i.m_used for i in info])), "status": rc,
            "logdets_per_s": 1e3 / mld, "logdet": ld[0], "logdet_std_err": ld[1],
            "logdet_m_mean": float(np.mean([i.m_used for i in ld[3]])), "autotune": tune512,
            "logdet_coloured": coloured, "samples_and_probes_one_block": one_block}

    # 3-D 256^3 Dirichlet 7-point, kappa^2 ~ U[0.01, 1], 16 samples; m_max capped
    # so that all 16 Lanczos bases (m_max + 3 vectors each) stay resident in HBM
    shape = (256, 256, 256)
    n = 256 ** 3
    ns, m3 = 16, M_MAX_3D
    k3 = torch.from_numpy(inputs.kappa2_uniform_field(shape, seed=KAPPA_SEED)).cuda()
    with gmrf.Problem(shape, "dirichlet", "shifted_laplacian", kappa2=k3, stream=stream.cuda_stream) as p:
        tune3 = p.autotune(ns)
        x = torch.empty(ns * n, dtype=torch.float32, device="cuda")
        p.sample(x, nsamples=ns, tol=TOL, m_max=m3, seed=1)
        ms, (rc, info) = timed(lambda i: p.sample(x, nsamples=ns, tol=TOL, m_max=m3, seed=40 + i), 3)
        gmrf.trace_reset()
        gmrf.trace_timing(True)
        _, (rc_t, info_t) = timed(lambda i: p.sample(x, nsamples=ns, tol=TOL, m_max=m3, seed=40 + i), 1)
        gmrf.trace_timing(False)
        st_ms, st_l, st_t = gmrf.trace_query("stencil_step")
        vec_steps = int(sum(i.m_used for i in info_t))   # vector-steps the traced launches did
        byts = stencil_step_bytes(n, vec_steps, st_t)
        ach = byts / (st_ms / 1e3) / 1e9
        out["3d_256"] = {
            "workload": "256^3 Dirichlet, Q = 7-point Laplacian + kappa^2 (i.i.d. U[0.01,1]), 16 samples per "
                        "call, tol 1e-6, m_max %d (all bases resident)" % m3,
            "samples_per_s": ns * 1e3 / ms, "ms_per_call": ms,
            "m_mean": float(np.mean([i.m_used for i in info])), "status": rc, "autotune": tune3,
            "stencil_step": {"kernel": "k_stencil3d_tma (TMA-staged fused step)",
                             "avg_launch_us": st_ms * 1e3 / max(st_t, 1), "launches": st_t,
                             "achieved_GBps": ach, "peak_GBps": peak, "frac": ach / peak,
                             "algorithmic_bytes_per_launch": byts / max(st_t, 1),
                             "bytes_rule": "16 n per vector-step (read q_{j-1}, v_{j-1}; write q_j, v_j) + "
                                           "4 n per launch (kappa^2, shared by the launch's vectors)"}}
        # the same 16 samples with a bfloat16 basis for the assembly (half the V_m memory)
        xb = torch.empty(ns * n, dtype=torch.float32, device="cuda")
        p.sample(xb, nsamples=ns, tol=TOL, m_max=m3, seed=40, v_storage="bf16")
        msb, (rcb, infob) = timed(lambda i: p.sample(xb, nsamples=ns, tol=TOL, m_max=m3, seed=40 + i,
                                                     v_storage="bf16"), 3)
        p.sample(x, nsamples=ns, tol=TOL, m_max=m3, seed=42)
        diff = float(torch.linalg.vector_norm((xb - x).view(ns, n).double(), dim=1).max() /
                     torch.linalg.vector_norm(x.view(ns, n).double(), dim=1).min())
        out["3d_256_bf16_basis"] = {
            "workload": "same 256^3 problem and 16 samples, V_m stored in bfloat16 for the assembly",
            "samples_per_s": ns * 1e3 / msb, "ms_per_call": msb, "status": rcb,
            "m_mean": float(np.mean([i.m_used for i in infob])),
            "basis_bytes_per_vector_step": {"fp32": 4 * n, "bf16": 2 * n},
            "max_rel_diff_vs_fp32_basis": diff}
        # two passes, no basis kept (O(n) memory per vector, twice the steps)
        p.sample(xb, nsamples=ns, tol=TOL, m_max=m3, seed=40, v_storage="none")
        mst, (rct, infot) = timed(lambda i: p.sample(xb, nsamples=ns, tol=TOL, m_max=m3, seed=40 + i,
                                                     v_storage="none"), 3)
        p.sample(x, nsamples=ns, tol=TOL, m_max=m3, seed=42)
        out["3d_256_two_pass"] = {
            "workload": "same 256^3 problem and 16 samples, no basis kept: the iteration runs twice and the "
                        "second pass adds ||z|| y_j v_j after every step",
            "samples_per_s": ns * 1e3 / mst, "ms_per_call": mst, "status": rct,
            "basis_bytes_per_vector": {"stored_fp32": 4 * n * (m3 + 1), "two_pass": 4 * n * 2 + 8 * n},
            "bitwise_equal_to_stored_basis": bool(torch.equal(xb, x))}
    # 2-D fused stencil step without a preconditioner (the streamed strip kernel), on
    # HBM-bound batches: 40 steps per vector (tol below reach), kernel time traced
    st2d = {}
    for shp, op, bc, nv in (((1024, 1024), "spde_squared", "neumann", 16),
                            ((2048, 2048), "shifted_laplacian", "dirichlet", 8)):
        n2 = shp[0] * shp[1]
        kk = torch.from_numpy(inputs.kappa2_gp_field(shp, seed=KAPPA_SEED, ell=64.0)).cuda()
        with gmrf.Problem(shp, bc, op, kappa2=kk, stream=stream.cuda_stream) as p:
            x2 = torch.empty(nv * n2, dtype=torch.float32, device="cuda")
            p.sample(x2, nsamples=nv, tol=1e-12, m_max=40, seed=1, raise_on_error=False)
            gmrf.trace_reset()
            gmrf.trace_timing(True)
            _, (rc2, inf2) = timed(lambda i: p.sample(x2, nsamples=nv, tol=1e-12, m_max=40, seed=60 + i,
                                                      raise_on_error=False), 1)
            gmrf.trace_timing(False)
            sm2, sl2, stt2 = gmrf.trace_query("stencil_step")
            vs2 = int(sum(i.m_used for i in inf2))
            by2 = stencil_step_bytes(n2, vs2, stt2)
            ach2 = by2 / (sm2 / 1e3) / 1e9
            st2d["%dx%d_%s_x%d" % (shp[0], shp[1], op, nv)] = {
                "kernel": "k_stencil2d_strip", "avg_launch_us": sm2 * 1e3 / max(stt2, 1), "launches": stt2,
                "achieved_GBps": ach2, "peak_GBps": peak, "frac": ach2 / peak,
                "algorithmic_bytes_per_launch": by2 / max(stt2, 1),
                "bytes_rule": "16 n per vector-step (read q_{j-1}, v_{j-1}; write q_j, v_j) + 4 n per launch "
                              "(kappa^2)"}
    out["2d_stencil_step"] = {"workload": "unpreconditioned 2-D fused step, 40 steps per vector, FP32", **st2d}
    out["cfg1_64x64_periodic_fp64"] = measure_cfg1(gmrf, torch, timed)
    if not getattr(args, "no_cpu_baseline", False):
        # the oracle beside the batched and 3-D workloads (bounded samples on the host cores)
        out["batched_512"]["cpu_oracle"] = cpu_oracle_rate("batched_512", out["batched_512"]["m_mean"])
        out["3d_256"]["cpu_oracle"] = cpu_oracle_rate("3d_128", out["3d_256"]["m_mean"])
    out["table1"] = measure_table1(gmrf, torch)
    out["figure3_ichol"] = measure_figure3(gmrf, torch, timed, cpu=not getattr(args, "no_cpu_baseline", False))
    out["serving"] = measure_serving(nreq=getattr(args, "serving_requests", 1000))
    return out


def measure_figure3(gmrf, torch, timed, cpu=True):
    """Section 5.2 (Figure 3): the sparse sampler on Q = (31^2 G)^2, G the
    5-point Dirichlet Laplacian of a 30 x 30 lattice (n = 900), without a
    preconditioner and with incomplete-Cholesky factors F of several drop
    thresholds (M = F F^T, Proposition 1): factor size, subspace size to the
    Theorem 1 estimate 1e-8 (FP64) and samples/s at 256 samples per call."""
    from paper_1312_1476_gb300 import inputs
    Q = inputs.figure3_matrix()
    n = 900
    m_max = 3000
    cfgs = [("none", None, None), ("jacobi (droptol inf)", float("inf"), 0.0),
            ("IC(0), shift 1e-2", -1.0, 1e-2), ("ICT droptol 1e-3, shift 1e-3", 1e-3, 1e-3),
            ("ICT droptol 1e-5, shift 1e-4", 1e-5, 1e-4), ("exact Cholesky (droptol 0)", 0.0, 0.0)]
    res = {"workload": "Figure 3 matrix (31^2 G)^2, n = 900, FP64, tol 1e-8, 256 samples per call; "
                       "IC drop rule: |update| < droptol * ||column of Q + shift diag(Q)||_1",
           "factors": {}}
    x = torch.empty(256 * n, dtype=torch.float64, device="cuda")
    for name, dt, sh in cfgs:
        F = None if dt is None else gmrf.ichol(Q, droptol=dt, shift=sh)
        with gmrf.SparseProblem(Q, F, precision="fp64") as p:
            p.sample(x, nsamples=256, tol=1e-8, m_max=m_max, seed=1)
            ms, (rc, info) = timed(lambda i: p.sample(x, nsamples=256, tol=1e-8, m_max=m_max, seed=3 + i), 2)
        ms_used = [i.m_used for i in info]
        res["factors"][name] = {"nnz_F": int(len(F[1])) if F is not None else 0,
                                "m_mean": float(np.mean(ms_used)), "m_max": int(max(ms_used)),
                                "samples_per_s": 256e3 / ms, "ms_per_call": ms, "status": rc}
    if cpu:
        # the oracle's map (dense eigendecomposition of A, FP64) for the ICT 1e-3 factor
        from oracle import sparse as osp
        Qs = osp.csr(*Q)
        F = osp.ichol(Qs, droptol=1e-3, shift=1e-3)
        z = inputs.gaussian_vectors(1, n, seed=2, dtype=np.float64)
        t0 = time.perf_counter()
        reps = 0
        while time.perf_counter() - t0 < 2.0:
            osp.sample_precond_dense(Qs, F, z)
            reps += 1
        dtm = (time.perf_counter() - t0) / reps
        res["cpu_oracle"] = {"value": 1.0 / dtm, "unit": "samples/s", "cores": os.cpu_count() or 1, "kind": "oracle",
                             "sample": "%d samples of the oracle's dense Proposition 1 map (eigendecomposition of "
                                       "A = F^{-1} Q F^{-T}, ICT 1e-3 factor, FP64)" % reps}
    return res


def measure_cfg1(gmrf, torch, timed):
    """64 x 64 periodic, Q = 0.1 I + 5-point Laplacian, FP64, tol 1e-10, m <= 300
    (the smallest configuration): one sample per call and 256 per call, with
    the oracle's Algorithm 1 on the host beside it."""
    from oracle import lanczos as olz, stencil
    from paper_1312_1476_gb300 import inputs
    shape, n = (64, 64), 4096
    res = {"workload": "64x64 periodic, Q = 0.1 I + 5-point Laplacian, FP64, tol 1e-10, m_max 300"}
    with gmrf.Problem(shape, "periodic", "shifted_laplacian", kappa2_const=0.1, precision="fp64") as p:
        x1 = torch.empty(n, dtype=torch.float64, device="cuda")
        xb = torch.empty(256 * n, dtype=torch.float64, device="cuda")
        p.sample(x1, nsamples=1, tol=1e-10, m_max=300, seed=1)
        p.sample(xb, nsamples=256, tol=1e-10, m_max=300, seed=1)
        ms1, (rc1, info1) = timed(lambda i: p.sample(x1, nsamples=1, tol=1e-10, m_max=300, seed=5 + i), 5)
        msb, (rcb, infob) = timed(lambda i: p.sample(xb, nsamples=256, tol=1e-10, m_max=300, seed=5 + i), 3)
    res.update({"samples_per_s_one_per_call": 1e3 / ms1, "ms_per_sample": ms1, "m_used": info1[0].m_used,
                "samples_per_s_256_per_call": 256e3 / msb, "status": max(rc1, rcb)})
    Q = stencil.precision_matrix(shape, "periodic", "shifted_laplacian", 0.1)
    z = inputs.gaussian_vectors(1, n, seed=2, dtype=np.float64)[0]
    t0 = time.perf_counter()
    reps = 0
    while time.perf_counter() - t0 < 2.0:
        olz.adaptive_sample(lambda v: Q @ v, z, 1e-10, 300)
        reps += 1
    dt = (time.perf_counter() - t0) / reps
    res["cpu_oracle"] = {"value": 1.0 / dt, "unit": "samples/s", "cores": os.cpu_count() or 1, "kind": "oracle",
                         "sample": "%d full samples (oracle Algorithm 1, sparse matvec, FP64)" % reps}
    return res


def cpu_oracle_rate(which, m_mean):
    """The oracle on the host cores: a few Lanczos steps of one vector of the
    workload, scaled to its mean m (a bounded sample, labelled)."""
    import scipy.fft
    from oracle import lanczos as olz, precond as opre, stencil
    from paper_1312_1476_gb300 import inputs
    cores = os.cpu_count() or 1
    k_steps = 6
    with scipy.fft.set_workers(cores):
        if which == "batched_512":
            shape = (512, 512)
            k2 = inputs.kappa2_gp_field(shape, seed=KAPPA_SEED, ell=64.0).astype(np.float64)
            Q = stencil.precision_matrix(shape, "neumann", "spde_squared", k2, 1.0)
            A = olz.preconditioned_operator(Q, shape, "neumann", "spde_squared", opre.kappa2_bar(k2), 1.0)
            label = "512x512 SPDE, mirror M"
        else:
            shape = (128, 128, 128)
            k3 = inputs.kappa2_uniform_field(shape, seed=KAPPA_SEED).astype(np.float64)
            Q = stencil.precision_matrix(shape, "dirichlet", "shifted_laplacian", k3, 1.0)
            A = lambda v: Q @ v  # noqa: E731
            label = "128^3 Dirichlet 7-point (the 256^3 recipe one size down; 256^3 does not fit a bounded sample)"
        z = inputs.gaussian_vectors(1, int(np.prod(shape)), seed=2, dtype=np.float64)[0]
        t0 = time.perf_counter()
        done = 0
        for st in olz.lanczos_steps(A, z):
            done += 1
            if done >= k_steps or st["breakdown"]:
                break
        per_step = (time.perf_counter() - t0) / done
    return {"value": 1.0 / (per_step * m_mean), "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": "%d Lanczos steps of one vector of %s (FP64), scaled to m = %.1f" % (done, label, m_mean)}


def measure_table1(gmrf, torch):
    """Table 1 (Section 5.1): Lanczos steps until the Theorem 1 estimate is
    below 1e-8 (FP64) for the sMMALA proposal of an LGCP on an N x N lattice of
    the unit torus, Q = prior + diag(Fisher information), preconditioned by the
    prior (circulant, applied by FFT) and without preconditioning."""
    from paper_1312_1476_gb300 import inputs
    pre, un, ms_sample, pre_solve = {}, {}, {}, {}
    for N in (16, 32, 64, 128, 256, 512, 1024, 2048, 4096):
        mdl = inputs.lgcp_smmala_model(N)
        kw = dict(kappa2=torch.from_numpy(mdl["d"]).cuda(), kappa2_const=mdl["kappa2_prior"], tau=mdl["tau"],
                  precision="fp64")
        x = torch.empty(N * N, dtype=torch.float64, device="cuda")
        with gmrf.Problem((N, N), "periodic", "spde_plus_diag", precond="circulant", **kw) as p:
            p.sample(x, nsamples=1, tol=1e-8, m_max=200, seed=1, check_every=1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, info = p.sample(x, nsamples=1, tol=1e-8, m_max=200, seed=2, check_every=1)
            torch.cuda.synchronize()
            ms_sample[N] = round((time.perf_counter() - t0) * 1e3, 3)
            pre[N] = info[0].m_used if rc == gmrf.OK else None
            # the proposal mean's solve with the same preconditioner (Section 5.1)
            gb = torch.from_numpy(inputs.lgcp_gradient(N)).cuda()
            rcs, infs = p.solve(gb, x, nrhs=1, tol=1e-8, m_max=200, check_every=1)
            pre_solve[N] = infs[0].m_used if rcs == gmrf.OK else None
        if N <= 128:
            with gmrf.Problem((N, N), "periodic", "spde_plus_diag", **kw) as p:
                rc, info = p.sample(x, nsamples=1, tol=1e-8, m_max=8192, seed=2, check_every=16,
                                    raise_on_error=False)
                un[N] = info[0].m_used if rc == gmrf.OK else None
    return {"workload": "LGCP sMMALA proposal on the unit torus (prior h^2 (kappa^2 + L/h^2)^2, kappa 10; "
                        "Fisher information diag(h^2 exp(x)), mean intensity 2000), FP64, tol 1e-8, one sample",
            "m_preconditioned": pre, "m_unpreconditioned": un, "ms_per_preconditioned_sample": ms_sample,
            "m_mean_solve_preconditioned": pre_solve,
            "paper_table1_context": {"preconditioned": 6, "unpreconditioned": {"16": 102, "32": 286, "64": 790,
                                                                              "128": 2166},
                                     "note": "the paper's prior is unspecified; counts are context"}}


def measure_serving(nreq=1000, baseline_nreq=24):
    """Config 5: a Poisson request stream of the serving mix (2-D SPDE
    128^2..1024^2 with the mirror preconditioner, 3-D 7-point 64^3..128^3,
    kappa^2 field and tau ~ U[0.5, 5] per request, 1-64 samples or a log det
    with 16-64 probes, tol 1e-6), served with continuous batching (the
    library's slot server: requests' vectors share launches and enter slots as
    they free up) at 0.25x, 0.5x, 1x and 2x the measured saturation rate, with
    nreq requests per rate; the same stream without packing (one library call
    per request, up to 16 in flight) at 1x and 2x; and the one-request,
    one-sample-at-a-time FP64 baseline at the same four rates on a bounded
    prefix of each stream (baseline_nreq requests: it saturates far below
    these rates)."""
    import torch
    from paper_1312_1476_gb300 import serve

    def stream(rate, count):
        return serve.make_mix(count, rate=rate, seed=4)

    res = {"requests_per_rate": nreq}
    # memory the earlier workloads left in torch's cache goes back to the device,
    # so the serving budget (a share of free HBM) does not depend on them
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    srv = serve.Server(mode="batched", keep_outputs=False)
    try:
        burst = stream(1e6, nreq)
        for r in burst:
            r.arrival = 0.0
        srv.prepare(burst)
        srv.serve(burst[:6], realtime=False)  # engines and graphs of the first grids
        sat = srv.serve(burst, realtime=False)[1]  # the results (device outputs) are dropped at once
        sat_rate = nreq / sat["wall_s"]
        res["saturation"] = dict(sat, rate_req_per_s=sat_rate)
        for frac in (0.25, 0.5, 1.0, 2.0):
            reqs = stream(frac * sat_rate, nreq)
            srv.prepare(reqs)
            met = srv.serve(reqs, realtime=True)[1]
            res["packed_rate_%gx" % frac] = dict(met, rate_req_per_s=frac * sat_rate)
    finally:
        srv.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()  # outputs cached by torch go back to the device for the library's own allocations
    off = serve.Server(mode="direct", max_inflight=16, keep_outputs=False)
    for frac in (1.0, 2.0):
        reqs = stream(frac * sat_rate, nreq)
        off.prepare(reqs)
        met = off.serve(reqs, realtime=True)[1]
        res["unpacked_rate_%gx" % frac] = dict(met, rate_req_per_s=frac * sat_rate)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    base = serve.Server(mode="direct", max_inflight=1, precision="fp64", block_width=1, keep_outputs=False)
    for frac in (0.25, 0.5, 1.0, 2.0):
        reqs = stream(frac * sat_rate, baseline_nreq)
        base.prepare(reqs, tune=False)
        met = base.serve(reqs, realtime=True)[1]
        res["fp64_one_at_a_time_rate_%gx" % frac] = dict(met, rate_req_per_s=frac * sat_rate)
    res["workload"] = ("config 5 mix: samples (1-64) and log dets (16-64 probes) of 2-D SPDE (mirror M, 128^2-1024^2) "
                       "and 3-D 7-point (64^3-128^3) GMRFs, kappa^2 and tau per request, tol 1e-6; latency = "
                       "completion - arrival; packed = continuous batching in the library's slot server, unpacked "
                       "= one library call per request")
    return res


def run_reference(args):
    """The oracle as the reference arm (CPU, FP64), same workload and metric:
    every step is one complete sample (Algorithm 1 on the preconditioned
    operator to tol 1e-6, then M^{-1/2}), W untimed and K timed steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import scipy.fft
    cores = os.cpu_count() or 1
    with scipy.fft.set_workers(cores):
        setup = oracle_headline_setup(args.precond)
        for i in range(args.warmup):
            oracle_headline_sample(setup, seed=1000 + i)
        times, ms = [], []
        for i in range(args.steps):
            t0 = time.perf_counter()
            ms.append(oracle_headline_sample(setup, seed=1000 + args.warmup + i))
            times.append(time.perf_counter() - t0)
    total = float(np.sum(times))
    value = args.steps / total
    sample = ("%d complete %dx%d samples (oracle Algorithm 1 + Proposition 1, FP64, tol %g, m mean %.1f, "
              "scipy.fft workers=%d), one per step" % (args.steps, GRID, GRID, TOL, float(np.mean(ms)), cores))
    out = {"impl": "reference", "metric": "GMRF samples/s at 1e-6 rel err (1024^2 grid), %HBM peak; serve p50/p99 ms",
           "value": value, "unit": "samples/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(args.precond),
           "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precond", choices=["circulant", "mirror"], default="mirror")
    ap.add_argument("--check-every", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--host-loop", action="store_true",
                    help="host-replayed step graphs instead of the device-side loop (for per-kernel profilers)")
    ap.add_argument("--no-variants", action="store_true", help="headline workload only")
    ap.add_argument("--serving-requests", type=int, default=1000, help="requests per rate of the serving sweep")
    ap.add_argument("--serving-only", action="store_true", help="run only the serving sweep (config 5)")
    args = ap.parse_args()
    if args.serving_only:
        import torch
        from paper_1312_1476_gb300 import _build
        _build.build()
        torch.cuda.init()
        print(json.dumps({"serving": measure_serving(nreq=args.serving_requests)}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
