"""Bounded runs of the library's hot path for profiler captures.

    python -m paper_1312_1476_gb300.profile_case <case> [--nsamples N] [--steps M] [--trace]

Each case builds one benchmark configuration on its synthetic inputs, runs
one sample call capped at M Lanczos steps (so it ends after M steps whatever
the tolerance) and exits.  The host drives the steps (replayed step graphs,
not the device-side loop), so a per-kernel profiler sees plain kernel nodes.  The sizes keep a capture small: one or a few
vectors, a few GB of device memory at most.  With --trace it then repeats the
call twice more, timed as a whole and then with CUDA events around every
launch, and reports each kernel class's time per vector-step (the sum of the
Lanczos steps of all vectors).

Cases:
  headline_1024  1024 x 1024 SPDE, zero-Neumann, mirror preconditioner, FP32
  batched_512    512 x 512 SPDE, mirror preconditioner, FP32, N vectors per launch
  3d_256         256^3 Dirichlet 7-point, kappa^2 i.i.d. U[0.01, 1], FP32
  3d_128         the same recipe at 128^3 (16 vectors of 8 MiB: a multi-vector launch
                 larger than L2 that a counter capture can replay)
  stencil2d_1024 1024 x 1024 SPDE, zero-Neumann, no preconditioner, FP32 (the
                 streamed 2-D step), N vectors per launch
  figure3_ichol  the Figure 3 matrix (31^2 G)^2 (n = 900, Section 5.2) in CSR,
                 incomplete-Cholesky factor (drop tolerance 1e-3, shift 1e-3),
                 FP64, N vectors per launch
"""
from __future__ import annotations

import argparse

import numpy as np


def run(case: str, nsamples: int, steps: int, trace: bool = False) -> dict:
    import torch
    from . import gmrf, inputs
    if case == "headline_1024":
        shape = (1024, 1024)
        k2 = torch.from_numpy(inputs.kappa2_gp_field(shape, seed=1)).cuda()
        prob = gmrf.Problem(shape, "neumann", "spde_squared", kappa2=k2, precond="mirror")
    elif case == "batched_512":
        shape = (512, 512)
        k2 = torch.from_numpy(inputs.kappa2_gp_field(shape, seed=1, ell=64.0)).cuda()
        prob = gmrf.Problem(shape, "neumann", "spde_squared", kappa2=k2, precond="mirror")
    elif case == "stencil2d_1024":
        shape = (1024, 1024)
        k2 = torch.from_numpy(inputs.kappa2_gp_field(shape, seed=1, ell=64.0)).cuda()
        prob = gmrf.Problem(shape, "neumann", "spde_squared", kappa2=k2)
    elif case in ("3d_256", "3d_128"):
        shape = (256, 256, 256) if case == "3d_256" else (128, 128, 128)
        k2 = torch.from_numpy(inputs.kappa2_uniform_field(shape, seed=1)).cuda()
        prob = gmrf.Problem(shape, "dirichlet", "shifted_laplacian", kappa2=k2)
    elif case == "figure3_ichol":
        Q = inputs.figure3_matrix()
        prob = gmrf.SparseProblem(Q, gmrf.ichol(Q, droptol=1e-3, shift=1e-3), precision="fp64")
        shape = (prob.n,)
    else:
        raise ValueError("unknown case %r" % case)
    n = int(np.prod(shape))
    out = {"case": case, "nsamples": nsamples}

    def call():
        rc, info = prob.sample(x, nsamples=nsamples, tol=1e-6, m_max=steps, seed=2, check_every=8,
                               raise_on_error=False)
        torch.cuda.synchronize()
        if rc not in (gmrf.OK, gmrf.ERR_NOT_CONVERGED):
            raise gmrf.GmrfError(rc, "profile case " + case)
        return rc, info

    with prob:
        # host-replayed step graphs: a per-kernel profiler then sees plain
        # kernel nodes (the kernels are the same as under the device-side loop)
        prob.set_tuning(block_width=0, zchunk=0, host_loop=True)
        x = torch.empty(nsamples * n, dtype=torch.float64 if prob.precision == "fp64" else torch.float32,
                        device="cuda")
        rc, info = call()
        out.update(m_used=[i.m_used for i in info], rc=rc)
        if trace:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            rc, info = call()
            e1.record()
            torch.cuda.synchronize()
            vs = sum(i.m_used for i in info)
            out["ms_call"] = round(e0.elapsed_time(e1), 3)
            out["us_per_vec_step"] = round(e0.elapsed_time(e1) * 1e3 / vs, 3)
            gmrf.trace_reset()
            gmrf.trace_timing(True)
            try:
                call()
            finally:
                gmrf.trace_timing(False)
            per = {}
            for c in gmrf.KERNEL_CLASSES:
                ms, _, launches = gmrf.trace_query(c)
                if launches:
                    per[c] = {"launches": launches, "us_per_launch": round(ms * 1e3 / launches, 2),
                              "us_per_vec_step": round(ms * 1e3 / vs, 3)}
            out["traced"] = per
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("case", choices=["headline_1024", "batched_512", "3d_256", "3d_128", "stencil2d_1024",
                                     "figure3_ichol"])
    ap.add_argument("--nsamples", type=int, default=1)
    ap.add_argument("--steps", type=int, default=24)
    ap.add_argument("--trace", action="store_true", help="also report per-kernel-class times")
    a = ap.parse_args(argv)
    print(run(a.case, a.nsamples, a.steps, a.trace))


if __name__ == "__main__":
    main()
