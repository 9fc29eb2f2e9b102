// gmrf_api.cu -- the C ABI (include/gmrf.h) and the host driver.
//
// The driver validates arguments, sizes the device workspaces from free HBM,
// stages host buffers, and issues the kernels of one call on the problem's
// stream:
//   noise (Philox) or caller z  ->  ||z||                   (Algorithm 1, start)
//   repeat: fused Lanczos steps, c at a time, then one poll of the per-vector
//           convergence flags                              (Algorithm 1 loop, Theorem 1)
//   T_m^{-1/2} e_1 (rational approximation)  ->  x = ||z|| V_m y  (last step)
//   preconditioned problems: x = M^{-1/2} u                 (Proposition 1)
// Vectors that converge early stop doing work (their kernels exit at entry).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <cstdlib>
#include <cstring>
#include <new>
#include <algorithm>
#include <vector>

#include "host.h"

using namespace gmrf;
using namespace host;

namespace host {

// Workspaces are stream-ordered allocations on the problem's work stream, so
// growing or freeing them never synchronises the device (other problems keep
// running concurrently).
int ensure(DevBuf& b, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return GMRF_OK;
  if (b.p) cudaFreeAsync(b.p, s);
  b.p = nullptr;
  b.bytes = 0;
  if (cudaMallocAsync(&b.p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return GMRF_ERR_OOM;
  }
  b.bytes = bytes;
  return GMRF_OK;
}

void release(DevBuf& b, cudaStream_t s) {
  if (b.p) cudaFreeAsync(b.p, s);
  b.p = nullptr;
  b.bytes = 0;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace host

namespace host {

size_t esize(const gmrf_problem* p) { return p->fp64 ? 8 : 4; }

// A sparse problem with an incomplete-Cholesky factor: the sample and solve
// map their Lanczos result through F^{-T} (and the solve its start vector
// through F^{-1}).
bool sparse_f(const gmrf_problem* p) { return p->sp && sparse_has_factor(p->sp); }

// Order the work stream after the caller's stream (entry) and the caller's
// stream after the work stream (exit).
int enter(gmrf_problem* p) {
  if (p->server && !p->in_server) return GMRF_ERR_INVALID;  // the problem serves its server only
  CK(cudaEventRecord(p->ev_in, p->stream));
  CK(cudaStreamWaitEvent(p->ws, p->ev_in, 0));
  return GMRF_OK;
}
int leave(gmrf_problem* p) {
  CK(cudaEventRecord(p->ev_out, p->ws));
  CK(cudaStreamWaitEvent(p->stream, p->ev_out, 0));
  return GMRF_OK;
}

int ensure_host_states(gmrf_problem* p, int nvec) {
  if (p->st_host_cap >= nvec) return GMRF_OK;
  delete[] p->st_host;
  p->st_host = new (std::nothrow) VecState[nvec];
  p->st_host_cap = p->st_host ? nvec : 0;
  return p->st_host ? GMRF_OK : GMRF_ERR_OOM;
}

// Buffers for a batch of nvec vectors with nslots stored basis vectors each.
// bf16_basis: keep a bfloat16 copy of V_m ([nvec][m_max + 1][n]) for the
// assembly; the FP32 ring then has nslots = 2.
int ensure_lanczos(gmrf_problem* p, int nvec, int nslots, int m_max, bool need_tm, LanczosBufs& b,
                   bool bf16_basis) {
  const size_t n = p->g.n, es = esize(p);
  CKR(ensure(p->W0, (size_t)nvec * n * es, p->ws));
  CKR(ensure(p->W1, (size_t)nvec * n * es, p->ws));
  CKR(ensure(p->V, (size_t)nvec * nslots * n * es, p->ws));
  CKR(ensure(p->st, sizeof(VecState) * nvec, p->ws));
  CKR(ensure(p->alpha, sizeof(double) * nvec * m_max, p->ws));
  CKR(ensure(p->beta, sizeof(double) * nvec * m_max, p->ws));
  CKR(ensure(p->alpha_f, sizeof(float) * nvec * m_max, p->ws));
  CKR(ensure(p->beta2_f, sizeof(float) * nvec * m_max, p->ws));
  int nblk = std::max(stencil_blocks_per_vector(p->g), 256);
  nblk = std::max(nblk, precond_blocks_per_vector(p->pre));
  CKR(ensure(p->partials, (size_t)nvec * nblk * sizeof(Dots<double>), p->ws));
  const bool fresh_counters = p->counters.bytes < sizeof(unsigned) * nvec;
  CKR(ensure(p->counters, sizeof(unsigned) * nvec, p->ws));
  if (fresh_counters) CK(cudaMemsetAsync(p->counters.p, 0, sizeof(unsigned) * nvec, p->ws));
  CKR(ensure(p->nodes, sizeof(TmNodes) * nvec, p->ws));
  CKR(ensure(p->y, sizeof(double) * nvec * m_max, p->ws));
  CKR(ensure(p->q, sizeof(double) * nvec, p->ws));
  if (need_tm) CKR(ensure(p->scratch, sizeof(double) * 2 * (size_t)nvec * m_max * kMaxNodes, p->ws));
  CKR(ensure_host_states(p, nvec));
  b.W[0] = p->W0.p;
  b.W[1] = p->W1.p;
  b.V = p->V.p;
  b.Vb = nullptr;
  if (bf16_basis) {
    CKR(ensure(p->Vb, (size_t)nvec * (size_t)(m_max + 1) * n * sizeof(__nv_bfloat16), p->ws));
    b.Vb = (__nv_bfloat16*)p->Vb.p;
  }
  b.st = (VecState*)p->st.p;
  b.alpha = (double*)p->alpha.p;
  b.beta = (double*)p->beta.p;
  b.alpha_f = (float*)p->alpha_f.p;
  b.beta2_f = (float*)p->beta2_f.p;
  b.partials = p->partials.p;
  b.counters = (unsigned*)p->counters.p;
  b.nvec = nvec;
  b.nslots = nslots;
  b.m_max = m_max;
  return GMRF_OK;
}

// Vectors per batch that fit in free device memory.
int batch_size(gmrf_problem* p, int want, int nslots, int m_max, bool need_tm, size_t extra_per_vec) {
  size_t freeb = 0, total = 0;
  if (cudaMemGetInfo(&freeb, &total) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  // memory already held by this problem's workspace can be reused
  const size_t held = p->W0.bytes + p->W1.bytes + p->V.bytes + p->scratch.bytes + p->stage.bytes +
                      p->stage2.bytes + p->work.bytes + p->Vb.bytes;
  const size_t n = p->g.n, es = esize(p);
  size_t per = (size_t)(nslots + 2) * n * es + extra_per_vec + 64 * (size_t)m_max + 4096;
  if (need_tm) per += sizeof(double) * 2 * (size_t)m_max * kMaxNodes;
  const size_t budget = (size_t)((double)(freeb + held) * 0.85);
  size_t c = budget / per;
  if (c > (size_t)want) c = want;
  if (c > 65535) c = 65535;
  return (int)c;
}

// The z chunk is a tunable of the TMA-staged 3-D step only.
bool tune_zchunk_ok(const gmrf_problem* p) {
  return p->precond == GMRF_PREC_NONE && stencil3d_tma_eligible(p->g, p->fp64);
}

int worst_status(const VecState* st, int nvec) {
  int worst = GMRF_OK;
  for (int s = 0; s < nvec; ++s) {
    int c = st[s].status;
    if (c == VS_DONE) continue;
    if (c == VS_RUNNING) c = GMRF_ERR_NOT_CONVERGED;
    if (worst == GMRF_OK || (worst == GMRF_ERR_NOT_CONVERGED && c != GMRF_ERR_NOT_CONVERGED)) worst = c;
  }
  return worst;
}

// Runs the Lanczos iteration on the vectors already in W[0].  Returns a
// gmrf code for launch failures only; per-vector outcomes are in st_host.
int launch_steps(gmrf_problem* p, const LanczosBufs& b, const StepParams& P, int c, cudaStream_t s) {
  for (int k = 0; k < c; ++k) {
    if (p->sp)
      CK(traced(KC_SPARSE_STEP, s, 1, [&] { return launch_sparse_step(*p->sp, b, P, s); }));
    else if (p->precond == GMRF_PREC_NONE)
      CK(traced(KC_STENCIL_STEP, s, 1,
                [&] { return launch_stencil_step(p->g, p->fp64, p->kappa2.p, p->kappa2_const, b, P, s); }));
    else
      CK(launch_precond_step(p->pre, p->g, p->fp64, p->kappa2.p, p->kappa2_const, b, P, s));
    if (b.Xacc) CK(traced(KC_ASSEMBLE, s, 1, [&] { return launch_accumulate(p->fp64, p->g.n, b, s); }));
  }
  return GMRF_OK;
}

// The device-side Lanczos loop: a graph whose WHILE node repeats a body of c
// steps and a condition kernel until no vector is running, or for at most ceil(m_max/c)
// + 2 condition evaluations, a bound it never reaches.  A call then needs one
// launch and one host wait.  Returns GMRF_OK with G.exec == nullptr when the
// runtime cannot build it (the caller then replays c-step graphs).
int capture_loop(gmrf_problem* p, const LanczosBufs& b, const StepParams& P, int c) {
  StepGraph& G = p->graph;
  const void* S = p->precond ? p->pre.S : nullptr;
  if (G.exec && G.loop && G.nvec == b.nvec && G.nslots == b.nslots && G.m_max == P.m_max && G.c == c &&
      G.tol == P.tol &&
      G.W0 == b.W[0] && G.V == b.V && G.Vb == b.Vb && G.st == b.st && G.S == S && G.partials == b.partials &&
      !G.timed && G.zchunk == p->g.zchunk && G.Xacc == b.Xacc && G.xscale == b.xscale && G.solve == P.solve &&
      G.Xacc2 == b.Xacc2 && G.y1 == b.y && G.y2 == b.y2)
    return GMRF_OK;
  G.reset();
  CKR(ensure(p->loopctr, sizeof(int), p->ws));
  cudaStream_t s = p->ws;
  cudaGraph_t graph = nullptr;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) {
    cudaGetLastError();
    return GMRF_OK;
  }
  auto fail = [&]() {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    G.reset();
    return GMRF_OK;  // the replayed graphs serve instead
  };
  // The condition starts at 0 on every launch; a condition kernel ahead of the
  // WHILE node sets it (to 1 when some vector is running), and the one at the
  // end of the body sets it for the next iteration.  So the loop can only run
  // while the condition kernels run; the host checks the states afterwards.
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault) != cudaSuccess) return fail();
  cudaMemsetParams mp = {};
  mp.dst = p->loopctr.p;
  mp.value = 0;
  mp.elementSize = sizeof(int);
  mp.width = 1;
  mp.height = 1;
  cudaGraphNode_t reset_node;
  if (cudaGraphAddMemsetNode(&reset_node, graph, nullptr, 0, &mp) != cudaSuccess) return fail();
  const int limit = (P.m_max + c - 1) / c + 2;  // condition evaluations: one ahead, one per body
  void* kargs[5];
  const VecState* st_arg = b.st;
  int nvec_arg = b.nvec;
  int* ctr_arg = (int*)p->loopctr.p;
  int limit_arg = limit;
  kargs[0] = &h;
  kargs[1] = &st_arg;
  kargs[2] = &nvec_arg;
  kargs[3] = &ctr_arg;
  kargs[4] = &limit_arg;
  cudaKernelNodeParams kp = {};
  kp.func = const_cast<void*>(loop_cond_kernel());
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(256);
  kp.sharedMemBytes = 0;
  kp.kernelParams = kargs;
  cudaGraphNode_t first_cond;
  if (cudaGraphAddKernelNode(&first_cond, graph, &reset_node, 1, &kp) != cudaSuccess) return fail();
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop_node;
  if (cudaGraphAddNode(&loop_node, graph, &first_cond, nullptr, 1, &cp) != cudaSuccess) return fail();
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  trace_capture_begin(&G.tr);
  if (cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    trace_capture_end();
    return fail();
  }
  int r = launch_steps(p, b, P, c, s);
  if (r == GMRF_OK && traced(KC_OTHER, s, 1, [&] {
        return launch_loop_cond(h, b.st, b.nvec, (int*)p->loopctr.p, limit, s);
      }) != cudaSuccess)
    r = GMRF_ERR_CUDA;
  cudaGraph_t captured = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &captured);
  trace_capture_end();
  if (r != GMRF_OK || e != cudaSuccess) return fail();
  const cudaError_t ei = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    G.exec = nullptr;
    G.reset();
    return GMRF_OK;
  }
  G.loop = true;
  G.nvec = b.nvec;
  G.nslots = b.nslots;
  G.m_max = P.m_max;
  G.c = c;
  G.tol = P.tol;
  G.solve = P.solve;
  G.W0 = b.W[0];
  G.V = b.V;
  G.Vb = b.Vb;
  G.zchunk = p->g.zchunk;
  G.Xacc = b.Xacc;
  G.Xacc2 = b.Xacc2;
  G.y1 = b.y;
  G.y2 = b.y2;
  G.xscale = b.xscale;
  G.st = b.st;
  G.S = S;
  G.partials = b.partials;
  G.timed = false;
  G.kernels_per_step = (p->precond && !p->sp ? 5 : 1) + (b.Xacc ? 1 : 0);
  return GMRF_OK;
}

int capture_steps(gmrf_problem* p, const LanczosBufs& b, const StepParams& P, int c) {
  StepGraph& G = p->graph;
  const bool timed = trace_timing_enabled();
  const void* S = p->precond ? p->pre.S : nullptr;
  if (G.exec && !G.loop && G.nvec == b.nvec && G.nslots == b.nslots && G.m_max == P.m_max && G.c == c &&
      G.tol == P.tol &&
      G.W0 == b.W[0] && G.V == b.V && G.Vb == b.Vb && G.st == b.st && G.S == S && G.partials == b.partials &&
      G.timed == timed && G.zchunk == p->g.zchunk && G.Xacc == b.Xacc && G.xscale == b.xscale &&
      G.solve == P.solve && G.Xacc2 == b.Xacc2 && G.y1 == b.y && G.y2 == b.y2)
    return GMRF_OK;
  G.reset();
  cudaStream_t s = p->ws;
  cudaGraph_t graph = nullptr;
  trace_capture_begin(&G.tr);
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const int r = launch_steps(p, b, P, c, s);
  const cudaError_t e = cudaStreamEndCapture(s, &graph);
  trace_capture_end();
  if (r != GMRF_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    G.reset();
    return r != GMRF_OK ? r : GMRF_ERR_CUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    G.exec = nullptr;
    G.reset();
    return GMRF_ERR_CUDA;
  }
  G.nvec = b.nvec;
  G.nslots = b.nslots;
  G.m_max = P.m_max;
  G.c = c;
  G.tol = P.tol;
  G.solve = P.solve;
  G.W0 = b.W[0];
  G.V = b.V;
  G.Vb = b.Vb;
  G.zchunk = p->g.zchunk;
  G.Xacc = b.Xacc;
  G.Xacc2 = b.Xacc2;
  G.y1 = b.y;
  G.y2 = b.y2;
  G.xscale = b.xscale;
  G.st = b.st;
  G.S = S;
  G.partials = b.partials;
  G.timed = timed;
  G.loop = false;
  G.kernels_per_step = (p->precond && !p->sp ? 5 : 1) + (b.Xacc ? 1 : 0);
  return GMRF_OK;
}

// init = false continues the vectors whose states were set running again
// (their bases, q and recurrence state are still in place).
StepParams step_params(gmrf_problem* p, const LanczosBufs& b, double tol, int m_max, bool solve) {
  StepParams P{};
  P.m_max = m_max;
  P.nslots = b.nslots;
  P.solve = solve ? 1 : 0;
  P.tol = tol;
  P.bd_tol = p->fp64 ? 1e-13 : 1e-6;
  P.vb = b.Vb;
  return P;
}

int run_lanczos(gmrf_problem* p, const LanczosBufs& b, double tol, int m_max, int check_every,
                bool solve, bool init) {
  cudaStream_t s = p->ws;
  if (init) CK(traced(KC_INIT, s, 1, [&] { return launch_lanczos_init(p->fp64, p->g.n, b, s); }));
  const StepParams P = step_params(p, b, tol, m_max, solve);
  const int c = std::min(check_every > 0 ? check_every : 16, m_max);
  if (p->precond != GMRF_PREC_NONE) CKR(precond_prepare(p->pre, b.nvec, s));
  StepGraph& G = p->graph;
  if (!trace_timing_enabled() && !p->host_loop) {
    // the device-side loop: one launch, one wait.  Its body runs at most 8
    // steps: each WHILE iteration costs a few microseconds (the condition
    // kernel and the body's launch), and a shorter body wastes fewer steps
    // after the last vector stops (1024^2 headline: 4.24 ms per sample with
    // 8-step bodies, 4.32 with 16, 4.60 with 1, 4.28 host-replayed).
    CKR(capture_loop(p, b, P, std::min(c, 8)));
    if (G.exec) {
      int iters = 0;
      CK(cudaGraphLaunch(G.exec, s));
      CK(cudaMemcpyAsync(&iters, p->loopctr.p, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(p->st_host, b.st, sizeof(VecState) * b.nvec, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      // launch counts: the condition kernel ahead of the loop, then each
      // iteration of the body (the counter holds both)
      trace_begin(KC_OTHER, s, 1);
      trace_end(KC_OTHER, s);
      for (int k = 1; k < iters; ++k) trace_replayed(&G.tr, 0);
      bool running = false;
      for (int v = 0; v < b.nvec; ++v) running |= (p->st_host[v].status == VS_RUNNING);
      if (!running) return GMRF_OK;
      // not expected: the replayed graphs finish whatever is still running
    }
  }
  CKR(capture_steps(p, b, P, c));
  int j = 0;
  while (j < m_max) {
    CK(cudaGraphLaunch(G.exec, s));
    CK(cudaMemcpyAsync(p->st_host, b.st, sizeof(VecState) * b.nvec, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bool running = false;
    int mmax = 0;
    for (int v = 0; v < b.nvec; ++v) {
      running |= (p->st_host[v].status == VS_RUNNING);
      mmax = std::max(mmax, p->st_host[v].m);
    }
    // steps of this replay in which some vector still iterated
    const int useful = std::max(0, std::min(c, mmax - j));
    trace_replayed(&G.tr, useful * G.kernels_per_step);
    j += c;
    if (!running) break;
  }
  return GMRF_OK;
}

// The vectors [off, off + cnt) of a Lanczos batch as a batch of their own
// (the T_m functions and the assembly of a mixed batch of samples and probes).
LanczosBufs sub_batch(const LanczosBufs& b, int off, int cnt, size_t n, size_t es) {
  LanczosBufs r = b;
  const size_t vo = (size_t)off * n * es;
  r.W[0] = (char*)b.W[0] + vo;
  r.W[1] = (char*)b.W[1] + vo;
  r.V = (char*)b.V + vo * b.nslots;
  r.Vb = nullptr;
  r.st = b.st + off;
  r.alpha = b.alpha + (size_t)off * b.m_max;
  r.beta = b.beta + (size_t)off * b.m_max;
  r.alpha_f = b.alpha_f + (size_t)off * b.m_max;
  r.beta2_f = b.beta2_f + (size_t)off * b.m_max;
  r.nvec = cnt;
  return r;
}

// ---- accuracy check of samples ------------------------------------------
// Theorem 1 bounds the error of x_m by lambda_min^{-1/2} ||r_m||, with
// r_m = z - A u_m the residual of the CG iterate u_m = ||z|| V_m T_m^{-1} e_1
// (A the iterated operator), and in exact arithmetic the recurrence gives
// ||r_m|| without forming u_m.  In finite precision the recurrence keeps
// shrinking while the residual of the computed u_m stops where the rounding of
// the applies of A leaves it.  So after the iteration the library forms u_m
// (in the same pass over V_m as x_m), computes r = z - A u_m directly (for an
// FP32 stencil in pairs of floats, since its products cancel heavily on a
// smooth u_m; in the problem's precision otherwise) and one product t = A r in
// the problem's precision (r no longer cancels), and estimates
//     est_direct = sqrt(r^T A^{-1} r) / ||x_m||,
// the square root of the quadratic form taken from the two-node Gauss-Radau
// rule of the Lanczos step from r with the node fixed at theta_min (Golub and
// Meurant: an upper estimate for 1/t when the node is at most lambda_min).
// In exact arithmetic this is at most the Theorem 1 estimate, since
// r^T A^{-1} r <= ||r||^2 / lambda_min; with rounding it follows where the
// residual actually sits in the spectrum (rounding noise in the high modes
// weighs little, as it does in the error of x_m).  A vector is GMRF_OK only
// if both estimates are <= tol; err_est reports the larger.

// Bytes per vector of the check's buffers: z, u_cg and r in the problem's
// precision (t = A r goes into u_cg's buffer).
size_t check_bytes_per_vec(const gmrf_problem* p) {
  const size_t n = p->g.n, es = esize(p);
  return 3 * n * es;  // z, u and r
}

// T_m^{-1} e_1 of the nvec vectors of b into p->ycg (stride m_max).
int check_tm(gmrf_problem* p, const LanczosBufs& b, cudaStream_t s) {
  CKR(ensure(p->ycg, sizeof(double) * 2 * (size_t)b.nvec * b.m_max, p->ws));
  double* ycg = (double*)p->ycg.p;
  CK(traced(KC_TM, s, 1, [&] { return launch_tm_inv(b, ycg + (size_t)b.nvec * b.m_max, ycg, s); }));
  return GMRF_OK;
}

// For nvec vectors z, u [nvec][n] (problem precision, device): r = z - A u
// with A the iterated operator (tau-free); with second = false writes
// (r.r, r.r, r.r) to p->rn[3 s .. 3 s + 2], with second = true also t = A r
// into u and (r.r, r.t, t.t) (r kept from the first call).  u is overwritten
// by the second call.
int check_residuals(gmrf_problem* p, int nvec, const void* z, void* u, bool second, cudaStream_t s) {
  const size_t n = p->g.n, es = esize(p), cnt = (size_t)nvec * n;
  CKR(ensure(p->chk, (size_t)nvec * (check_bytes_per_vec(p) - 2 * n * es), p->ws));
  CKR(ensure(p->rn, (sizeof(double) * 3 + sizeof(Dots<double>) * kResidBlocks) * (size_t)nvec, p->ws));
  double* out = (double*)p->rn.p;
  void* part = out + 3 * (size_t)nvec;
  auto apply = [&](const void* in, void* res) -> cudaError_t {
    if (p->sp) return launch_sparse_ops(*p->sp, sparse_f(p) ? 1 : 0, in, res, nvec, s);  // A, or Q without F
    if (p->precond != GMRF_PREC_NONE)
      return launch_precond_operator(p->pre, p->g, p->fp64, p->kappa2.p, p->kappa2_const, in, res, nvec, s);
    return launch_stencil_apply(p->g, p->fp64, p->kappa2.p, p->kappa2_const, in, res, nvec, s);
  };
  const int kl = p->sp ? 1 : (p->precond != GMRF_PREC_NONE ? 5 : 1);
  // FP32 lattice without a preconditioner: r = z - Q u formed in pairs of
  // floats (the stencil's own terms cancel on a smooth u)
  const bool df_resid = !p->sp && p->precond == GMRF_PREC_NONE && !p->fp64;
  void* r = p->chk.p;
  if (!second) {
    if (df_resid) {
      CK(traced(KC_PRE_APPLY, s, 2, [&] {
        return launch_resid_df(p->g, (const float*)p->kappa2.p, p->kappa2_const, (const float*)z, (const float*)u,
                               (float*)r, nvec, part, out, s);
      }));
    } else {
      CK(traced(KC_PRE_APPLY, s, kl, [&] { return apply(u, r); }));
      CK(traced(KC_OTHER, s, 1, [&] { return launch_resid_form(p->fp64, z, p->fp64, r, cnt, s); }));
      CK(traced(KC_OTHER, s, 2, [&] { return launch_dots3(p->fp64, r, r, n, nvec, part, out, s); }));
    }
  } else {
    // t = A r into u's buffer (u is not needed after r)
    CK(traced(KC_PRE_APPLY, s, kl, [&] { return apply(r, u); }));
    CK(traced(KC_OTHER, s, 2, [&] { return launch_dots3(p->fp64, r, u, n, nvec, part, out, s); }));
  }
  return GMRF_OK;
}

// Theorem 1's form with the direct residual, theta_min^{-1/2} ||r|| / ||x_m||
// (an upper estimate of est_direct), INFINITY when it cannot be formed.
double crude_estimate(const VecState& v, double rr) {
  const double xnorm = v.znorm * std::sqrt(v.energy);
  if (!(xnorm > 0.0) || !(v.theta > 0.0) || !std::isfinite(rr)) return INFINITY;
  const double e = std::sqrt(std::max(rr, 0.0) / v.theta) / xnorm;
  return std::isfinite(e) ? e : INFINITY;
}

// The direct estimates of nvec vectors after their assembly: z, u as for
// check_residuals, states on the device (copied to hst).  est[s] is Theorem
// 1's form with the direct residual where that is already <= tol, else the
// Gauss-Radau est_direct (a second product A r, run for the batch only when
// some vector needs it); each vector's value depends only on that vector.
int check_vectors(gmrf_problem* p, int nvec, const void* z, void* u, const VecState* st_dev, VecState* hst,
                  double tol, double* est, cudaStream_t s) {
  std::vector<double> d3((size_t)3 * nvec);
  CKR(check_residuals(p, nvec, z, u, false, s));
  CK(cudaMemcpyAsync(d3.data(), p->rn.p, sizeof(double) * 3 * nvec, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hst, st_dev, sizeof(VecState) * nvec, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  bool second = false;
  for (int i = 0; i < nvec; ++i) {
    est[i] = crude_estimate(hst[i], d3[3 * i]);
    const bool checked = (hst[i].status == VS_DONE || hst[i].status == GMRF_ERR_NOT_CONVERGED) && hst[i].m > 0;
    if (checked && !(est[i] <= tol)) second = true;
  }
  if (!second) return GMRF_OK;
  CKR(check_residuals(p, nvec, z, u, true, s));
  CK(cudaMemcpyAsync(d3.data(), p->rn.p, sizeof(double) * 3 * nvec, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < nvec; ++i)
    if (!(est[i] <= tol)) est[i] = direct_estimate(hst[i], d3.data() + 3 * i);
  return GMRF_OK;
}

// est_direct of a vector from (r.r, r.t, t.t) and its state (INFINITY when
// it cannot be formed).
double direct_estimate(const VecState& v, const double* d3) {
  const double rr = d3[0];
  const double xnorm = v.znorm * std::sqrt(v.energy);
  if (!(xnorm > 0.0) || !std::isfinite(rr)) return INFINITY;
  if (rr <= 0.0) return 0.0;
  const double a1 = d3[1] / rr;                            // Rayleigh quotient of r
  const double b2 = std::max(d3[2] / rr - a1 * a1, 0.0);  // beta_1^2 of the step from r
  const double node = v.theta;
  double q;  // estimate of r^T A^{-1} r / r^T r
  if (!(node > 0.0)) return INFINITY;
  if (a1 > node * (1.0 + 1e-12)) {
    const double omega = node + b2 / (a1 - node);
    q = omega / (a1 * omega - b2);
  } else {
    q = 1.0 / std::max(std::min(a1, node), 1e-300);
  }
  const double est = std::sqrt(rr * q) / xnorm;
  return std::isfinite(est) ? est : INFINITY;
}

// After a check: vectors that stopped on the recurrence estimate (status
// done, err_est > 0) while est_direct > tol are set running again with a
// minimum step count m + max(2, m / 8) (in mmin and the state), when more
// steps can help: est_direct within 20 tol in the first round, falling by 30 %
// per round after it, at most 3 rounds, m below m_max.  A direct estimate far
// above tol, or one that stopped falling, is the floor of the arithmetic: the
// vector keeps its result and the check reports it.  Returns whether any
// vector was resumed.
bool check_resume(VecState* st, const double* est, const double* est_prev, int* mmin, int nvec, double tol, int m_max,
                  int round) {
  bool any = false;
  for (int s = 0; s < nvec; ++s) {
    VecState& v = st[s];
    if (round >= 3 || v.status != VS_DONE || v.m == 0 || !(v.err_est > 0.0) || v.m >= m_max) continue;
    const double e = est[s];
    if (e <= tol) continue;
    const bool progress = round == 0 ? e <= 20.0 * tol : e <= 0.7 * est_prev[s];
    if (!progress) continue;
    v.m_min = std::min(m_max, v.m + std::max(2, v.m / 8));
    v.status = VS_RUNNING;
    mmin[s] = v.m_min;
    any = true;
  }
  return any;
}

// Host side: the direct estimates folded into the states.
void check_apply(VecState* st, const double* est, int nvec, double tol) {
  for (int s = 0; s < nvec; ++s) {
    VecState& v = st[s];
    if (!(v.status == VS_DONE || v.status == GMRF_ERR_NOT_CONVERGED) || v.m == 0) continue;
    const double e = est[s];
    if (!(v.err_est >= e)) v.err_est = e;
    if (v.status == VS_DONE && !(e <= tol)) v.status = GMRF_ERR_NOT_CONVERGED;
  }
}

void fill_info(const VecState* st, int nvec, gmrf_result_info* info) {
  if (!info) return;
  for (int s = 0; s < nvec; ++s) {
    info[s].m_used = st[s].m;
    int c = st[s].status;
    if (c == VS_DONE) c = GMRF_OK;
    if (c == VS_RUNNING) c = GMRF_ERR_NOT_CONVERGED;
    info[s].status = c;
    info[s].err_est = st[s].err_est;
  }
}

}  // namespace host

extern "C" {

const char* gmrf_strerror(int code) {
  switch (code) {
    case GMRF_OK: return "ok";
    case GMRF_ERR_INVALID: return "invalid argument";
    case GMRF_ERR_OOM: return "out of device memory";
    case GMRF_ERR_NOT_CONVERGED: return "not converged within m_max";
    case GMRF_ERR_NOT_SPD: return "operator is not symmetric positive definite";
    case GMRF_ERR_NUMERIC: return "non-finite value during the iteration";
    case GMRF_ERR_CUDA: return "CUDA runtime error";
    case GMRF_ERR_TIMEOUT: return "device wait timed out";
    case GMRF_ERR_UNSUPPORTED: return "unsupported combination";
    default: return "unknown error";
  }
}

int gmrf_size(const gmrf_problem* p, int64_t* n) {
  if (!p || !n) return GMRF_ERR_INVALID;
  *n = (int64_t)p->g.n;
  return GMRF_OK;
}

int gmrf_create(const gmrf_desc* d, void* stream, gmrf_problem** out) {
  if (!d || !out) return GMRF_ERR_INVALID;
  *out = nullptr;
  if (d->dim != 2 && d->dim != 3) return GMRF_ERR_INVALID;
  if (d->bc < 0 || d->bc > 2 || d->op < 0 || d->op > 2 || d->precond < 0 || d->precond > 2) return GMRF_ERR_INVALID;
  if (d->precision != GMRF_FP32 && d->precision != GMRF_FP64) return GMRF_ERR_INVALID;
  if (d->reserved != 0) return GMRF_ERR_INVALID;
  if (d->nx < 2 || d->ny < 2 || (d->dim == 3 && d->nz < 2)) return GMRF_ERR_INVALID;
  if (d->nx > (1 << 30) || d->ny > (1 << 30) || (d->dim == 3 && d->nz > (1 << 30))) return GMRF_ERR_INVALID;
  if (!(d->tau > 0.0) || !std::isfinite(d->tau)) return GMRF_ERR_INVALID;
  const int64_t nz = d->dim == 3 ? d->nz : 1;
  const double nd = (double)d->nx * (double)d->ny * (double)nz;
  if (nd > 4.0e9) return GMRF_ERR_INVALID;
  const bool plus_diag = d->op == GMRF_OP_SPDE_PLUS_DIAG;
  if ((!d->kappa2 || plus_diag) && (!(d->kappa2_const >= 0.0) || !std::isfinite(d->kappa2_const)))
    return GMRF_ERR_INVALID;
  // a constant kappa^2 = 0 leaves the constant vector in the null space unless the boundary is Dirichlet
  if ((!d->kappa2 || plus_diag) && d->bc != GMRF_BC_DIRICHLET && !(d->kappa2_const > 0.0)) return GMRF_ERR_INVALID;
  if (d->dim == 3 && d->op != GMRF_OP_SHIFTED_LAPLACIAN) return GMRF_ERR_UNSUPPORTED;
  if (d->precond != GMRF_PREC_NONE) {
    if (d->dim != 2) return GMRF_ERR_UNSUPPORTED;
    if (!precond_size_ok(d->nx) || !precond_size_ok(d->ny)) return GMRF_ERR_UNSUPPORTED;
    if (!(d->kappa2_precond <= 0.0 || std::isfinite(d->kappa2_precond))) return GMRF_ERR_INVALID;
    if (plus_diag) {
      // M is the prior itself: R = tau D is diagonal only with matched boundaries and kappa_bar = kappa_c
      const bool matched = (d->precond == GMRF_PREC_CIRCULANT && d->bc == GMRF_BC_PERIODIC) ||
                           (d->precond == GMRF_PREC_MIRROR && d->bc == GMRF_BC_NEUMANN);
      if (!matched || (d->kappa2_precond > 0.0 && d->kappa2_precond != d->kappa2_const))
        return GMRF_ERR_UNSUPPORTED;
    }
  }
  gmrf_problem* p = new (std::nothrow) gmrf_problem();
  if (!p) return GMRF_ERR_OOM;
  p->g.dim = d->dim;
  p->g.nx = (int)d->nx;
  p->g.ny = (int)d->ny;
  p->g.nz = (int)nz;
  p->g.n = (size_t)d->nx * d->ny * nz;
  p->g.bc = d->bc;
  p->g.op = d->op;
  p->precond = d->precond;
  p->fp64 = d->precision == GMRF_FP64;
  p->tau = d->tau;
  p->kappa2_const = d->kappa2_const;
  p->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return GMRF_ERR_CUDA;
  }
  auto fail = [&](int code) {
    gmrf_destroy(p);
    return code;
  };
  {
    // keep freed workspace in this process's default memory pool (no trim at
    // every synchronisation), once per device
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
      std::lock_guard<std::mutex> lock(mu);
      cudaMemPool_t pool;
      if (!done[dev] && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        done[dev] = true;
      }
    }
    cudaGetLastError();
  }
  if (cudaStreamCreateWithFlags(&p->ws, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(GMRF_ERR_CUDA);
  }
  if (enter(p) != GMRF_OK) return fail(GMRF_ERR_CUDA);
  double sum_log = 0.0, nzero = 0.0;
  if (d->kappa2) {
    if (ensure(p->kappa2, sizeof(float) * p->g.n, p->ws) != GMRF_OK) return fail(GMRF_ERR_OOM);
    const cudaMemcpyKind kind = is_device_ptr(d->kappa2) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(p->kappa2.p, d->kappa2, sizeof(float) * p->g.n, kind, p->ws) != cudaSuccess)
      return fail(GMRF_ERR_CUDA);
    DevBuf stats;
    if (ensure(stats, kFieldStatsBytes, p->ws) != GMRF_OK) return fail(GMRF_ERR_OOM);
    double h[4] = {0, 0, 0, 0};
    trace_begin(KC_OTHER, p->ws, 2);
    bool ok = launch_field_stats((const float*)p->kappa2.p, p->g.n, (double*)stats.p, p->ws) == cudaSuccess;
    trace_end(KC_OTHER, p->ws);
    ok = ok && cudaMemcpyAsync(h, stats.p, sizeof(h), cudaMemcpyDeviceToHost, p->ws) == cudaSuccess &&
         cudaStreamSynchronize(p->ws) == cudaSuccess;
    release(stats, p->ws);
    if (!ok) return fail(GMRF_ERR_CUDA);
    if (h[0] > 0.5) return fail(GMRF_ERR_INVALID);
    nzero = h[1];
    sum_log = h[2];
    // (K + L) with K = 0 is singular without a Dirichlet boundary; the diagonal
    // of SPDE_PLUS_DIAG may vanish (kappa_c^2 > 0 was checked)
    if (!plus_diag && d->bc != GMRF_BC_DIRICHLET && nzero > (double)p->g.n - 0.5) return fail(GMRF_ERR_INVALID);
  } else {
    if (d->bc != GMRF_BC_DIRICHLET && !(d->kappa2_const > 0.0)) return fail(GMRF_ERR_INVALID);
    sum_log = d->kappa2_const > 0 ? (double)p->g.n * std::log(d->kappa2_const) : 0.0;
    nzero = d->kappa2_const > 0 ? 0.0 : (double)p->g.n;
  }
  if (d->precond != GMRF_PREC_NONE) {
    double kb = plus_diag ? d->kappa2_const : d->kappa2_precond;
    if (!(kb > 0.0)) {
      const double npos = (double)p->g.n - nzero;
      kb = npos > 0.5 ? std::exp(sum_log / npos) : 0.0;
    }
    if (!(kb > 0.0) && d->precond != GMRF_PREC_NONE && d->bc != GMRF_BC_DIRICHLET) return fail(GMRF_ERR_INVALID);
    if (!(kb > 0.0)) return fail(GMRF_ERR_INVALID);
    p->kbar2 = kb;
    const int r = precond_build(p->pre, p->g, d->precond, d->op, kb, p->fp64, p->ws, &p->logdet_M);
    if (r != GMRF_OK) return fail(r);
  }
  if (leave(p) != GMRF_OK || cudaStreamSynchronize(p->ws) != cudaSuccess) return fail(GMRF_ERR_CUDA);
  trace_collect();
  *out = p;
  return GMRF_OK;
}

int gmrf_create_sparse(const gmrf_sparse_desc* d, void* stream, gmrf_problem** out) {
  if (!d || !out) return GMRF_ERR_INVALID;
  *out = nullptr;
  if (d->precision != GMRF_FP32 && d->precision != GMRF_FP64) return GMRF_ERR_INVALID;
  if (d->reserved != 0 || !(d->tau > 0.0) || !std::isfinite(d->tau)) return GMRF_ERR_INVALID;
  if (!d->rowptr || !d->colind || !d->val || d->n < 1) return GMRF_ERR_INVALID;
  if (d->f_rowptr && (!d->f_colind || !d->f_val)) return GMRF_ERR_INVALID;
  gmrf_problem* p = new (std::nothrow) gmrf_problem();
  if (!p) return GMRF_ERR_OOM;
  // the lattice fields describe a 1-D index space of n cells (no stencil is used)
  p->g.dim = 1;
  p->g.nx = (int)std::min<int64_t>(d->n, 1 << 30);
  p->g.ny = 1;
  p->g.nz = 1;
  p->g.n = (size_t)d->n;
  p->g.bc = GMRF_BC_DIRICHLET;
  p->g.op = GMRF_OP_SHIFTED_LAPLACIAN;
  p->precond = GMRF_PREC_NONE;
  p->fp64 = d->precision == GMRF_FP64;
  p->tau = d->tau;
  p->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return GMRF_ERR_CUDA;
  }
  auto fail = [&](int code) {
    gmrf_destroy(p);
    return code;
  };
  if (cudaStreamCreateWithFlags(&p->ws, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(GMRF_ERR_CUDA);
  }
  if (enter(p) != GMRF_OK) return fail(GMRF_ERR_CUDA);
  double ldf = 0.0;
  const int r = sparse_create(&p->sp, d, p->fp64, p->ws, &ldf);
  if (r != GMRF_OK) return fail(r);
  p->logdet_M = ldf;  // log det(F F^T); 0 without F
  if (leave(p) != GMRF_OK || cudaStreamSynchronize(p->ws) != cudaSuccess) return fail(GMRF_ERR_CUDA);
  *out = p;
  return GMRF_OK;
}

void gmrf_destroy(gmrf_problem* p) {
  if (!p) return;
  async_shutdown(p);  // submitted calls finish first
  if (p->server) gmrf_server_destroy(p->server);
  if (p->ws) cudaStreamSynchronize(p->ws);
  p->graph.reset();
  DevBuf* bufs[] = {&p->kappa2, &p->W0, &p->W1, &p->V, &p->st, &p->alpha, &p->beta, &p->alpha_f, &p->beta2_f,
                    &p->partials, &p->counters, &p->y, &p->scratch, &p->nodes, &p->q, &p->out2, &p->stage,
                    &p->stage2, &p->work, &p->Vb, &p->xacc, &p->accn, &p->solvew, &p->ycg, &p->ucg,
                    &p->xacc2, &p->chk, &p->rn, &p->zre, &p->mmin, &p->loopctr};
  for (DevBuf* b : bufs) release(*b, p->ws);
  precond_free(p->pre, p->ws);
  sparse_free(p->sp, p->ws);
  p->sp = nullptr;
  if (p->ws) cudaStreamSynchronize(p->ws);
  delete[] p->st_host;
  if (p->ev_in) cudaEventDestroy(p->ev_in);
  if (p->ev_out) cudaEventDestroy(p->ev_out);
  if (p->ws) cudaStreamDestroy(p->ws);
  delete p;
}

int gmrf_sample(gmrf_problem* p, const gmrf_sample_opts* o, void* x_out, gmrf_result_info* info) {
  if (!p || !o || !x_out) return GMRF_ERR_INVALID;
  if (!(o->tol > 0.0) || !std::isfinite(o->tol) || o->m_max < 1 || o->m_max > 8192 || o->nsamples < 1 ||
      (o->v_storage != GMRF_VSTORE_NATIVE && o->v_storage != GMRF_VSTORE_BF16 &&
       o->v_storage != GMRF_VSTORE_NONE))
    return GMRF_ERR_INVALID;
  const bool bf16 = o->v_storage == GMRF_VSTORE_BF16;
  const bool two_pass = o->v_storage == GMRF_VSTORE_NONE;
  if (bf16 && p->fp64) return GMRF_ERR_UNSUPPORTED;
  if (p->sp && o->v_storage != GMRF_VSTORE_NATIVE) return GMRF_ERR_UNSUPPORTED;
  const size_t n = p->g.n, es = esize(p);
  const int m_max = o->m_max;
  const int nslots = (bf16 || two_pass) ? 2 : m_max + 1;
  const bool x_dev = is_device_ptr(x_out);
  const bool z_dev = o->z_in && is_device_ptr(o->z_in);
  const size_t extra = (x_dev ? 0 : n * es) + (p->precond ? precond_extra_bytes(p->pre, es) : 0) +
                       (sparse_f(p) ? n * es : 0) + (bf16 ? (size_t)(m_max + 1) * n * sizeof(__nv_bfloat16) : 0) +
                       (two_pass ? 2 * 2 * n * sizeof(float) + (p->precond ? n * es : 0) : 0) +
                       check_bytes_per_vec(p);
  int chunk = batch_size(p, o->nsamples, nslots, m_max, true, extra);
  if (p->tune_bw > 0 && chunk > p->tune_bw) chunk = p->tune_bw;
  if (chunk < 1) return GMRF_ERR_OOM;
  cudaStream_t s = p->ws;
  CKR(enter(p));
  std::vector<VecState> all((size_t)o->nsamples);
  for (int s0 = 0; s0 < o->nsamples; s0 += chunk) {
    const int c = std::min(chunk, o->nsamples - s0);
    LanczosBufs b;
    CKR(ensure_lanczos(p, c, nslots, m_max, true, b, bf16));
    CKR(ensure(p->ucg, (size_t)c * n * es, p->ws));
    CKR(ensure(p->zre, (size_t)c * n * es, p->ws));
    CKR(ensure(p->mmin, sizeof(int) * c, p->ws));
    CK(cudaMemsetAsync(p->mmin.p, 0, sizeof(int) * c, s));
    b.m_min = (const int*)p->mmin.p;
    auto load_z = [&](void* dst) -> int {
      if (o->z_in) {
        const char* src = (const char*)o->z_in + (size_t)s0 * n * es;
        CK(cudaMemcpyAsync(dst, src, (size_t)c * n * es, z_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           s));
      } else {
        CK(traced(KC_RNG, s, 1, [&] { return launch_rng(0, p->fp64, c, (int64_t)n, o->seed, s0, dst, s); }));
      }
      return GMRF_OK;
    };
    void* xdst = (char*)x_out + (size_t)s0 * n * es;
    if (!x_dev) {
      CKR(ensure(p->stage, (size_t)c * n * es, p->ws));
      xdst = p->stage.p;
    }
    CKR(load_z(p->zre.p));  // z for the accuracy check (kept: W[0] becomes a q buffer)
    std::vector<double> est((size_t)c), est_prev((size_t)c, 0.0);
    std::vector<int> mmin((size_t)c, 0);
    CKR(load_z(b.W[0]));
    CKR(run_lanczos(p, b, o->tol, m_max, o->check_every));
    for (int round = 0;; ++round) {
      CK(traced(KC_TM, s, 3, [&] {
        return launch_tm_inv_sqrt(b, p->fp64, (TmNodes*)p->nodes.p, (double*)p->scratch.p, (double*)p->y.p, s);
      }));
      CKR(check_tm(p, b, s));
      LanczosBufs bx = b;
      if (two_pass) {
        // second pass: the same iteration again (bitwise: same z, same kernels,
        // same step counts), adding ||z|| y_j v_j to x (and the check's u_cg)
        // after every step instead of keeping V_m
        const size_t xb = (size_t)c * n * (p->fp64 ? sizeof(double) : 2 * sizeof(float));
        CKR(ensure(p->xacc, xb, p->ws));
        CKR(ensure(p->xacc2, xb, p->ws));
        CKR(ensure(p->accn, sizeof(int) * c, p->ws));
        CK(cudaMemsetAsync(p->xacc.p, 0, xb, s));
        CK(cudaMemsetAsync(p->xacc2.p, 0, xb, s));
        CK(cudaMemsetAsync(p->accn.p, 0, sizeof(int) * c, s));
        bx.Xacc = p->xacc.p;
        bx.acc = (int*)p->accn.p;
        bx.y = (const double*)p->y.p;
        bx.xscale = p->precond == GMRF_PREC_NONE ? 1.0 / std::sqrt(p->tau) : 1.0;
        bx.Xacc2 = p->xacc2.p;
        bx.y2 = (const double*)p->ycg.p;
        CKR(load_z(b.W[0]));
        CKR(run_lanczos(p, bx, o->tol, m_max, o->check_every));
      }
      // x_m = ||z|| V_m y (one pass) or the accumulated sum (two passes), and
      // with it the check's u_cg = ||z|| V_m T_m^{-1} e_1
      auto assemble = [&](double extra, void* dst) -> cudaError_t {
        if (two_pass) {
          const cudaError_t e = launch_accumulate_finish(p->fp64, n, bx, p->xacc2.p, p->ucg.p, s);
          return e != cudaSuccess ? e : launch_accumulate_finish(p->fp64, n, bx, p->xacc.p, dst, s);
        }
        return launch_assemble_dual(p->fp64, n, b, (double*)p->y.p, m_max, extra, dst, (const double*)p->ycg.p,
                                    p->ucg.p, s);
      };
      if (sparse_f(p)) {
        // u = ||z|| V_m y, then x = tau^{-1/2} F^{-T} u (Proposition 1 with M = F F^T)
        CKR(ensure(p->work, (size_t)c * n * es, p->ws));
        CK(traced(KC_ASSEMBLE, s, 1, [&] { return assemble(1.0, p->work.p); }));
        CK(traced(KC_PRE_APPLY, s, 1, [&] { return launch_sparse_ops(*p->sp, 2, p->work.p, xdst, c, s); }));
        CK(traced(KC_OTHER, s, 1,
                  [&] { return launch_scale(p->fp64, xdst, (size_t)c * n, 1.0 / std::sqrt(p->tau), s); }));
      } else if (p->precond == GMRF_PREC_NONE) {
        CK(traced(KC_ASSEMBLE, s, 1, [&] { return assemble(1.0 / std::sqrt(p->tau), xdst); }));
      } else {
        // u = ||z|| V_m y, then x = M^{-1/2} u = tau^{-1/2} B_bar^{-p/2} u (Proposition 1)
        CKR(ensure(p->work, (size_t)c * n * es, p->ws));
        CK(traced(KC_ASSEMBLE, s, 1, [&] { return assemble(1.0, p->work.p); }));
        CK(traced(KC_PRE_APPLY, s, 3, [&] {
          return launch_precond_apply(p->pre, p->g, p->fp64, PRE_INV_SQRT, p->work.p, xdst, c, s);
        }));
        CK(traced(KC_OTHER, s, 1,
                  [&] { return launch_scale(p->fp64, xdst, (size_t)c * n, 1.0 / std::sqrt(p->tau), s); }));
      }
      // accuracy check: the direct residual r = z - A u_cg
      CKR(check_vectors(p, c, p->zre.p, p->ucg.p, b.st, p->st_host, o->tol, est.data(), s));
      trace_collect();
      // vectors whose recurrence estimate met tol but whose direct estimate did
      // not, by a margin more steps can close, continue for more steps
      if (!check_resume(p->st_host, est.data(), est_prev.data(), mmin.data(), c, o->tol, m_max, round)) break;
      est_prev = est;
      if (two_pass) {
        // rerun both passes from z with the new minimum step counts (the
        // other vectors repeat their steps bitwise)
        CK(cudaMemcpyAsync(p->mmin.p, mmin.data(), sizeof(int) * c, cudaMemcpyHostToDevice, s));
        CKR(load_z(b.W[0]));
        CKR(run_lanczos(p, b, o->tol, m_max, o->check_every));
      } else {
        // continue the resumed vectors in place (their states now RUNNING)
        CK(cudaMemcpyAsync(b.st, p->st_host, sizeof(VecState) * c, cudaMemcpyHostToDevice, s));
        CKR(run_lanczos(p, b, o->tol, m_max, o->check_every, false, false));
      }
    }
    check_apply(p->st_host, est.data(), c, o->tol);
    if (!x_dev)
      CK(cudaMemcpyAsync((char*)x_out + (size_t)s0 * n * es, xdst, (size_t)c * n * es, cudaMemcpyDeviceToHost, s));
    std::memcpy(all.data() + s0, p->st_host, sizeof(VecState) * c);
  }
  CK(cudaStreamSynchronize(s));
  CKR(leave(p));
  fill_info(all.data(), o->nsamples, info);
  return worst_status(all.data(), o->nsamples);
}

int gmrf_solve(gmrf_problem* p, const gmrf_solve_opts* o, const void* b_in, void* x_out, gmrf_result_info* info) {
  if (!p || !o || !b_in || !x_out) return GMRF_ERR_INVALID;
  if (!(o->tol > 0.0) || !std::isfinite(o->tol) || o->m_max < 1 || o->m_max > 8192 || o->nrhs < 1 ||
      o->reserved != 0)
    return GMRF_ERR_INVALID;
  const size_t n = p->g.n, es = esize(p);
  const int m_max = o->m_max;
  const int nslots = m_max + 1;
  const bool x_dev = is_device_ptr(x_out);
  const bool b_dev = is_device_ptr(b_in);
  const size_t extra = (x_dev ? 0 : n * es) + (b_dev ? 0 : n * es) +
                       (p->precond ? precond_extra_bytes(p->pre, es) + n * es : 0) + (sparse_f(p) ? n * es : 0) +
                       sizeof(double) * m_max;
  int chunk = batch_size(p, o->nrhs, nslots, m_max, false, extra);
  if (p->tune_bw > 0 && chunk > p->tune_bw) chunk = p->tune_bw;
  if (chunk < 1) return GMRF_ERR_OOM;
  cudaStream_t s = p->ws;
  CKR(enter(p));
  std::vector<VecState> all((size_t)o->nrhs);
  for (int s0 = 0; s0 < o->nrhs; s0 += chunk) {
    const int c = std::min(chunk, o->nrhs - s0);
    LanczosBufs b;
    CKR(ensure_lanczos(p, c, nslots, m_max, false, b));
    CKR(ensure(p->solvew, sizeof(double) * (size_t)c * m_max, p->ws));
    const char* bsrc = (const char*)b_in + (size_t)s0 * n * es;
    // start vector: b (no preconditioner), F^{-1} b (sparse with F) or
    // B_bar^{-p/2} b, normalised by the first step
    if (sparse_f(p)) {
      const void* dsrc = bsrc;
      if (!b_dev) {
        CKR(ensure(p->stage2, (size_t)c * n * es, p->ws));
        CK(cudaMemcpyAsync(p->stage2.p, bsrc, (size_t)c * n * es, cudaMemcpyHostToDevice, s));
        dsrc = p->stage2.p;
      }
      CK(traced(KC_PRE_APPLY, s, 1, [&] { return launch_sparse_ops(*p->sp, 3, dsrc, b.W[0], c, s); }));
    } else if (p->precond == GMRF_PREC_NONE) {
      CK(cudaMemcpyAsync(b.W[0], bsrc, (size_t)c * n * es, b_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         s));
    } else {
      const void* dsrc = bsrc;
      if (!b_dev) {
        CKR(ensure(p->stage2, (size_t)c * n * es, p->ws));
        CK(cudaMemcpyAsync(p->stage2.p, bsrc, (size_t)c * n * es, cudaMemcpyHostToDevice, s));
        dsrc = p->stage2.p;
      }
      CK(traced(KC_PRE_APPLY, s, 3,
                [&] { return launch_precond_apply(p->pre, p->g, p->fp64, PRE_INV_SQRT, dsrc, b.W[0], c, s); }));
    }
    CKR(run_lanczos(p, b, o->tol, m_max, o->check_every, true));
    CK(traced(KC_TM, s, 1, [&] { return launch_tm_inv(b, (double*)p->solvew.p, (double*)p->y.p, s); }));
    void* xdst = (char*)x_out + (size_t)s0 * n * es;
    if (!x_dev) {
      CKR(ensure(p->stage, (size_t)c * n * es, p->ws));
      xdst = p->stage.p;
    }
    // x_m = ||b~|| V_m T_m^{-1} e_1; Q = tau Q~ (the steps run on Q~ or A, both tau-free)
    if (sparse_f(p)) {
      // u = A^{-1} F^{-1} b, then x = tau^{-1} F^{-T} u
      CKR(ensure(p->work, (size_t)c * n * es, p->ws));
      CK(traced(KC_ASSEMBLE, s, 1,
                [&] { return launch_assemble(p->fp64, n, b, (double*)p->y.p, m_max, 1.0, p->work.p, s); }));
      CK(traced(KC_PRE_APPLY, s, 1, [&] { return launch_sparse_ops(*p->sp, 2, p->work.p, xdst, c, s); }));
      CK(traced(KC_OTHER, s, 1, [&] { return launch_scale(p->fp64, xdst, (size_t)c * n, 1.0 / p->tau, s); }));
    } else if (p->precond == GMRF_PREC_NONE) {
      CK(traced(KC_ASSEMBLE, s, 1, [&] {
        return launch_assemble(p->fp64, n, b, (double*)p->y.p, m_max, 1.0 / p->tau, xdst, s);
      }));
    } else {
      // u = ||b~|| V_m T_m^{-1} e_1 = A^{-1} b~, then x = tau^{-1} B_bar^{-p/2} u
      CKR(ensure(p->work, (size_t)c * n * es, p->ws));
      CK(traced(KC_ASSEMBLE, s, 1,
                [&] { return launch_assemble(p->fp64, n, b, (double*)p->y.p, m_max, 1.0, p->work.p, s); }));
      CK(traced(KC_PRE_APPLY, s, 3,
                [&] { return launch_precond_apply(p->pre, p->g, p->fp64, PRE_INV_SQRT, p->work.p, xdst, c, s); }));
      CK(traced(KC_OTHER, s, 1, [&] { return launch_scale(p->fp64, xdst, (size_t)c * n, 1.0 / p->tau, s); }));
    }
    if (!x_dev)
      CK(cudaMemcpyAsync((char*)x_out + (size_t)s0 * n * es, xdst, (size_t)c * n * es, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(p->st_host, b.st, sizeof(VecState) * c, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    trace_collect();
    std::memcpy(all.data() + s0, p->st_host, sizeof(VecState) * c);
  }
  CKR(leave(p));
  fill_info(all.data(), o->nrhs, info);
  return worst_status(all.data(), o->nrhs);
}

int gmrf_logdet(gmrf_problem* p, const gmrf_logdet_opts* o, double* logdet, double* std_err, double* q_out,
                gmrf_result_info* info) {
  if (!p || !o || !logdet || !std_err) return GMRF_ERR_INVALID;
  if (!(o->tol > 0.0) || !std::isfinite(o->tol) || o->m_max < 1 || o->m_max > 8192 || o->nprobes < 1 ||
      o->colour_dist < 0 || o->colour_dist > 15)
    return GMRF_ERR_INVALID;
  if (p->sp && o->colour_dist != 0) return GMRF_ERR_UNSUPPORTED;  // colouring needs the lattice
  const size_t n = p->g.n, es = esize(p);
  const int m_max = o->m_max;
  const bool z_dev = o->probes_in && is_device_ptr(o->probes_in);
  // coloured estimator (Section 6.1): ncol probe vectors per draw
  const int P = o->colour_dist + 1;
  int ncol = 1;
  for (int d = 0; d < p->g.dim; ++d) ncol *= P;
  const int64_t nq64 = (int64_t)o->nprobes * ncol;
  if (nq64 > (1 << 24)) return GMRF_ERR_INVALID;
  const int nq = (int)nq64;
  int chunk = batch_size(p, nq, 2, m_max, false, 0);
  if (p->tune_bw > 0 && chunk > p->tune_bw) chunk = p->tune_bw;
  if (chunk < 1) return GMRF_ERR_OOM;
  cudaStream_t s = p->ws;
  CKR(enter(p));
  CKR(ensure(p->stage2, sizeof(double) * (nq + 2), p->ws));
  double* qall = (double*)p->stage2.p;
  std::vector<VecState> all((size_t)nq);
  for (int s0 = 0; s0 < nq; s0 += chunk) {
    const int c = std::min(chunk, nq - s0);
    LanczosBufs b;
    CKR(ensure_lanczos(p, c, 2, m_max, false, b));
    if (o->probes_in) {
      const char* src = (const char*)o->probes_in + (size_t)s0 * n * es;
      CK(cudaMemcpyAsync(b.W[0], src, (size_t)c * n * es, z_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         s));
    } else if (ncol > 1) {
      CK(traced(KC_RNG, s, 1, [&] {
        return launch_rng_coloured(p->fp64, c, (int64_t)n, o->seed, s0, p->g.nx, p->g.ny, P, ncol, b.W[0], s);
      }));
    } else {
      CK(traced(KC_RNG, s, 1, [&] { return launch_rng(1, p->fp64, c, (int64_t)n, o->seed, s0, b.W[0], s); }));
    }
    CKR(run_lanczos(p, b, o->tol, m_max, o->check_every));
    CK(traced(KC_TM, s, 2, [&] { return launch_tm_log(b, p->fp64, (TmNodes*)p->nodes.p, qall + s0, s); }));
    CK(cudaMemcpyAsync(p->st_host, b.st, sizeof(VecState) * c, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::memcpy(all.data() + s0, p->st_host, sizeof(VecState) * c);
  }
  // log det Q = mean q_i + log det M(tau-free) + n log tau   (Section 6.2, plus sign)
  const double shift = p->logdet_M + (double)n * std::log(p->tau);
  CK(traced(KC_TM, s, 1, [&] { return launch_logdet_reduce(qall, nq, ncol, shift, qall + nq, s); }));
  double res[2];
  CK(cudaMemcpyAsync(res, qall + nq, sizeof(res), cudaMemcpyDeviceToHost, s));
  if (q_out) CK(cudaMemcpyAsync(q_out, qall, sizeof(double) * nq, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  trace_collect();
  CKR(leave(p));
  *logdet = res[0];
  *std_err = res[1];
  fill_info(all.data(), nq, info);
  return worst_status(all.data(), nq);
}

int gmrf_sample_logdet(gmrf_problem* p, const gmrf_sample_opts* so, const gmrf_logdet_opts* lo, void* x_out,
                       gmrf_result_info* sinfo, double* logdet, double* std_err, double* q_out,
                       gmrf_result_info* linfo) {
  if (!p || !so || !lo || !x_out || !logdet || !std_err) return GMRF_ERR_INVALID;
  if (!(so->tol > 0.0) || !std::isfinite(so->tol) || so->m_max < 1 || so->m_max > 8192 || so->nsamples < 1 ||
      so->v_storage != GMRF_VSTORE_NATIVE || lo->tol != so->tol || lo->m_max != so->m_max || lo->nprobes < 1 ||
      lo->colour_dist < 0 || lo->colour_dist > 15)
    return GMRF_ERR_INVALID;
  if (p->sp && lo->colour_dist != 0) return GMRF_ERR_UNSUPPORTED;
  const size_t n = p->g.n, es = esize(p);
  const int m_max = so->m_max, nslots = m_max + 1;
  const int P = lo->colour_dist + 1;
  int ncol = 1;
  for (int d = 0; d < p->g.dim; ++d) ncol *= P;
  const int64_t total64 = (int64_t)so->nsamples + (int64_t)lo->nprobes * ncol;
  if (total64 > (1 << 24)) return GMRF_ERR_INVALID;
  const int ns = so->nsamples, nq = (int)(total64 - ns), total = (int)total64;
  const bool x_dev = is_device_ptr(x_out);
  const bool z_dev = so->z_in && is_device_ptr(so->z_in);
  const bool r_dev = lo->probes_in && is_device_ptr(lo->probes_in);
  const size_t extra = (x_dev ? 0 : n * es) + (p->precond ? precond_extra_bytes(p->pre, es) + n * es : 0) +
                       (sparse_f(p) ? n * es : 0) + check_bytes_per_vec(p);
  int chunk = batch_size(p, total, nslots, m_max, true, extra);
  if (p->tune_bw > 0 && chunk > p->tune_bw) chunk = p->tune_bw;
  if (chunk < 1) return GMRF_ERR_OOM;
  cudaStream_t s = p->ws;
  CKR(enter(p));
  CKR(ensure(p->stage2, sizeof(double) * (nq + 2), p->ws));
  double* qall = (double*)p->stage2.p;
  std::vector<VecState> all((size_t)total);
  for (int t0 = 0; t0 < total; t0 += chunk) {
    const int c = std::min(chunk, total - t0);
    const int nsc = std::max(0, std::min(ns, t0 + c) - t0);  // samples of this chunk come first
    const int nqc = c - nsc, q0 = std::max(0, t0 - ns);     // then probes q0 .. q0 + nqc - 1
    LanczosBufs b;
    CKR(ensure_lanczos(p, c, nslots, m_max, true, b));
    // the same z and probes as gmrf_sample and gmrf_logdet (per-vector streams)
    auto load_z = [&]() -> int {
      if (so->z_in)
        CK(cudaMemcpyAsync(b.W[0], (const char*)so->z_in + (size_t)t0 * n * es, (size_t)nsc * n * es,
                           z_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
      else
        CK(traced(KC_RNG, s, 1, [&] { return launch_rng(0, p->fp64, nsc, (int64_t)n, so->seed, t0, b.W[0], s); }));
      return GMRF_OK;
    };
    if (nsc > 0) CKR(load_z());
    if (nqc > 0) {
      void* dst = (char*)b.W[0] + (size_t)nsc * n * es;
      if (lo->probes_in)
        CK(cudaMemcpyAsync(dst, (const char*)lo->probes_in + (size_t)q0 * n * es, (size_t)nqc * n * es,
                           r_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
      else if (ncol > 1)
        CK(traced(KC_RNG, s, 1, [&] {
          return launch_rng_coloured(p->fp64, nqc, (int64_t)n, lo->seed, q0, p->g.nx, p->g.ny, P, ncol, dst, s);
        }));
      else
        CK(traced(KC_RNG, s, 1, [&] { return launch_rng(1, p->fp64, nqc, (int64_t)n, lo->seed, q0, dst, s); }));
    }
    CKR(run_lanczos(p, b, so->tol, m_max, so->check_every));
    std::vector<double> est((size_t)std::max(nsc, 1)), est_prev((size_t)std::max(nsc, 1), 0.0);
    std::vector<int> mmin((size_t)std::max(nsc, 1), 0);
    void* xdst = (char*)x_out + (size_t)t0 * n * es;
    if (nsc > 0) {
      CKR(ensure(p->ucg, (size_t)nsc * n * es, p->ws));
      CKR(ensure(p->zre, (size_t)nsc * n * es, p->ws));
      if (!x_dev) {
        CKR(ensure(p->stage, (size_t)nsc * n * es, p->ws));
        xdst = p->stage.p;
      }
    }
    // the samples' z for the accuracy check (as in gmrf_sample)
    if (nsc > 0) {
      if (so->z_in)
        CK(cudaMemcpyAsync(p->zre.p, (const char*)so->z_in + (size_t)t0 * n * es, (size_t)nsc * n * es,
                           z_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
      else
        CK(traced(KC_RNG, s, 1, [&] { return launch_rng(0, p->fp64, nsc, (int64_t)n, so->seed, t0, p->zre.p, s); }));
    }
    for (int round = 0; nsc > 0; ++round) {
      const LanczosBufs bs = sub_batch(b, 0, nsc, n, es);
      CK(traced(KC_TM, s, 3, [&] {
        return launch_tm_inv_sqrt(bs, p->fp64, (TmNodes*)p->nodes.p, (double*)p->scratch.p, (double*)p->y.p, s);
      }));
      CKR(check_tm(p, bs, s));
      const double* ycg = (const double*)p->ycg.p;
      if (sparse_f(p)) {
        CKR(ensure(p->work, (size_t)nsc * n * es, p->ws));
        CK(traced(KC_ASSEMBLE, s, 1, [&] {
          return launch_assemble_dual(p->fp64, n, bs, (double*)p->y.p, m_max, 1.0, p->work.p, ycg, p->ucg.p, s);
        }));
        CK(traced(KC_PRE_APPLY, s, 1, [&] { return launch_sparse_ops(*p->sp, 2, p->work.p, xdst, nsc, s); }));
        CK(traced(KC_OTHER, s, 1,
                  [&] { return launch_scale(p->fp64, xdst, (size_t)nsc * n, 1.0 / std::sqrt(p->tau), s); }));
      } else if (p->precond == GMRF_PREC_NONE) {
        CK(traced(KC_ASSEMBLE, s, 1, [&] {
          return launch_assemble_dual(p->fp64, n, bs, (double*)p->y.p, m_max, 1.0 / std::sqrt(p->tau), xdst, ycg,
                                      p->ucg.p, s);
        }));
      } else {
        CKR(ensure(p->work, (size_t)nsc * n * es, p->ws));
        CK(traced(KC_ASSEMBLE, s, 1, [&] {
          return launch_assemble_dual(p->fp64, n, bs, (double*)p->y.p, m_max, 1.0, p->work.p, ycg, p->ucg.p, s);
        }));
        CK(traced(KC_PRE_APPLY, s, 3, [&] {
          return launch_precond_apply(p->pre, p->g, p->fp64, PRE_INV_SQRT, p->work.p, xdst, nsc, s);
        }));
        CK(traced(KC_OTHER, s, 1,
                  [&] { return launch_scale(p->fp64, xdst, (size_t)nsc * n, 1.0 / std::sqrt(p->tau), s); }));
      }
      // accuracy check of the samples, with the same resumption as gmrf_sample
      CKR(check_vectors(p, nsc, p->zre.p, p->ucg.p, b.st, p->st_host, so->tol, est.data(), s));
      trace_collect();
      if (!check_resume(p->st_host, est.data(), est_prev.data(), mmin.data(), nsc, so->tol, m_max, round)) break;
      est_prev = est;
      CK(cudaMemcpyAsync(b.st, p->st_host, sizeof(VecState) * nsc, cudaMemcpyHostToDevice, s));
      CKR(run_lanczos(p, b, so->tol, m_max, so->check_every, false, false));
    }
    if (nsc > 0 && !x_dev)
      CK(cudaMemcpyAsync((char*)x_out + (size_t)t0 * n * es, xdst, (size_t)nsc * n * es, cudaMemcpyDeviceToHost, s));
    if (nqc > 0) {
      const LanczosBufs bq = sub_batch(b, nsc, nqc, n, es);
      CK(traced(KC_TM, s, 2, [&] { return launch_tm_log(bq, p->fp64, (TmNodes*)p->nodes.p, qall + q0, s); }));
    }
    CK(cudaMemcpyAsync(p->st_host, b.st, sizeof(VecState) * c, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    trace_collect();
    if (nsc > 0) check_apply(p->st_host, est.data(), nsc, so->tol);
    std::memcpy(all.data() + t0, p->st_host, sizeof(VecState) * c);
  }
  const double shift = p->logdet_M + (double)n * std::log(p->tau);
  CK(traced(KC_TM, s, 1, [&] { return launch_logdet_reduce(qall, nq, ncol, shift, qall + nq, s); }));
  double res[2];
  CK(cudaMemcpyAsync(res, qall + nq, sizeof(res), cudaMemcpyDeviceToHost, s));
  if (q_out) CK(cudaMemcpyAsync(q_out, qall, sizeof(double) * nq, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  trace_collect();
  CKR(leave(p));
  *logdet = res[0];
  *std_err = res[1];
  fill_info(all.data(), ns, sinfo);
  fill_info(all.data() + ns, nq, linfo);
  return worst_status(all.data(), total);
}

int gmrf_apply(gmrf_problem* p, int32_t which, int64_t nvec, const void* v, void* y) {
  if (!p || !v || !y || nvec < 1 || nvec > 65535 || which < 0 || which > 2) return GMRF_ERR_INVALID;
  if (which > 0 && (p->sp ? !sparse_f(p) : p->precond == GMRF_PREC_NONE)) return GMRF_ERR_INVALID;
  const size_t n = p->g.n, es = esize(p), bytes = (size_t)nvec * n * es;
  cudaStream_t s = p->ws;
  CKR(enter(p));
  const bool vd = is_device_ptr(v), yd = is_device_ptr(y);
  const void* vin = v;
  void* yout = y;
  if (!vd) {
    CKR(ensure(p->stage, bytes, p->ws));
    CK(cudaMemcpyAsync(p->stage.p, v, bytes, cudaMemcpyHostToDevice, s));
    vin = p->stage.p;
  }
  if (!yd) {
    CKR(ensure(p->stage2, bytes, p->ws));
    yout = p->stage2.p;
  }
  if (p->sp) {
    // 0: tau Q v; 1: A v; 2: tau^{-1/2} F^{-T} v
    const int mode = which == 0 ? 0 : (which == 1 ? 1 : 2);
    CK(traced(KC_PRE_APPLY, s, 1, [&] { return launch_sparse_ops(*p->sp, mode, vin, yout, (int)nvec, s); }));
    if (which != 1) {
      const double f = which == 0 ? p->tau : 1.0 / std::sqrt(p->tau);
      CK(traced(KC_OTHER, s, 1, [&] { return launch_scale(p->fp64, yout, (size_t)nvec * n, f, s); }));
    }
  } else if (which == 0) {
    CK(traced(KC_STENCIL_STEP, s, 1, [&] {
      return launch_stencil_apply(p->g, p->fp64, p->kappa2.p, p->kappa2_const, vin, yout, (int)nvec, s);
    }));
    CK(traced(KC_OTHER, s, 1, [&] { return launch_scale(p->fp64, yout, (size_t)nvec * n, p->tau, s); }));
  } else if (which == 1) {
    CK(traced(KC_PRE_APPLY, s, 5, [&] {
      return launch_precond_operator(p->pre, p->g, p->fp64, p->kappa2.p, p->kappa2_const, vin, yout, (int)nvec, s);
    }));
  } else {
    CK(traced(KC_PRE_APPLY, s, 3,
              [&] { return launch_precond_apply(p->pre, p->g, p->fp64, PRE_INV_SQRT, vin, yout, (int)nvec, s); }));
    CK(traced(KC_OTHER, s, 1, [&] { return launch_scale(p->fp64, yout, (size_t)nvec * n, 1.0 / std::sqrt(p->tau), s); }));
  }
  if (!yd) CK(cudaMemcpyAsync(y, yout, bytes, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  trace_collect();
  CKR(leave(p));
  return GMRF_OK;
}

int gmrf_rng(int32_t kind, int32_t precision, int64_t nvec, int64_t n, uint64_t seed, void* out, void* stream) {
  if (!out || kind < 0 || kind > 2 || nvec < 1 || n < 1 || nvec > 65535 || n > ((int64_t)1 << 34)) return GMRF_ERR_INVALID;
  if (precision != GMRF_FP32 && precision != GMRF_FP64) return GMRF_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const bool fp64 = precision == GMRF_FP64;
  const size_t es = kind == 2 ? 4 : (fp64 ? 8 : 4);
  const size_t per = kind == 2 ? (size_t)4 * ((n + 3) / 4) : (size_t)n;
  const size_t bytes = (size_t)nvec * per * es;
  if (is_device_ptr(out)) {
    CK(launch_rng(kind, fp64, nvec, n, seed, 0, out, s));
    CK(cudaStreamSynchronize(s));
    return GMRF_OK;
  }
  void* d = nullptr;
  if (cudaMallocAsync(&d, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return GMRF_ERR_OOM;
  }
  int rc = GMRF_OK;
  if (launch_rng(kind, fp64, nvec, n, seed, 0, d, s) != cudaSuccess ||
      cudaMemcpyAsync(out, d, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
    cudaGetLastError();
    rc = GMRF_ERR_CUDA;
  }
  cudaFreeAsync(d, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    rc = GMRF_ERR_CUDA;
  }
  return rc;
}

int gmrf_set_tuning(gmrf_problem* p, const gmrf_tuning* t) {
  if (!p || !t || t->block_width < 0 || t->zchunk < 0 || (t->host_loop != 0 && t->host_loop != 1))
    return GMRF_ERR_INVALID;
  p->tune_bw = t->block_width;
  p->host_loop = t->host_loop != 0;
  p->g.zchunk = tune_zchunk_ok(p) ? t->zchunk : 0;
  p->graph.reset();
  return GMRF_OK;
}

int gmrf_autotune(gmrf_problem* p, int32_t nvec_max, gmrf_tuning* out) {
  if (!p || !out || nvec_max < 1) return GMRF_ERR_INVALID;
  const size_t n = p->g.n, es = esize(p);
  constexpr int kSteps = 8, kMmax = 64;
  const size_t extra = p->precond ? precond_extra_bytes(p->pre, es) : 0;
  int cap = batch_size(p, nvec_max, 2, kMmax, false, extra);
  if (cap < 1) return GMRF_ERR_OOM;
  cudaStream_t s = p->ws;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return GMRF_ERR_CUDA;
  }
  int ncand = 0;
  // vector-steps per second of kSteps Lanczos steps (after kSteps untimed
  // ones) on `bw` Rademacher vectors, with the problem's current tiling
  auto measure = [&](int bw, double* rate) -> int {
    LanczosBufs b;
    CKR(ensure_lanczos(p, bw, 2, kMmax, false, b));
    CK(launch_rng(1, p->fp64, bw, (int64_t)n, 0x5EEDull, 0, b.W[0], s));
    CK(launch_lanczos_init(p->fp64, n, b, s));
    StepParams P{};
    P.m_max = kMmax;
    P.nslots = 2;
    P.tol = 1e-300;  // never met: every vector runs all timed steps
    P.bd_tol = p->fp64 ? 1e-13 : 1e-6;
    if (p->precond != GMRF_PREC_NONE) CKR(precond_prepare(p->pre, bw, s));
    CKR(capture_steps(p, b, P, kSteps));
    CK(cudaGraphLaunch(p->graph.exec, s));
    CK(cudaEventRecord(e0, s));
    CK(cudaGraphLaunch(p->graph.exec, s));
    CK(cudaEventRecord(e1, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    *rate = ms > 0.f ? (double)bw * kSteps / (ms * 1e-3) : 0.0;
    ++ncand;
    return GMRF_OK;
  };
  int rc = enter(p);
  int best_z = 0, best_bw = cap;
  double best = -1.0;
  if (rc == GMRF_OK && tune_zchunk_ok(p)) {
    // z planes per work item of the 3-D step, at a moderate block width
    const int bw0 = std::min(cap, 16);
    for (int z = p->g.nz; z >= 8 && rc == GMRF_OK; z /= 2) {
      p->g.zchunk = z;
      double r = 0.0;
      rc = measure(bw0, &r);
      if (rc == GMRF_OK && r > best) {
        best = r;
        best_z = z;
      }
    }
    p->g.zchunk = best_z;
  }
  if (rc == GMRF_OK) {
    // block width: powers of two up to the memory cap, and the cap itself;
    // the smallest width within 3% of the best rate wins (less memory, less
    // waiting for a full batch)
    std::vector<int> cands;
    for (int w = 1; w < cap; w *= 2) cands.push_back(w);
    cands.push_back(cap);
    std::vector<double> rates;
    for (int w : cands) {
      double r = 0.0;
      rc = measure(w, &r);
      if (rc != GMRF_OK) break;
      rates.push_back(r);
    }
    if (rc == GMRF_OK) {
      const double top = *std::max_element(rates.begin(), rates.end());
      for (size_t i = 0; i < cands.size(); ++i)
        if (rates[i] >= 0.97 * top) {
          best_bw = cands[i];
          best = rates[i];
          break;
        }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->graph.reset();
  const int rl = leave(p);
  if (rc != GMRF_OK) {
    p->g.zchunk = 0;
    return rc;
  }
  if (rl != GMRF_OK) return rl;
  p->tune_bw = best_bw;
  out->block_width = best_bw;
  out->zchunk = p->g.zchunk;
  out->vec_steps_per_s = best;
  out->candidates = ncand;
  out->host_loop = p->host_loop ? 1 : 0;
  return GMRF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of gmrf_apply(which = 2): y = M^{-1/2} v.
//
// Its only scratch, the transform workspace, is this file-scope device array
// of GMRF_NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library holds it
// until the process exits.  In host code the symbol is only a stand-in, so
// its device address is looked up with cudaGetSymbolAddress once per device,
// on the first call for a problem of that device; the entry point checks
// first that this device is the current one, so the lookup runs with it
// current.
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[GMRF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// dev must be the current device.
int noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return GMRF_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return GMRF_ERR_CUDA;
    }
    g_noalloc_addr[dev] = ptr;
  }
  *out = g_noalloc_addr[dev];
  return GMRF_OK;
}

}  // namespace

extern "C" int gmrf_apply_inv_sqrt_noalloc(gmrf_problem* p, int64_t nvec, const void* v, void* y) {
  if (!p || !v || !y || nvec < 1 || nvec > 65535) return GMRF_ERR_INVALID;
  if (p->sp) return GMRF_ERR_UNSUPPORTED;
  if (p->precond == GMRF_PREC_NONE) return GMRF_ERR_INVALID;
  if (!is_device_ptr(v) || !is_device_ptr(y)) return GMRF_ERR_INVALID;
  if (precond_apply_scratch_bytes(p->pre, (int)nvec) > (size_t)GMRF_NOALLOC_SCRATCH_BYTES) return GMRF_ERR_INVALID;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return GMRF_ERR_CUDA;
  }
  if (cur != p->device) return GMRF_ERR_INVALID;  // the problem's device must be current
  void* scratch = nullptr;
  CKR(noalloc_scratch(p->device, &scratch));
  cudaStream_t s = p->ws;
  CKR(enter(p));
  // the spectrum is fully written by the forward row pass before it is read:
  // nothing in the shared scratch has to start at zero
  CK(traced(KC_PRE_APPLY, s, 3, [&] {
    return launch_precond_apply_with(p->pre, p->g, p->fp64, v, y, (int)nvec, scratch, s);
  }));
  CK(traced(KC_OTHER, s, 1, [&] { return launch_scale(p->fp64, y, (size_t)nvec * p->g.n, 1.0 / std::sqrt(p->tau), s); }));
  CK(cudaStreamSynchronize(s));
  trace_collect();
  CKR(leave(p));
  return GMRF_OK;
}
