// host.h -- the host driver's problem record and the helpers that the C-ABI
// translation units share (gmrf_api.cu, server.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "internal.h"
#include "precond.h"
#include "trace.h"

namespace host {

using namespace gmrf;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Grow-only, stream-ordered workspace (no device synchronisation).
int ensure(DevBuf& b, size_t bytes, cudaStream_t s);
void release(DevBuf& b, cudaStream_t s);
bool is_device_ptr(const void* p);

}  // namespace host

using namespace gmrf;
using host::DevBuf;

#define CK(x)                               \
  do {                                      \
    cudaError_t e_ = (x);                   \
    if (e_ != cudaSuccess) {                \
      cudaGetLastError();                   \
      return GMRF_ERR_CUDA;                 \
    }                                       \
  } while (0)
#define CKR(x)                 \
  do {                         \
    int r_ = (x);              \
    if (r_ != GMRF_OK) return r_; \
  } while (0)

// The Lanczos loop's CUDA graph: `c` steps captured once and replayed until
// every vector has converged (the kernels read the step index from device
// state).  Keyed by everything the captured launches depend on.
struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  GraphTrace tr;
  int nvec = -1, nslots = 0, m_max = 0, c = 0, kernels_per_step = 1, zchunk = 0, solve = 0;
  double tol = 0.0;
  const void *W0 = nullptr, *V = nullptr, *Vb = nullptr, *st = nullptr, *S = nullptr, *partials = nullptr;
  const void* Xacc = nullptr;
  const void* Xacc2 = nullptr;
  const void* y1 = nullptr;
  const void* y2 = nullptr;
  double xscale = 0.0;
  bool timed = false;
  bool loop = false;   // exec is the device-side loop (a WHILE node over one step), else c steps to replay
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    tr.release();
    nvec = -1;
  }
};

struct gmrf_problem {
  Grid g;
  int precond = GMRF_PREC_NONE;
  bool fp64 = false;
  double tau = 1.0;
  double kappa2_const = 0.0;
  double kbar2 = 0.0;
  double logdet_M = 0.0;  // log det of the tau-free preconditioner (B_bar^p)
  int device = 0;                  // the device current at create (the problem's memory lives there)
  cudaStream_t stream = nullptr;   // the caller's stream
  cudaStream_t ws = nullptr;       // the library's work stream (graphs are captured on it)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  StepGraph graph;
  DevBuf kappa2;  // float [n] or empty (constant)
  PrecondTables pre;
  SparseOp* sp = nullptr;  // general sparse Q (gmrf_create_sparse), else null
  // Lanczos workspace (grow-only)
  DevBuf W0, W1, V, st, alpha, beta, alpha_f, beta2_f, partials, counters, y, scratch, nodes, q, out2, stage,
      stage2, work, Vb, xacc, accn, solvew;
  // accuracy check of samples: T_m^{-1} e_1 and its workspace, the CG iterate
  // u_cg, the product A u_cg (FP64 pair for FP32 stencils), the residual norms
  DevBuf ycg, ucg, xacc2, chk, rn, zre, mmin;
  DevBuf loopctr;  // iteration counter of the device-side Lanczos loop
  VecState* st_host = nullptr;
  int st_host_cap = 0;
  // a continuous-batching server attached to the problem (server.cu): while it
  // exists, only its own calls (in_server) may use the problem's workspace
  gmrf_server* server = nullptr;
  bool in_server = false;
  int tune_bw = 0;  // vectors per Lanczos launch (0: as many as fit)
  bool host_loop = false;  // host-replayed step graphs instead of the device-side loop
};

namespace host {

size_t esize(const gmrf_problem* p);
bool sparse_f(const gmrf_problem* p);
int enter(gmrf_problem* p);
int leave(gmrf_problem* p);
int ensure_host_states(gmrf_problem* p, int nvec);
int ensure_lanczos(gmrf_problem* p, int nvec, int nslots, int m_max, bool need_tm, LanczosBufs& b,
                   bool bf16_basis = false);
int batch_size(gmrf_problem* p, int want, int nslots, int m_max, bool need_tm, size_t extra_per_vec);
int worst_status(const VecState* st, int nvec);
int capture_steps(gmrf_problem* p, const LanczosBufs& b, const StepParams& P, int c);
int run_lanczos(gmrf_problem* p, const LanczosBufs& b, double tol, int m_max, int check_every, bool solve = false,
                bool init = true);
// The step parameters run_lanczos uses.
StepParams step_params(gmrf_problem* p, const LanczosBufs& b, double tol, int m_max, bool solve);
LanczosBufs sub_batch(const LanczosBufs& b, int off, int cnt, size_t n, size_t es);
size_t check_bytes_per_vec(const gmrf_problem* p);
int check_tm(gmrf_problem* p, const LanczosBufs& b, cudaStream_t s);
int check_residuals(gmrf_problem* p, int nvec, const void* z, void* u, bool second, cudaStream_t s);
double direct_estimate(const VecState& v, const double* d3);
double crude_estimate(const VecState& v, double rr);
int check_vectors(gmrf_problem* p, int nvec, const void* z, void* u, const VecState* st_dev, VecState* hst,
                  double tol, double* est, cudaStream_t s);
bool check_resume(VecState* st, const double* est, const double* est_prev, int* mmin, int nvec, double tol, int m_max,
                  int round);
void check_apply(VecState* st, const double* est, int nvec, double tol);
void fill_info(const VecState* st, int nvec, gmrf_result_info* info);

}  // namespace host
