// internal.h -- launchers shared between the kernel translation units and the
// host driver (gmrf_api.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace gmrf {

// Geometry + operator of a lattice problem, as the kernels see it.
struct Grid {
  int dim;
  int nx, ny, nz;
  size_t n;
  int bc;      // gmrf_bc
  int op;      // gmrf_op
  int zchunk = 0;  // 3-D FP32 stencil step: z planes per work item (0: chosen from the grid)
};

// Per-batch Lanczos buffers (all device pointers).  Element type T is float
// or double; `V` holds `nslots` basis vectors per vector:
// V[(s * nslots + slot) * n + i].
struct LanczosBufs {
  void* W[2];          // q of the previous / current step, [nvec][n]
  void* V;             // basis ring
  __nv_bfloat16* Vb;   // bfloat16 basis [nvec][m_max + 1][n] for the assembly, or null
  VecState* st;        // [nvec]
  double* alpha;       // [nvec][m_max]
  double* beta;        // [nvec][m_max]
  float* alpha_f;      // [nvec][m_max]
  float* beta2_f;      // [nvec][m_max]
  void* partials;      // [nvec][max blocks] Dots<T>
  unsigned* counters;  // [nvec]
  int nvec;
  int nslots;
  int m_max;
  // Two-pass sampling (second pass): after each step x += ||z|| extra y_j v_j
  // into Xacc ([nvec][2][n] float sum/compensation, or [nvec][n] double);
  // acc[s] counts the basis vectors already added.  Xacc null: no accumulation.
  void* Xacc = nullptr;
  int* acc = nullptr;
  const double* y = nullptr;  // [nvec][m_max] from the first pass
  double xscale = 1.0;
  // optional second accumulation, x2 += ||z|| y2_j v_j into Xacc2 (same layout as Xacc)
  void* Xacc2 = nullptr;
  const double* y2 = nullptr;
  // [nvec] minimum step counts for the stopping rule, read at init (null: 0)
  const int* m_min = nullptr;
};

// lanczos_stencil.cu --------------------------------------------------------
// Blocks per vector of the fused stencil step for this grid.
int stencil_blocks_per_vector(const Grid& g);
// Fused step j of Algorithm 1 with the matrix-free stencil Q: forms v_j,
// stores it, q_j = Q v_j - beta_{j-1} v_{j-1}, dot products, alpha_j, beta_j,
// stopping rule.  W[j&1] is read, W[(j+1)&1] written.
cudaError_t launch_stencil_step(const Grid& g, bool fp64, const void* kappa2, double kappa2_const,
                                const LanczosBufs& b, const StepParams& P, cudaStream_t s);
// y = Q v for nvec vectors (no Lanczos bookkeeping).
cudaError_t launch_stencil_apply(const Grid& g, bool fp64, const void* kappa2, double kappa2_const,
                                 const void* v, void* y, int nvec, cudaStream_t s);

// stencil3d_tma.cu -------------------------------------------------------------
// The TMA-staged 3-D 7-point step / apply serves FP32 grids with Dirichlet or
// zero-Neumann boundaries, nx a multiple of 4 and >= 128.
bool stencil3d_tma_eligible(const Grid& g, bool fp64);
// Work items (partial sums) per vector of that kernel.
int stencil3d_tma_items_per_vector(const Grid& g);

// misc.cu --------------------------------------------------------------------
cudaError_t launch_rng(int kind, bool fp64, int64_t nvec, int64_t n, uint64_t seed, int64_t soff, void* out,
                       cudaStream_t s);
// Coloured Rademacher probes of the distance-(P-1) lattice colouring (ncol
// colours): vector soff + s of the output is draw (soff + s) / ncol restricted
// to colour (soff + s) % ncol.
cudaError_t launch_rng_coloured(bool fp64, int64_t nvec, int64_t n, uint64_t seed, int64_t soff, int nx, int ny,
                                int P, int ncol, void* out, cudaStream_t s);
// out4[0] = #(kappa2 < 0 or not finite), [1] = #zeros, [2] = sum log kappa2 over positives.
// out4 must have kFieldStatsBytes of device memory (results + per-block parts).
constexpr size_t kFieldStatsBytes = 4 * sizeof(double) + 256 * sizeof(Dots<float>);
cudaError_t launch_field_stats(const float* k, size_t n, double* out4, cudaStream_t s);
// ||z|| of each vector of W[0] into st[].znorm, and resets the state.
cudaError_t launch_lanczos_init(bool fp64, size_t n, const LanczosBufs& b, cudaStream_t s);
// x[s] = scale[s] * V_m y  (scale = ||z|| * extra), y from tm buffers.
cudaError_t launch_assemble(bool fp64, size_t n, const LanczosBufs& b, const double* y, int y_stride,
                            double extra_scale, void* x, cudaStream_t s);
// The same x, plus x2[s] = ||z|| V_m y2 from the same pass over V_m.
cudaError_t launch_assemble_dual(bool fp64, size_t n, const LanczosBufs& b, const double* y, int y_stride,
                                 double extra_scale, void* x, const double* y2, void* x2, cudaStream_t s);
// Two-pass sampling: add the newest basis vector of each vector to Xacc
// (and, with b.Xacc2, to Xacc2) after a step, and x = X (sum + compensation)
// at the end; the same arithmetic, in the same order, as launch_assemble.
cudaError_t launch_accumulate(bool fp64, size_t n, const LanczosBufs& b, cudaStream_t s);
cudaError_t launch_accumulate_finish(bool fp64, size_t n, const LanczosBufs& b, const void* X, void* x,
                                     cudaStream_t s);
// r = z - r in place for count elements of float or double.
cudaError_t launch_resid_form(bool z64, const void* z, bool r64, void* r, size_t count, cudaStream_t s);
// out[3 s .. 3 s + 2] = (r.r, r.t, t.t) in FP64 sums for nvec vectors [nvec][n]
// of float or double; part: kResidBlocks * nvec Dots<double> of scratch.
constexpr int kResidBlocks = 128;
cudaError_t launch_dots3(bool r64, const void* r, const void* t, size_t n, int nvec, void* part, double* out,
                         cudaStream_t s);
// out[3 s .. 3 s + 2] from the kResidBlocks partials of each of nvec vectors.
cudaError_t launch_dots3_final(const void* part, int nvec, double* out, cudaStream_t s);
// r = z - Q u for nvec FP32 vectors [nvec][n] of a lattice problem without a
// preconditioner, Q applied in pair-of-floats arithmetic (resid_df.cu), r
// rounded to FP32; out[3 s] = r.r (out[3 s + 1], out[3 s + 2] = 0); part:
// kResidBlocks * nvec Dots<double> of scratch.
cudaError_t launch_resid_df(const Grid& g, const float* kappa2, double kappa2_const, const float* z, const float* u,
                            float* r, int nvec, void* part, double* out, cudaStream_t s);
// The condition kernel of the device-side Lanczos loop: sets h to 1 while some
// of the nvec vectors is running and ++*ctr < limit, else 0.
cudaError_t launch_loop_cond(cudaGraphConditionalHandle h, const VecState* st, int nvec, int* ctr, int limit,
                             cudaStream_t s);
const void* loop_cond_kernel();  // the kernel itself, for a graph kernel node
cudaError_t launch_scale(bool fp64, void* x, size_t count, double a, cudaStream_t s);

// tridiag.cu ----------------------------------------------------------------
struct TmNodes {
  double s_lo;  // first node
  double h;     // node spacing
  int L;        // number of nodes
  int pad;
};
constexpr int kMaxNodes = 384;
// y[s] = T_m^{-1/2} e_1 (rational approximation from the Stieltjes integral),
// y stride = m_max.  scratch: >= nvec * kMaxNodes * m_max * 2 doubles.
cudaError_t launch_tm_inv_sqrt(const LanczosBufs& b, bool fp64, TmNodes* nodes, double* scratch, double* y,
                               cudaStream_t s);
// sparse.cu -----------------------------------------------------------------
// A general sparse Q (CSR) with an optional incomplete-Cholesky factor F of
// the preconditioner M = F F^T (Section 5.2).  Device copies, level schedules.
struct SparseOp;
// Validates and copies desc (see gmrf_create_sparse); *logdet_f = 2 sum log F_ii.
int sparse_create(SparseOp** out, const gmrf_sparse_desc* desc, bool fp64, cudaStream_t s, double* logdet_f);
void sparse_free(SparseOp* S, cudaStream_t s);
bool sparse_has_factor(const SparseOp* S);
int sparse_size(const SparseOp* S);
// One Lanczos step (Algorithm 1) on A = F^{-1} Q F^{-T} (or on Q without F):
// one block per vector, the same buffers and state as the lattice steps.
cudaError_t launch_sparse_step(const SparseOp& S, const LanczosBufs& b, const StepParams& P, cudaStream_t s);
// nvec vectors [nvec][n]: mode 0 y = Q v, 1 y = A v, 2 y = F^{-T} v, 3 y = F^{-1} v (modes 1-3 need F).
cudaError_t launch_sparse_ops(const SparseOp& S, int mode, const void* in, void* out, int nvec, cudaStream_t s);

// async.cu: runs what was submitted for p, then joins its worker (gmrf_destroy).
void async_shutdown(const gmrf_problem* p);
// y[s] = T_m^{-1} e_1 (linear solve), y and dwork stride = m_max (dwork: nvec * m_max doubles).
cudaError_t launch_tm_inv(const LanczosBufs& b, double* dwork, double* y, cudaStream_t s);
// q[s] = ||v_s||^2 e_1^T log(T_m) e_1 (Gauss quadrature, rational form).
cudaError_t launch_tm_log(const LanczosBufs& b, bool fp64, TmNodes* nodes, double* q, cudaStream_t s);
// out[0] = mean(q) + shift, out[1] = sd(q)/sqrt(N) (one block).
// out[0] = mean over draws of the sums of `group` consecutive q + shift,
// out[1] = standard error of that mean.
cudaError_t launch_logdet_reduce(const double* q, int nq, int group, double shift, double* out, cudaStream_t s);

}  // namespace gmrf
