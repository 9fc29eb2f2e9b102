// precond.h -- the constant-coefficient preconditioner of Section 5.1 and the
// preconditioned Lanczos step (Proposition 1).  Internal to the library.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "internal.h"

namespace gmrf {

enum { PRE_INV_SQRT = 0 };

// Form of the preconditioned operator A = M^{-1/2} Q M^{-1/2} (tau-free):
//   FORM_SHIFT  A = I + P R P, P = B_bar^{-1/2}, R = K - kappa_bar^2 (+ boundary edges)   (shifted Laplacian)
//   FORM_CTC    A = C^T C, C = I + R B_bar^{-1}, same R                                   (SPDE squared)
//   FORM_DIAG   A = I + P D P, P = B_bar^{-1}, R = D the diagonal field, no edge terms     (SPDE plus diagonal)
enum { FORM_SHIFT = 1, FORM_CTC = 2, FORM_DIAG = 3 };

// Tables and workspace of the preconditioner M = tau * B_bar^p with
// B_bar = kappa_bar^2 I + L_prec (L_prec the torus Laplacian for CIRCULANT,
// the cell-centred Neumann Laplacian for MIRROR), p = 1 (shifted Laplacian)
// or 2 (SPDE squared).  Its inverse square root (without tau) is
// P = B_bar^{-p/2}, diagonal in the transform basis with symbol
// (kappa_bar^2 + lambda_x + lambda_y)^{-p/2}.
struct PrecondTables {
  int kind = 0;   // GMRF_PREC_CIRCULANT or GMRF_PREC_MIRROR
  int power = 1;  // p (symbol exponent)
  int form = FORM_SHIFT;
  int nx = 0, ny = 0, lognx = 0, logny = 0;
  bool fp64 = false;
  double kbar2 = 0.0;
  void* lamx = nullptr;  // R[nx]: 1-D Laplacian eigenvalues in transform order
  void* lamy = nullptr;  // R[ny]
  void* twx = nullptr;   // C[nx]: exp(-2 pi i t / nx)
  void* twy = nullptr;   // C[ny]
  void* dctx = nullptr;  // C[nx+1]: exp(-i pi t / (2 nx))
  void* dcty = nullptr;  // C[ny+1]
  // FP32 mirror passes: for each pair k = 0 .. N/4 of a line of N points (L =
  // N/2), the 16 floats {tw[k], tw[L-k], dct[k], dct[N-k], dct[L-k],
  // dct[N-L+k], lam of the pair's four coefficients} (k = 0: lam[0], lam[L]),
  // stored as planes of N/4 + 1 float4 so that consecutive pairs are
  // contiguous: rows (N = nx) the first three planes, columns (N = ny) all four
  void* pairx = nullptr;
  void* pairy = nullptr;
  void* S = nullptr;     // spectral workspace, per vector spec_elems() complex/real pairs
  size_t S_bytes = 0;
  void* G = nullptr;     // g = C v workspace (SPDE squared), per vector n reals
  size_t G_bytes = 0;
  void* Wg = nullptr;    // w workspace (fast path with boundary terms in y), per vector n reals
  size_t Wg_bytes = 0;
  int rb = 4;            // rows per row-kernel block (generic path)
  int bc = 0;            // boundary condition of the problem
  bool fast = false;     // FP32 register-FFT kernels with the transposed spectrum
};

bool precond_size_ok(int64_t n);
int precond_build(PrecondTables& t, const Grid& g, int kind, int op, double kbar2, bool fp64, cudaStream_t s,
                  double* logdet_M);
void precond_free(PrecondTables& t, cudaStream_t s);
int precond_blocks_per_vector(const PrecondTables& t);
// Workspace for nvec vectors and kernel attributes; call before capturing
// the preconditioned steps into a CUDA graph.
int precond_prepare(PrecondTables& t, int nvec, cudaStream_t s);
size_t precond_extra_bytes(const PrecondTables& t, size_t es);
// Fused preconditioned Lanczos step j (A = M^{-1/2} Q M^{-1/2}, applied as
// C^T C with C = I + R B_bar^{-1} for the squared operator and as
// I + P R P for the shifted one, R = B - B_bar).
cudaError_t launch_precond_step(PrecondTables& t, const Grid& g, bool fp64, const void* kappa2, double kappa2_const,
                                const LanczosBufs& b, const StepParams& P, cudaStream_t s);
// out = B_bar^{-p/2} in for nvec vectors (tau not applied).
cudaError_t launch_precond_apply(PrecondTables& t, const Grid& g, bool fp64, int which, const void* in, void* out,
                                 int nvec, cudaStream_t s);
// Same as launch_precond_apply, but the spectrum lives in the caller's
// workspace S of at least precond_apply_scratch_bytes(t, nvec) bytes; no
// device memory is allocated.
size_t precond_apply_scratch_bytes(const PrecondTables& t, int nvec);
cudaError_t launch_precond_apply_with(PrecondTables& t, const Grid& g, bool fp64, const void* in, void* out, int nvec,
                                      void* S, cudaStream_t s);
// y = A v for nvec vectors.
cudaError_t launch_precond_operator(PrecondTables& t, const Grid& g, bool fp64, const void* kappa2,
                                    double kappa2_const, const void* v, void* y, int nvec, cudaStream_t s);

}  // namespace gmrf
