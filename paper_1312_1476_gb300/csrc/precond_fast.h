// precond_fast.h -- entry points of the FP32 warp-FFT preconditioner kernels
// (precond_fast.cuh), one translation unit per preconditioner kind.
#pragma once

#include <cuda_runtime.h>

#include "precond.h"

namespace gmrf {
namespace fast {

// Arguments of the FP32 register-FFT preconditioner kernels.
struct Args {
  int nx, ny, bc, power;
  int form;      // FORM_SHIFT / FORM_CTC / FORM_DIAG (precond.h)
  float kbar2, dscale;
  float roff;    // R = K - roff
  const float* lamx;
  const float* lamy;
  const float2* twx;   // exp(-2 pi i t / nx)
  const float2* twy;   // exp(-2 pi i t / ny)
  const float2* dctx;  // exp(-i pi t / (2 nx)), t <= nx
  const float2* dcty;
  const float4* pairx; // mirror rows: 3 planes of nx/4 + 1 float4 (see PrecondTables::pairx)
  const float4* pairy; // mirror columns: 4 planes of ny/4 + 1 float4 (see PrecondTables::pairy)
  float* T;            // transposed spectrum
  size_t tstride;      // floats per vector
  float* G;            // g = C v (squared operator)
  float* Wg;           // w when the y-boundary terms need a separate pass
  const float* in;
  float* out;
  const float* kappa2;
  float kappa2_const;
  size_t n;
  float* W0;
  float* W1;
  float* V;
  StepParams P;
  VecState* st;
  double* alpha;
  double* beta;
  float* alpha_f;
  float* beta2_f;
  Dots<float>* partials;
  unsigned* counters;
};

}  // namespace fast

// The FP32 path with register FFTs covers nx in [128, 2048] and ny in
// [64, 1024] (circulant) or [128, 2048] (mirror), powers of two.
bool fast_eligible(int kind, bool fp64, int nx, int ny);
int fast_rows_per_block(int kind, int nx);

cudaError_t fast_step_circ(const fast::Args& a, int nvec, cudaStream_t s);
cudaError_t fast_apply_circ(const fast::Args& a, int nvec, cudaStream_t s);
cudaError_t fast_operator_circ(const fast::Args& a, int nvec, cudaStream_t s);
cudaError_t fast_step_mirror(const fast::Args& a, int nvec, cudaStream_t s);
cudaError_t fast_apply_mirror(const fast::Args& a, int nvec, cudaStream_t s);
cudaError_t fast_operator_mirror(const fast::Args& a, int nvec, cudaStream_t s);

}  // namespace gmrf
