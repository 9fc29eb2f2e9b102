// stencil_args.h -- kernel arguments of the fused stencil step (Algorithm 1
// with the matrix-free lattice apply of Q, Section 2), shared by the
// register-pipelined kernels and the TMA-staged 3-D kernel.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace gmrf {

template <typename T>
struct StencilArgs {
  const T* Win;  // apply mode: v
  T* Wout;       // apply mode: y
  T* W0;         // step mode: q ping-pong, W[j & 1] read, W[(j+1) & 1] written
  T* W1;
  T* V;  // basis ring base
  const float* kappa2;
  T kappa2_const;
  int nx, ny, nz;
  size_t n;
  int nzc;  // z chunks (3-D)
  StepParams P;
  VecState* st;
  double* alpha;
  double* beta;
  float* alpha_f;
  float* beta2_f;
  Dots<T>* partials;
  unsigned* counters;
};

struct Grid;

// stencil3d_tma.cu (eligibility and item counts are declared in internal.h)
// 16-byte alignment of the vector and coefficient pointers the kernel maps.
bool stencil3d_tma_pointers_ok(const void* win, const void* wout, const float* kappa2);
// step = true: fused Lanczos step on a.W0/W1/V; false: a.Wout = Q a.Win.
cudaError_t launch_stencil3d_tma(const Grid& g, const StencilArgs<float>& a, int nvec, bool step, cudaStream_t s);

// stencil2d_strip.cu: the 2-D step streamed down strips of rows, for grids
// with nx a multiple of 128 (FP32) / 64 (FP64) and at least 65536 cells.
bool stencil2d_strip_eligible(const Grid& g, bool fp64);
int stencil2d_strip_blocks_per_vector(const Grid& g, bool fp64);
bool stencil2d_strip_pointers_ok(const void* win, const void* wout, const float* kappa2);
template <typename T>
cudaError_t launch_stencil2d_strip(const Grid& g, const StencilArgs<T>& a, int nvec, bool step, cudaStream_t s);

}  // namespace gmrf
