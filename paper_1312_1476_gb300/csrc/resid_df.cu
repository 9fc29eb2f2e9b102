// resid_df.cu -- the residual r = z - Q u of an FP32 iterate u on a lattice
// precision (no preconditioner), for the accuracy check of samples.
//
// Theorem 1 bounds the error of the Lanczos sample by the residual of the CG
// iterate u_m = ||z|| V_m T_m^{-1} e_1.  Near convergence Q u_m agrees with z
// to about the tolerance, so z - Q u_m cancels almost all of its digits, and
// for a smooth u_m so do the stencil's own terms.  Formed in FP32 the result
// would be rounding noise.  Here every product is exact (TwoProd by FMA) and
// every sum is carried as an unevaluated pair of floats (TwoSum), about 48
// significant bits, all on the FP32 pipe: FP64 arithmetic runs far slower
// than FP32 on this GPU, and a pair of floats resolves r to the same relative
// accuracy that FP64 would.  r is rounded to FP32 once formed (its own digits
// do not cancel any more), and r.r is summed per block in Dot2 form.
//
// Operators (the same definitions as the Lanczos step kernels):
//   shifted:         (B u)_c = kappa_c^2 u_c + sum over the edges of c of (u_c - u_nb)
//   squared (2-D):   Q u = B (B u)
//   plus-diag (2-D): Q u = B_c (B_c u) + D u, B_c with the constant kappa2_const, D = diag(field)
// Dirichlet neighbours outside the grid are 0 (the edge is there), Neumann
// edges leaving the grid are absent, periodic neighbours wrap; for the
// squared forms B u outside a Dirichlet grid is 0.
//
// Launch: grid (kResidBlocks, nvec); block b of vector s walks the grid rows
// b, b + kResidBlocks, ...  The partial sums depend on the grid alone, so a
// vector's r.r does not depend on the batch it is checked in.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace gmrf {
namespace {

constexpr int kThreads = 256;

struct RGeo {
  int nx, ny, nz;
};

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// a * b for a pair a and a float b, to the pair's precision
__device__ __forceinline__ df df_mul_f(df a, float b) {
  const df p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// a * b for two pairs, to the pair's precision
__device__ __forceinline__ df df_mul(df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  return fast_two_sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}

__device__ __forceinline__ df df_of(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

__device__ __forceinline__ size_t cell(const RGeo& g, int x, int y, int z) {
  return (size_t)x + (size_t)g.nx * ((size_t)y + (size_t)g.ny * z);
}

// Neighbour (x + dx, y + dy, z + dz) of a cell under the boundary condition:
// returns false when the edge is absent (Neumann); otherwise *ghost tells a
// Dirichlet neighbour outside the grid (value 0), else (nxo, nyo, nzo) is the
// neighbour, wrapped on a periodic grid.
template <int BC>
__device__ __forceinline__ bool neighbour(const RGeo& g, int x, int y, int z, int dx, int dy, int dz, int& nxo,
                                          int& nyo, int& nzo, bool& ghost) {
  nxo = x + dx;
  nyo = y + dy;
  nzo = z + dz;
  const bool in = nxo >= 0 && nxo < g.nx && nyo >= 0 && nyo < g.ny && nzo >= 0 && nzo < g.nz;
  ghost = false;
  if (in) return true;
  if (BC == GMRF_BC_NEUMANN) return false;
  if (BC == GMRF_BC_DIRICHLET) {
    ghost = true;
    return true;
  }
  nxo = nxo < 0 ? nxo + g.nx : (nxo >= g.nx ? nxo - g.nx : nxo);
  nyo = nyo < 0 ? nyo + g.ny : (nyo >= g.ny ? nyo - g.ny : nyo);
  nzo = nzo < 0 ? nzo + g.nz : (nzo >= g.nz ? nzo - g.nz : nzo);
  return true;
}

__constant__ int kDir[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};

// (B u)_c for the float field u, coefficient kap at c
template <int BC, int DIM>
__device__ __forceinline__ df b_float(const float* __restrict__ u, const RGeo& g, int x, int y, int z, df kap) {
  const float uc = __ldg(u + cell(g, x, y, z));
  df acc = df_mul_f(kap, uc);
#pragma unroll
  for (int d = 0; d < 2 * DIM; ++d) {
    int a, b, c;
    bool ghost;
    if (!neighbour<BC>(g, x, y, z, kDir[d][0], kDir[d][1], kDir[d][2], a, b, c, ghost)) continue;
    const float un = ghost ? 0.f : __ldg(u + cell(g, a, b, c));
    acc = df_add(acc, two_sum(uc, -un));
  }
  return acc;
}

template <int OP>
__device__ __forceinline__ df kap_at(const float* __restrict__ k2, df kc, size_t i) {
  if (OP == GMRF_OP_SPDE_PLUS_DIAG || !k2) return kc;
  return {__ldg(k2 + i), 0.f};
}

// (Q u)_c
template <int OP, int BC, int DIM>
__device__ __forceinline__ df q_at(const float* __restrict__ u, const float* __restrict__ k2, df kc, const RGeo& g,
                                   int x, int y, int z) {
  const size_t ic = cell(g, x, y, z);
  if (OP == GMRF_OP_SHIFTED_LAPLACIAN) return b_float<BC, DIM>(u, g, x, y, z, kap_at<OP>(k2, kc, ic));
  // squared forms (2-D): B applied to g = B u
  const df kcc = kap_at<OP>(k2, kc, ic);
  const df gc = b_float<BC, 2>(u, g, x, y, 0, kcc);
  df acc = df_mul(kcc, gc);
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    int a, b, c;
    bool ghost;
    if (!neighbour<BC>(g, x, y, 0, kDir[d][0], kDir[d][1], 0, a, b, c, ghost)) continue;
    const df gn = ghost ? df{0.f, 0.f} : b_float<BC, 2>(u, g, a, b, 0, kap_at<OP>(k2, kc, cell(g, a, b, 0)));
    acc = df_add(acc, df_add(gc, df_neg(gn)));
  }
  if (OP == GMRF_OP_SPDE_PLUS_DIAG && k2) acc = df_add(acc, two_prod(__ldg(k2 + ic), __ldg(u + ic)));
  return acc;
}

template <int OP, int BC, int DIM>
__global__ void __launch_bounds__(kThreads) k_resid_df(RGeo g, const float* __restrict__ k2, double kappa2_const,
                                                     const float* __restrict__ z, const float* __restrict__ u,
                                                     float* __restrict__ r, size_t n, Dots<double>* part) {
  __shared__ Dots<double> red[kThreads / 32];
  const int s = blockIdx.y;
  const float* us = u + (size_t)s * n;
  const float* zs = z + (size_t)s * n;
  float* rs = r + (size_t)s * n;
  const df kc = df_of(kappa2_const);
  df acc = {0.f, 0.f};
  const int rows = g.ny * g.nz;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int y = row % g.ny, zz = row / g.ny;
    for (int x = threadIdx.x; x < g.nx; x += kThreads) {
      const size_t i = cell(g, x, y, zz);
      const df qu = q_at<OP, BC, DIM>(us, k2, kc, g, x, y, zz);
      const df rd = df_add({__ldg(zs + i), 0.f}, df_neg(qu));
      const float rv = __fadd_rn(rd.hi, rd.lo);
      rs[i] = rv;
      Dots<float>::dot2(acc, rv, rv);
    }
  }
  Dots<double> d;
  d.s1 = df_to_double(acc);
  d.s2 = 0.0;
  d.s3 = 0.0;
  d = block_reduce(d, red);
  if (threadIdx.x == 0) part[(size_t)s * gridDim.x + blockIdx.x] = d;
}

template <int OP, int BC, int DIM>
cudaError_t launch_one(const RGeo& g, const float* k2, double kc, const float* z, const float* u, float* r, size_t n,
                       int nvec, Dots<double>* part, cudaStream_t s) {
  k_resid_df<OP, BC, DIM><<<dim3(kResidBlocks, nvec), kThreads, 0, s>>>(g, k2, kc, z, u, r, n, part);
  return cudaGetLastError();
}

template <int OP, int DIM>
cudaError_t launch_bc(int bc, const RGeo& g, const float* k2, double kc, const float* z, const float* u, float* r,
                      size_t n, int nvec, Dots<double>* part, cudaStream_t s) {
  switch (bc) {
    case GMRF_BC_PERIODIC: return launch_one<OP, GMRF_BC_PERIODIC, DIM>(g, k2, kc, z, u, r, n, nvec, part, s);
    case GMRF_BC_NEUMANN: return launch_one<OP, GMRF_BC_NEUMANN, DIM>(g, k2, kc, z, u, r, n, nvec, part, s);
    case GMRF_BC_DIRICHLET: return launch_one<OP, GMRF_BC_DIRICHLET, DIM>(g, k2, kc, z, u, r, n, nvec, part, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_resid_df(const Grid& g, const float* kappa2, double kappa2_const, const float* z, const float* u,
                            float* r, int nvec, void* part, double* out, cudaStream_t s) {
  const RGeo geo{g.nx, g.ny, g.dim == 3 ? g.nz : 1};
  Dots<double>* pt = (Dots<double>*)part;
  cudaError_t e = cudaErrorInvalidValue;
  if (g.dim == 3) {
    if (g.op == GMRF_OP_SHIFTED_LAPLACIAN)
      e = launch_bc<GMRF_OP_SHIFTED_LAPLACIAN, 3>(g.bc, geo, kappa2, kappa2_const, z, u, r, g.n, nvec, pt, s);
  } else if (g.op == GMRF_OP_SHIFTED_LAPLACIAN) {
    e = launch_bc<GMRF_OP_SHIFTED_LAPLACIAN, 2>(g.bc, geo, kappa2, kappa2_const, z, u, r, g.n, nvec, pt, s);
  } else if (g.op == GMRF_OP_SPDE_SQUARED) {
    e = launch_bc<GMRF_OP_SPDE_SQUARED, 2>(g.bc, geo, kappa2, kappa2_const, z, u, r, g.n, nvec, pt, s);
  } else if (g.op == GMRF_OP_SPDE_PLUS_DIAG) {
    e = launch_bc<GMRF_OP_SPDE_PLUS_DIAG, 2>(g.bc, geo, kappa2, kappa2_const, z, u, r, g.n, nvec, pt, s);
  }
  if (e != cudaSuccess) return e;
  return launch_dots3_final(part, nvec, out, s);
}

}  // namespace gmrf
