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

#include <cstdint>

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

// ---- the shifted operators on pairs of cells (x, x + 1), x even, on paired
// FP32 instructions: the same pair-of-floats arithmetic per cell, half the
// issue slots.  Absent Neumann edges take the centre value (an exact zero
// term), Dirichlet ghosts 0, periodic neighbours wrap.
struct df2 {
  float2 hi, lo;
};
__device__ __forceinline__ float2 x2_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ df2 two_sum2(float2 a, float2 b) {
  const float2 s = x2_add(a, b);
  const float2 bb = x2_sub(s, a);
  return {s, x2_add(x2_sub(a, x2_sub(s, bb)), x2_sub(b, bb))};
}
__device__ __forceinline__ df2 fast_two_sum2(float2 a, float2 b) {  // |a| >= |b| per half
  const float2 s = x2_add(a, b);
  return {s, x2_sub(b, x2_sub(s, a))};
}
__device__ __forceinline__ df2 df_add2(df2 a, df2 b) {
  const df2 s = two_sum2(a.hi, b.hi);
  return fast_two_sum2(s.hi, x2_add(s.lo, x2_add(a.lo, b.lo)));
}
// a * b for a pair-of-floats a (the same for both cells) and the cells' floats b
__device__ __forceinline__ df2 df_mul_f2(df2 a, float2 b) {
  const float2 p = x2_mul(a.hi, b);
  const float2 e = x2_fma(a.hi, b, x2_neg(p));  // exact error of p
  return fast_two_sum2(p, x2_fma(a.lo, b, e));
}

template <int BC>
__device__ __forceinline__ float2 nb_pair(const float* __restrict__ u, const RGeo& g, int x, int y, int z, float2 c,
                                          int dy, int dz) {
  int yy = y + dy, zz = z + dz;
  const bool in = yy >= 0 && yy < g.ny && zz >= 0 && zz < g.nz;
  if (!in) {
    if (BC == GMRF_BC_NEUMANN) return c;
    if (BC == GMRF_BC_DIRICHLET) return make_float2(0.f, 0.f);
    yy = yy < 0 ? yy + g.ny : (yy >= g.ny ? yy - g.ny : yy);
    zz = zz < 0 ? zz + g.nz : (zz >= g.nz ? zz - g.nz : zz);
  }
  return __ldg(reinterpret_cast<const float2*>(u + cell(g, x, yy, zz)));
}
template <int BC>
__device__ __forceinline__ float nb_x(const float* __restrict__ u, const RGeo& g, int xx, int y, int z, float c) {
  if (xx < 0 || xx >= g.nx) {
    if (BC == GMRF_BC_NEUMANN) return c;
    if (BC == GMRF_BC_DIRICHLET) return 0.f;
    xx = xx < 0 ? xx + g.nx : xx - g.nx;
  }
  return __ldg(u + cell(g, xx, y, z));
}

template <int BC, int DIM>
__global__ void __launch_bounds__(kThreads) k_resid_df_pair(RGeo g, const float* __restrict__ k2, double kappa2_const,
                                                          const float* __restrict__ z, const float* __restrict__ u,
                                                          float* __restrict__ r, size_t n, Dots<double>* part) {
  __shared__ Dots<double> red[kThreads / 32];
  const int s = blockIdx.y;
  const float* us = u + (size_t)s * n;
  const float* zs = z + (size_t)s * n;
  float* rs = r + (size_t)s * n;
  const df kc1 = df_of(kappa2_const);
  const df2 kcp = {make_float2(kc1.hi, kc1.hi), make_float2(kc1.lo, kc1.lo)};
  const int px = g.nx / 2;
  const int npairs = px * g.ny * g.nz;
  df acc = {0.f, 0.f};
  for (int p = blockIdx.x * kThreads + threadIdx.x; p < npairs; p += gridDim.x * kThreads) {
    const int row = p / px;
    const int x = 2 * (p - row * px), y = row % g.ny, zz = row / g.ny;
    const size_t i = cell(g, x, y, zz);
    const float2 c = __ldg(reinterpret_cast<const float2*>(us + i));
    const df2 kap = k2 ? df2{__ldg(reinterpret_cast<const float2*>(k2 + i)), make_float2(0.f, 0.f)} : kcp;
    df2 q = df_mul_f2(kap, c);
    // x neighbours: (x - 1, x) on the left, (x + 1, x + 2) on the right
    const float2 lft = make_float2(nb_x<BC>(us, g, x - 1, y, zz, c.x), c.x);
    const float2 rgt = make_float2(c.y, nb_x<BC>(us, g, x + 2, y, zz, c.y));
    q = df_add2(q, two_sum2(c, x2_neg(lft)));
    q = df_add2(q, two_sum2(c, x2_neg(rgt)));
    q = df_add2(q, two_sum2(c, x2_neg(nb_pair<BC>(us, g, x, y, zz, c, -1, 0))));
    q = df_add2(q, two_sum2(c, x2_neg(nb_pair<BC>(us, g, x, y, zz, c, 1, 0))));
    if (DIM == 3) {
      q = df_add2(q, two_sum2(c, x2_neg(nb_pair<BC>(us, g, x, y, zz, c, 0, -1))));
      q = df_add2(q, two_sum2(c, x2_neg(nb_pair<BC>(us, g, x, y, zz, c, 0, 1))));
    }
    const df2 rd = df_add2({__ldg(reinterpret_cast<const float2*>(zs + i)), make_float2(0.f, 0.f)},
                           {x2_neg(q.hi), x2_neg(q.lo)});
    const float2 rv = x2_add(rd.hi, rd.lo);
    *reinterpret_cast<float2*>(rs + i) = rv;
    Dots<float>::dot2(acc, rv.x, rv.x);
    Dots<float>::dot2(acc, rv.y, rv.y);
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
  // pairs of cells: even rows (8-byte aligned pairs in every row of every vector) and aligned arrays
  const bool al = ((uintptr_t)u % 8 == 0) && ((uintptr_t)z % 8 == 0) && ((uintptr_t)r % 8 == 0) &&
                  ((uintptr_t)k2 % 8 == 0);
  if (OP == GMRF_OP_SHIFTED_LAPLACIAN && g.nx % 2 == 0 && al &&
      (int64_t)(g.nx / 2) * g.ny * g.nz < (int64_t)INT32_MAX - (int64_t)kResidBlocks * kThreads) {
    k_resid_df_pair<BC, DIM><<<dim3(kResidBlocks, nvec), kThreads, 0, s>>>(g, k2, kc, z, u, r, n, part);
    return cudaGetLastError();
  }
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
