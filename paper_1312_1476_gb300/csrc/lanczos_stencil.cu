// lanczos_stencil.cu -- one Lanczos step of Algorithm 1 fused with the
// matrix-free lattice apply of Q (Section 2: "a routine that computes the
// matrix-vector product without ever forming or storing Q").
//
// Step j (0-based) for vector s, in one pass over the grid:
//   v_j   = (q_{j-1} - alpha_{j-1} v_{j-1}) / beta_{j-1}     (v_0 = z / ||z||)
//           formed on load from W_in = q_{j-1} and the stored v_{j-1}, also
//           on the halo cells, and written to the basis ring;
//   q_j   = Q v_j - beta_{j-1} v_{j-1}                         -> W_out
//   sums  v_j.q_j, q_j.q_j, v_j.v_j  (compensated FP32 or FP64)
// and the last block of the vector forms alpha_j = v_j.q_j and
//   beta_j = ||q_j - alpha_j v_j|| = sqrt(q.q - 2 alpha v.q + alpha^2 v.v)
// and applies the stopping rule (common.cuh).
//
// Stencils (difference form: (L v)_i = sum over existing edges (v_i - v_nb),
// which keeps the FP32 rounding relative to the result for smooth v):
//   shifted:  B v = kappa^2 v + L v            (5-point 2-D, 7-point 3-D)
//   squared:  Q v = B (B v)                    (13-point 2-D, two passes in smem)
// 2-D: 32x16 tiles with a halo of 1 (shifted) or 2 (squared) in shared memory.
// 3-D: 32x8 tiles in x-y marching over a chunk of z planes with the inputs of
// later planes prefetched; the centre column is kept in registers, the plane
// with its x-y halo in a double-buffered shared tile.
#include <cuda_runtime.h>

#include "internal.h"
#include "stencil_args.h"

namespace gmrf {
namespace {

constexpr int TX = 32;
constexpr int TY = 16;
constexpr int NT = TX * TY;

__device__ __forceinline__ int wrapi(int g, int n) {
  g %= n;
  return g < 0 ? g + n : g;
}

template <typename T>
__device__ __forceinline__ T kap_at(const float* k, T kc, size_t i) {
  return k ? (T)__ldg(k + i) : kc;
}

// B applied at smem position (cx, cy) of array a with pitch W, for the cell at
// global (gx, gy) with coefficient kap.  Neumann edges leaving the grid are
// absent; Dirichlet and periodic neighbours come from the (zero / wrapped) halo.
template <typename T, int BC, int W>
__device__ __forceinline__ T bop2(const T* a, int cx, int cy, int gx, int gy, int nx, int ny, T kap) {
  const T c = a[cy * W + cx];
  T r = kap * c;
  if (BC != GMRF_BC_NEUMANN || gx > 0) r += c - a[cy * W + cx - 1];
  if (BC != GMRF_BC_NEUMANN || gx < nx - 1) r += c - a[cy * W + cx + 1];
  if (BC != GMRF_BC_NEUMANN || gy > 0) r += c - a[(cy - 1) * W + cx];
  if (BC != GMRF_BC_NEUMANN || gy < ny - 1) r += c - a[(cy + 1) * W + cx];
  return r;
}

// STEP = true: fused Lanczos step.  STEP = false: y = Q v (Win = v, Wout = y).
// SPDE_PLUS_DIAG: Q v = B(B v) + D v with B = kappa_c^2 I + L (constant
// coefficient, kappa2_const) and D = diag(kappa2 field, or 0).
template <typename T, int OP, int BC, bool STEP>
__global__ void __launch_bounds__(NT) k_stencil2d(StencilArgs<T> a) {
  constexpr bool SQ = OP != GMRF_OP_SHIFTED_LAPLACIAN;  // B applied twice
  constexpr int H = SQ ? 2 : 1;
  constexpr int VW = TX + 2 * H, VH = TY + 2 * H;
  constexpr int GW = TX + 2, GH = TY + 2;
  __shared__ T vs[VH * VW];
  __shared__ T gs[SQ ? GH * GW : 1];
  __shared__ Dots<T> red[NT / 32];
  __shared__ int s_int[4];
  __shared__ float s_flt[4];

  const int s = blockIdx.z;
  int j = 0;
  if (STEP) {
    if (a.st[s].status != VS_RUNNING) return;
    j = a.st[s].m;
  }
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int nx = a.nx, ny = a.ny;
  const size_t n = a.n;
  const T* Win = (STEP ? ((j & 1) ? a.W1 : a.W0) : a.Win) + (size_t)s * n;
  T* Wout = (STEP ? ((j & 1) ? a.W0 : a.W1) : a.Wout) + (size_t)s * n;
  const T* Vp = nullptr;
  T* Vc = nullptr;
  T coef = 0, inv_b = 1, bprev = 0;
  if (STEP) {
    const size_t base = (size_t)s * a.P.nslots;
    Vc = a.V + (base + (size_t)(j % a.P.nslots)) * n;
    if (j == 0) {
      inv_b = (T)a.st[s].vscale;
    } else {
      Vp = a.V + (base + (size_t)((j - 1) % a.P.nslots)) * n;
      const size_t mo = (size_t)s * a.P.m_max + (j - 1);
      coef = (T)a.alpha[mo];
      bprev = (T)a.beta[mo];
      inv_b = (T)a.st[s].vscale;
    }
  }
  // ---- load v_j on tile + halo
  for (int idx = tid; idx < VH * VW; idx += NT) {
    const int cy = idx / VW, cx = idx - cy * VW;
    int gx = x0 - H + cx, gy = y0 - H + cy;
    bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
    if (!in && BC == GMRF_BC_PERIODIC) {
      gx = wrapi(gx, nx);
      gy = wrapi(gy, ny);
      in = true;
    }
    T val = 0;
    if (in) {
      const size_t i = (size_t)gx + (size_t)nx * gy;
      const T w = Win[i];
      if (!STEP) val = w;
      else if (j == 0) val = w * inv_b;
      else val = (w - coef * Vp[i]) * inv_b;
    }
    vs[idx] = val;
  }
  __syncthreads();
  if (SQ) {
    for (int idx = tid; idx < GH * GW; idx += NT) {
      const int py = idx / GW, px = idx - py * GW;
      int gx = x0 - 1 + px, gy = y0 - 1 + py;
      bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
      if (!in && BC == GMRF_BC_PERIODIC) {
        gx = wrapi(gx, nx);
        gy = wrapi(gy, ny);
        in = true;
      }
      T g = 0;
      if (in) {
        const T kap = OP == GMRF_OP_SPDE_PLUS_DIAG ? a.kappa2_const
                                                   : kap_at<T>(a.kappa2, a.kappa2_const, (size_t)gx + (size_t)nx * gy);
        g = bop2<T, BC, VW>(vs, px + 1, py + 1, gx, gy, nx, ny, kap);
      }
      gs[idx] = g;
    }
    __syncthreads();
  }
  const int gx = x0 + tx, gy = y0 + ty;
  const bool own = gx < nx && gy < ny;
  Dots<T> d;
  d.zero();
  if (own) {
    const size_t i = (size_t)gx + (size_t)nx * gy;
    const T kap = OP == GMRF_OP_SPDE_PLUS_DIAG ? a.kappa2_const : kap_at<T>(a.kappa2, a.kappa2_const, i);
    T qv;
    if (SQ) qv = bop2<T, BC, GW>(gs, tx + 1, ty + 1, gx, gy, nx, ny, kap);
    else qv = bop2<T, BC, VW>(vs, tx + H, ty + H, gx, gy, nx, ny, kap);
    if (OP == GMRF_OP_SPDE_PLUS_DIAG && a.kappa2) qv += (T)__ldg(a.kappa2 + i) * vs[(ty + H) * VW + tx + H];
    if (!STEP) {
      Wout[i] = qv;
    } else {
      const T v = vs[(ty + H) * VW + tx + H];
      T q = qv;
      if (j > 0) q -= bprev * Vp[i];
      Wout[i] = q;
      Vc[i] = v;
      if (a.P.vb) vb_store1(vb_at(a.P, s, j, a.n, i), (float)v);
      d.add(v, q);
    }
  }
  if (!STEP) return;
  d = block_reduce(d, red);
  const int nblk = gridDim.x * gridDim.y;
  if (tid == 0) a.partials[(size_t)s * nblk + blockIdx.x + gridDim.x * blockIdx.y] = d;
  if (last_block(a.counters, s, nblk, &s_int[3]))
    finish_step<T>(a.P, j, s, a.partials, nblk, a.st, a.alpha, a.beta, a.alpha_f, a.beta2_f, red, s_int, s_flt);
}

// 3-D shifted Laplacian (7-point), z-march over a chunk of planes, software
// pipelined: the raw inputs (q_{j-1}, v_{j-1}, kappa^2) of a thread's own
// cells are loaded two planes ahead and those of the x-y halo ring one plane
// ahead, so the loads of later planes are in flight while a plane is
// computed; the plane with its halo lives in a double-buffered shared tile
// (one barrier per plane).  Each thread owns VX adjacent cells along x
// (vector loads), the block a (32 VX) x 8 tile.
constexpr int TY3 = 8;
constexpr int NT3 = TX * TY3;

template <typename T, int VX>
struct Raw {
  T w[VX], vp[VX];
  float k[VX];
};

template <typename T, int VX>
__device__ __forceinline__ void vload(const T* p, T* o) {
  if (VX == 1) o[0] = p[0];
  else if (VX == 2 && sizeof(T) == 4) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    o[0] = v.x; o[1] = v.y;
  } else if (VX == 4 && sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else if (VX == 2 && sizeof(T) == 8) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
  } else {
#pragma unroll
    for (int e = 0; e < VX; ++e) o[e] = p[e];
  }
}
template <typename T, int VX>
__device__ __forceinline__ void vstore(T* p, const T* o) {
  if (VX == 1) p[0] = o[0];
  else if (VX == 2 && sizeof(T) == 4) *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
  else if (VX == 4 && sizeof(T) == 4) *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  else if (VX == 2 && sizeof(T) == 8) *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
  else {
#pragma unroll
    for (int e = 0; e < VX; ++e) p[e] = o[e];
  }
}

template <typename T, int BC, bool STEP, int VX>
__global__ void __launch_bounds__(NT3) k_stencil3d(StencilArgs<T> a) {
  constexpr int BX = TX * VX;  // tile width in cells
  constexpr int PW = BX + 2, PH = TY3 + 2, PSZ = PW * PH;
  constexpr int NRING = 2 * PW + 2 * TY3;
  constexpr int RPT = (NRING + NT3 - 1) / NT3;  // ring cells per thread
  __shared__ T ps[2][PSZ];
  __shared__ Dots<T> red[NT3 / 32];
  __shared__ int s_int[4];
  __shared__ float s_flt[4];
  const int s = blockIdx.z / a.nzc;
  const int zc = blockIdx.z - s * a.nzc;
  int j = 0;
  if (STEP) {
    if (a.st[s].status != VS_RUNNING) return;
    j = a.st[s].m;
  }
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t n = a.n, plane = (size_t)nx * ny;
  const int zper = (nz + a.nzc - 1) / a.nzc;
  const int z0 = zc * zper, z1 = min(nz, z0 + zper);
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * TY3;
  const T* Win = (STEP ? ((j & 1) ? a.W1 : a.W0) : a.Win) + (size_t)s * n;
  T* Wout = (STEP ? ((j & 1) ? a.W0 : a.W1) : a.Wout) + (size_t)s * n;
  const T* Vp = nullptr;
  T* Vc = nullptr;
  T coef = 0, inv_b = 1, bprev = 0;
  if (STEP) {
    const size_t base = (size_t)s * a.P.nslots;
    Vc = a.V + (base + (size_t)(j % a.P.nslots)) * n;
    if (j == 0) {
      inv_b = (T)a.st[s].vscale;
    } else {
      Vp = a.V + (base + (size_t)((j - 1) % a.P.nslots)) * n;
      const size_t mo = (size_t)s * a.P.m_max + (j - 1);
      coef = (T)a.alpha[mo];
      bprev = (T)a.beta[mo];
      inv_b = (T)a.st[s].vscale;
    }
  }
  auto fv = [&](T w, T vp) -> T {
    if (!STEP) return w;
    if (j == 0) return w * inv_b;
    return (w - coef * vp) * inv_b;
  };
  // raw inputs of one cell (ring); outside the grid per boundary condition
  auto load1 = [&](int gx, int gy, int gz, T& w, T& vp) {
    w = vp = (T)0;
    bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz;
    if (!in && BC == GMRF_BC_PERIODIC) {
      gx = wrapi(gx, nx);
      gy = wrapi(gy, ny);
      gz = wrapi(gz, nz);
      in = true;
    }
    if (!in) return;
    const size_t i = (size_t)gx + (size_t)nx * gy + plane * gz;
    w = Win[i];
    if (STEP && j > 0) vp = Vp[i];
  };
  // raw inputs of the thread's VX cells (x = gx .. gx + VX - 1, all inside or
  // all outside the grid in x since nx % VX == 0)
  const int gx = x0 + tx * VX, gy = y0 + ty;
  const bool own = gx < nx && gy < ny;
  auto loadv = [&](int gz, Raw<T, VX>& r) {
#pragma unroll
    for (int e = 0; e < VX; ++e) {
      r.w[e] = r.vp[e] = (T)0;
      r.k[e] = 0.f;
    }
    int zz = gz, yy = gy;
    bool in = own && gz >= 0 && gz < nz;
    if (!in && BC == GMRF_BC_PERIODIC && own) {
      zz = wrapi(gz, nz);
      in = true;
    }
    if (!in) {
      if (BC == GMRF_BC_PERIODIC && !own) {
        // partial tile in a periodic grid: wrapped neighbours still needed
#pragma unroll
        for (int e = 0; e < VX; ++e) load1(gx + e, gy, gz, r.w[e], r.vp[e]);
      }
      return;
    }
    const size_t i = (size_t)gx + (size_t)nx * yy + plane * zz;
    vload<T, VX>(Win + i, r.w);
    if (STEP && j > 0) vload<T, VX>(Vp + i, r.vp);
    if (a.kappa2) {
      if (VX == 4) {
        const float4 kk = *reinterpret_cast<const float4*>(a.kappa2 + i);
        r.k[0] = kk.x; r.k[1] = kk.y; r.k[2 % VX] = kk.z; r.k[3 % VX] = kk.w;
      } else if (VX == 2) {
        const float2 kk = *reinterpret_cast<const float2*>(a.kappa2 + i);
        r.k[0] = kk.x; r.k[1 % VX] = kk.y;
      } else {
        r.k[0] = __ldg(a.kappa2 + i);
      }
    } else {
#pragma unroll
      for (int e = 0; e < VX; ++e) r.k[e] = (float)a.kappa2_const;
    }
  };
  // halo ring cells of this thread
  int rcx[RPT], rcy[RPT];
  bool rin[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int r = tid + q * NT3;
    rin[q] = r < NRING;
    rcx[q] = rcy[q] = 0;
    if (r < PW) { rcx[q] = r; rcy[q] = 0; }
    else if (r < 2 * PW) { rcx[q] = r - 2 * 0 - PW; rcy[q] = PH - 1; }
    else if (r < 2 * PW + TY3) { rcx[q] = 0; rcy[q] = r - 2 * PW + 1; }
    else if (r < NRING) { rcx[q] = PW - 1; rcy[q] = r - 2 * PW - TY3 + 1; }
  }
  Dots<T> d;
  d.zero();
  Raw<T, VX> rc, r1, r2;
  T rgw[RPT], rgv[RPT];
  T vdn[VX], vc[VX];
#pragma unroll
  for (int e = 0; e < VX; ++e) vdn[e] = vc[e] = (T)0;
  if (z0 < z1) {
    Raw<T, VX> rm;
    loadv(z0 - 1, rm);
    loadv(z0, rc);
    loadv(z0 + 1, r1);
    loadv(z0 + 2, r2);
#pragma unroll
    for (int q = 0; q < RPT; ++q)
      if (rin[q]) load1(x0 - 1 + rcx[q], y0 - 1 + rcy[q], z0, rgw[q], rgv[q]);
#pragma unroll
    for (int e = 0; e < VX; ++e) {
      vdn[e] = fv(rm.w[e], rm.vp[e]);
      vc[e] = fv(rc.w[e], rc.vp[e]);
    }
  }
  for (int z = z0; z < z1; ++z) {
    const int b = (z - z0) & 1;
    T vup[VX];
#pragma unroll
    for (int e = 0; e < VX; ++e) vup[e] = fv(r1.w[e], r1.vp[e]);
    // loads for later planes, in flight while this plane is computed
    Raw<T, VX> r3;
    loadv(z + 3, r3);
    T rgwn[RPT], rgvn[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      rgwn[q] = rgvn[q] = (T)0;
      if (rin[q]) load1(x0 - 1 + rcx[q], y0 - 1 + rcy[q], z + 1, rgwn[q], rgvn[q]);
    }
#pragma unroll
    for (int e = 0; e < VX; ++e) ps[b][(ty + 1) * PW + tx * VX + e + 1] = vc[e];
#pragma unroll
    for (int q = 0; q < RPT; ++q)
      if (rin[q]) ps[b][rcy[q] * PW + rcx[q]] = fv(rgw[q], rgv[q]);
    __syncthreads();
    if (own) {
      const size_t i = (size_t)gx + (size_t)nx * gy + plane * z;
      T qo[VX];
#pragma unroll
      for (int e = 0; e < VX; ++e) {
        T r = bop2<T, BC, PW>(ps[b], tx * VX + e + 1, ty + 1, gx + e, gy, nx, ny, (T)rc.k[e]);
        if (BC != GMRF_BC_NEUMANN || z > 0) r += vc[e] - vdn[e];
        if (BC != GMRF_BC_NEUMANN || z < nz - 1) r += vc[e] - vup[e];
        if (STEP && j > 0) r -= bprev * rc.vp[e];
        qo[e] = r;
        if (STEP) d.add(vc[e], r);
      }
      vstore<T, VX>(Wout + i, qo);
      if (STEP) {
        vstore<T, VX>(Vc + i, vc);
        if (a.P.vb) {
          __nv_bfloat16* pb = vb_at(a.P, s, j, n, i);
          if (VX == 4) vb_store4(pb, (float)vc[0], (float)vc[1 % VX], (float)vc[2 % VX], (float)vc[3 % VX]);
          else if (VX == 2) vb_store2(pb, (float)vc[0], (float)vc[1 % VX]);
          else vb_store1(pb, (float)vc[0]);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < VX; ++e) {
      vdn[e] = vc[e];
      vc[e] = vup[e];
    }
    rc = r1;
    r1 = r2;
    r2 = r3;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      rgw[q] = rgwn[q];
      rgv[q] = rgvn[q];
    }
  }
  if (!STEP) return;
  d = block_reduce(d, red);
  const int nblk = gridDim.x * gridDim.y * a.nzc;
  if (tid == 0) a.partials[(size_t)s * nblk + blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * zc)] = d;
  if (last_block(a.counters, s, nblk, &s_int[3]))
    finish_step<T>(a.P, j, s, a.partials, nblk, a.st, a.alpha, a.beta, a.alpha_f, a.beta2_f, red, s_int, s_flt);
}

// cells per thread along x for the 3-D kernel
int vx3(const Grid& g, bool fp64) {
  if (!fp64 && g.nx % 4 == 0 && g.nx >= 128) return 4;
  if (g.nx % 2 == 0 && g.nx >= 64) return 2;
  return 1;
}

int nz_chunks(const Grid& g, int vx) {
  if (g.dim != 3) return 1;
  const int tiles = ((g.nx + TX * vx - 1) / (TX * vx)) * ((g.ny + TY3 - 1) / TY3);
  int c = 1;
  while (c < g.nz && tiles * c < 4 * 152 && (g.nz + 2 * c - 1) / (2 * c) >= 8) c *= 2;
  return c;
}

template <typename T, bool STEP>
cudaError_t dispatch(const Grid& g, StencilArgs<T> a, int nvec, cudaStream_t s) {
  dim3 blk(TX, TY);
  dim3 grd((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, nvec);
  if (g.dim == 3) {
    if (g.op != GMRF_OP_SHIFTED_LAPLACIAN) return cudaErrorNotSupported;
    if constexpr (sizeof(T) == 4) {
      if (stencil3d_tma_eligible(g, false) &&
          (STEP || stencil3d_tma_pointers_ok(a.Win, a.Wout, a.kappa2)))
        return launch_stencil3d_tma(g, a, nvec, STEP, s);
    }
    const int vx = vx3(g, sizeof(T) == 8);
    a.nzc = nz_chunks(g, vx);
    blk = dim3(TX, TY3);
    grd = dim3((g.nx + TX * vx - 1) / (TX * vx), (g.ny + TY3 - 1) / TY3, nvec * a.nzc);
#define GMRF_L3(BCV, VXV) k_stencil3d<T, BCV, STEP, VXV><<<grd, blk, 0, s>>>(a)
#define GMRF_L3V(BCV) \
  do {                \
    if (vx == 4) GMRF_L3(BCV, 4); \
    else if (vx == 2) GMRF_L3(BCV, 2); \
    else GMRF_L3(BCV, 1); \
  } while (0)
    switch (g.bc) {
      case GMRF_BC_PERIODIC: GMRF_L3V(GMRF_BC_PERIODIC); break;
      case GMRF_BC_NEUMANN: GMRF_L3V(GMRF_BC_NEUMANN); break;
      default: GMRF_L3V(GMRF_BC_DIRICHLET); break;
    }
#undef GMRF_L3V
#undef GMRF_L3
    return cudaGetLastError();
  }
  a.nzc = 1;
  if (stencil2d_strip_eligible(g, sizeof(T) == 8) &&
      (STEP || stencil2d_strip_pointers_ok(a.Win, a.Wout, a.kappa2)))
    return launch_stencil2d_strip<T>(g, a, nvec, STEP, s);
#define GMRF_L2(OPV, BCV) k_stencil2d<T, OPV, BCV, STEP><<<grd, blk, 0, s>>>(a)
  if (g.op == GMRF_OP_SPDE_SQUARED) {
    switch (g.bc) {
      case GMRF_BC_PERIODIC: GMRF_L2(GMRF_OP_SPDE_SQUARED, GMRF_BC_PERIODIC); break;
      case GMRF_BC_NEUMANN: GMRF_L2(GMRF_OP_SPDE_SQUARED, GMRF_BC_NEUMANN); break;
      default: GMRF_L2(GMRF_OP_SPDE_SQUARED, GMRF_BC_DIRICHLET); break;
    }
  } else if (g.op == GMRF_OP_SPDE_PLUS_DIAG) {
    switch (g.bc) {
      case GMRF_BC_PERIODIC: GMRF_L2(GMRF_OP_SPDE_PLUS_DIAG, GMRF_BC_PERIODIC); break;
      case GMRF_BC_NEUMANN: GMRF_L2(GMRF_OP_SPDE_PLUS_DIAG, GMRF_BC_NEUMANN); break;
      default: GMRF_L2(GMRF_OP_SPDE_PLUS_DIAG, GMRF_BC_DIRICHLET); break;
    }
  } else {
    switch (g.bc) {
      case GMRF_BC_PERIODIC: GMRF_L2(GMRF_OP_SHIFTED_LAPLACIAN, GMRF_BC_PERIODIC); break;
      case GMRF_BC_NEUMANN: GMRF_L2(GMRF_OP_SHIFTED_LAPLACIAN, GMRF_BC_NEUMANN); break;
      default: GMRF_L2(GMRF_OP_SHIFTED_LAPLACIAN, GMRF_BC_DIRICHLET); break;
    }
  }
#undef GMRF_L2
  return cudaGetLastError();
}

template <typename T>
StencilArgs<T> make_args(const Grid& g, const void* kappa2, double kc) {
  StencilArgs<T> a{};
  a.kappa2 = (const float*)kappa2;
  a.kappa2_const = (T)kc;
  a.nx = g.nx;
  a.ny = g.ny;
  a.nz = g.dim == 3 ? g.nz : 1;
  a.n = g.n;
  return a;
}

}  // namespace

int stencil_blocks_per_vector(const Grid& g) {
  if (g.dim == 3) {
    // the widest tile (VX = 1) has the most blocks; the TMA kernel's items
    const int r = ((g.nx + TX - 1) / TX) * ((g.ny + TY3 - 1) / TY3) * nz_chunks(g, 1);
    const int t = stencil3d_tma_eligible(g, false) ? stencil3d_tma_items_per_vector(g) : 0;
    return r > t ? r : t;
  }
  int r = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
  for (int fp64 = 0; fp64 < 2; ++fp64)
    if (stencil2d_strip_eligible(g, fp64 != 0)) r = std::max(r, stencil2d_strip_blocks_per_vector(g, fp64 != 0));
  return r;
}

cudaError_t launch_stencil_step(const Grid& g, bool fp64, const void* kappa2, double kappa2_const,
                                const LanczosBufs& b, const StepParams& P, cudaStream_t s) {
  if (fp64) {
    auto a = make_args<double>(g, kappa2, kappa2_const);
    a.W0 = (double*)b.W[0];
    a.W1 = (double*)b.W[1];
    a.V = (double*)b.V;
    a.P = P;
    a.st = b.st; a.alpha = b.alpha; a.beta = b.beta; a.alpha_f = b.alpha_f; a.beta2_f = b.beta2_f;
    a.partials = (Dots<double>*)b.partials;
    a.counters = b.counters;
    return dispatch<double, true>(g, a, b.nvec, s);
  }
  auto a = make_args<float>(g, kappa2, kappa2_const);
  a.W0 = (float*)b.W[0];
  a.W1 = (float*)b.W[1];
  a.V = (float*)b.V;
  a.P = P;
  a.st = b.st; a.alpha = b.alpha; a.beta = b.beta; a.alpha_f = b.alpha_f; a.beta2_f = b.beta2_f;
  a.partials = (Dots<float>*)b.partials;
  a.counters = b.counters;
  return dispatch<float, true>(g, a, b.nvec, s);
}

cudaError_t launch_stencil_apply(const Grid& g, bool fp64, const void* kappa2, double kappa2_const,
                                 const void* v, void* y, int nvec, cudaStream_t s) {
  if (fp64) {
    auto a = make_args<double>(g, kappa2, kappa2_const);
    a.Win = (const double*)v;
    a.Wout = (double*)y;
    return dispatch<double, false>(g, a, nvec, s);
  }
  auto a = make_args<float>(g, kappa2, kappa2_const);
  a.Win = (const float*)v;
  a.Wout = (float*)y;
  return dispatch<float, false>(g, a, nvec, s);
}

}  // namespace gmrf
