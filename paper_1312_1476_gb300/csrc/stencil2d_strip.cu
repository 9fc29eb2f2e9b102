// stencil2d_strip.cu -- the fused 2-D Lanczos step of Algorithm 1 with the
// matrix-free lattice apply of Q (Section 2), streamed down strips of rows.
//
// A block owns one strip of BX = 32 VX columns (VX = 16 bytes / element: 4
// floats or 2 doubles per lane) and a chunk of rows of one vector, and marches
// down the rows in slabs of 8 (one row per warp).  Every input row of the
// strip (q_{j-1}, v_{j-1}, kappa^2) is read once, by 16-byte asynchronous
// copies (cp.async) issued two slabs ahead into rolling shared-memory rings
// of 32 rows with a 16-byte x halo on either side; v_j is formed in place of
// q_{j-1} once a slab's copies have landed.  The squared operators keep a ring of
// g = B v as well:
//   shifted   q = B v                  (5-point, needs v rows y-1 .. y+1)
//   squared   q = B g,  g = B v        (13-point, v rows y-2 .. y+2)
//   plus_diag q = B g + D v,  B = kappa_c^2 I + L
// with B v = kappa^2 v + sum over existing edges (v_i - v_nb) as in the
// tile kernel (Neumann edges leaving the grid are absent, Dirichlet
// neighbours are 0, periodic ones wrap).  Rows are loaded H rows ahead of the
// rows whose q is formed (H = 1 shifted, 2 squared); a slab's new rows only
// overwrite ring slots of rows no longer read.  One record of partial dot
// products per block; the row chunk depends on the grid only, so the sums of
// a vector do not depend on the rest of its batch.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "internal.h"
#include "stencil_args.h"

namespace gmrf {
namespace {

// ring rows: a slab reads rows y0 - 2 .. y0 + 9 while the copies of the next
// two slabs (rows up to y0 + 25) are in flight: a span of 28 rows, so copies
// issued during a slab never land in a slot that is read
constexpr int SR = 32;
constexpr int DEPTH = 2;     // slabs copied ahead
constexpr int SNT = 256;     // threads: 8 warps, one row each per slab

template <typename T>
__host__ __device__ constexpr int strip_vx() { return 16 / (int)sizeof(T); }
template <typename T>
__host__ __device__ constexpr int strip_bx() { return 32 * strip_vx<T>(); }

__device__ __forceinline__ int ring(int y) { return (y + SR) & (SR - 1); }  // y >= -2

template <typename T, int VX>
__device__ __forceinline__ void ld16(const T* p, T (&o)[VX]) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
}
template <typename T, int VX>
__device__ __forceinline__ void st16(T* p, const T (&o)[VX]) {
  if constexpr (sizeof(T) == 4) *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  else *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
}
// VX floats of kappa^2 (16 bytes for FP32, 8 for FP64)
// asynchronous global -> shared copies; valid = false fills zeros and reads nothing
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? BYTES : 0;
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// VX floats of a shared-memory ring row (16-byte aligned for FP32, 8 for FP64)
template <int VX>
__device__ __forceinline__ void ldk_s(const float* p, float (&o)[VX]) {
  if constexpr (VX == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else {
    const float2 v = *reinterpret_cast<const float2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
}

template <typename T, int OP, int BC, bool STEP>
__global__ void __launch_bounds__(SNT) k_stencil2d_strip(StencilArgs<T> a, int ychunk) {
  constexpr int VX = strip_vx<T>(), BX = strip_bx<T>(), PW = BX + 2 * VX;
  constexpr bool SQ = OP != GMRF_OP_SHIFTED_LAPLACIAN;
  constexpr int H = SQ ? 2 : 1;
  // dynamic shared memory (strip_smem_bytes): vr | gr (squared) | vpr (step) | kr;
  // vr holds q_{j-1} as copied, then v_j; vpr v_{j-1} with the halo columns
  extern __shared__ __align__(16) unsigned char smraw[];
  T* vr = reinterpret_cast<T*>(smraw);
  T* gr = vr + SR * PW;
  T* vpr = gr + (SQ ? SR * PW : 0);
  float* kr = reinterpret_cast<float*>(vpr + (STEP ? SR * PW : 0));
  __shared__ Dots<T> red[SNT / 32];
  __shared__ int s_int[4];
  __shared__ float s_flt[4];

  const int s = blockIdx.z;
  int j = 0;
  if (STEP) {
    if (a.st[s].status != VS_RUNNING) return;
    j = a.st[s].m;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nx = a.nx, ny = a.ny;
  const int x0 = blockIdx.x * BX;
  const int ya = blockIdx.y * ychunk;
  const int yb = min(ny, ya + ychunk);
  const size_t n = a.n;
  const T* Win = (STEP ? ((j & 1) ? a.W1 : a.W0) : a.Win) + (size_t)s * n;
  T* Wout = (STEP ? ((j & 1) ? a.W0 : a.W1) : a.Wout) + (size_t)s * n;
  const T* Vp = nullptr;
  T* Vc = nullptr;
  T coef = 0, inv_b = 1, bprev = 0;
  if (STEP) {
    const size_t base = (size_t)s * a.P.nslots;
    Vc = a.V + (base + (size_t)(j % a.P.nslots)) * n;
    inv_b = (T)a.st[s].vscale;
    if (j > 0) {
      Vp = a.V + (base + (size_t)((j - 1) % a.P.nslots)) * n;
      const size_t mo = (size_t)s * a.P.m_max + (j - 1);
      coef = (T)a.alpha[mo];
      bprev = (T)a.beta[mo];
    }
  }
  const bool kfield = a.kappa2 != nullptr;
  const T kc = a.kappa2_const;

  // Row y of the strip (any y >= -2; outside the grid: wrapped or zero):
  // copy_row() issues the lane's asynchronous copies (its interior vector;
  // lanes 0 / 1 also the left / right halo vector), form_row() turns the
  // landed q_{j-1} into v_j in place.
  auto copy_row = [&](int y) {
    int gy = y;
    bool rin = gy >= 0 && gy < ny;
    if (!rin && BC == GMRF_BC_PERIODIC) {
      gy = gy < 0 ? gy + ny : gy - ny;
      rin = true;
    }
    const size_t row0 = (size_t)(rin ? gy : 0) * nx;
    const int sl = ring(y);
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      if (part == 1 && lane >= 2) continue;
      int xx = part == 0 ? x0 + VX * lane : (lane == 0 ? x0 - VX : x0 + BX);
      const int col = part == 0 ? VX + VX * lane : (lane == 0 ? 0 : VX + BX);
      bool in = rin && xx >= 0 && xx < nx;
      if (rin && !in && BC == GMRF_BC_PERIODIC) {
        xx = xx < 0 ? xx + nx : xx - nx;
        in = true;
      }
      const size_t i = row0 + (in ? xx : 0);
      cp_async<16>(vr + sl * PW + col, Win + i, in);
      if (STEP && j > 0) cp_async<16>(vpr + sl * PW + col, Vp + i, in);
      if (kfield) cp_async<4 * VX>(kr + sl * PW + col, a.kappa2 + i, in);
    }
  };
  auto form_row = [&](int y) {
    if (!STEP) return;
    const int sl = ring(y);
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      if (part == 1 && lane >= 2) continue;
      const int col = part == 0 ? VX + VX * lane : (lane == 0 ? 0 : VX + BX);
      // the same expression for interior and halo cells: a halo cell is another
      // strip's interior cell and must get the same v_j bitwise
      T v[VX];
      ld16<T, VX>(vr + sl * PW + col, v);
      if (j > 0) {
        T vp[VX];
        ld16<T, VX>(vpr + sl * PW + col, vp);
#pragma unroll
        for (int e = 0; e < VX; ++e) v[e] = (v[e] - coef * vp[e]) * inv_b;
      } else {
#pragma unroll
        for (int e = 0; e < VX; ++e) v[e] = v[e] * inv_b;
      }
      st16<T, VX>(vr + sl * PW + col, v);
    }
  };
  // B applied at ring column c of row y (global column xg), reading array src
  auto bop = [&](const T* src, int y, int c, int xg, T kap) -> T {
    const int sl = ring(y);
    const T c0 = src[sl * PW + c];
    T r = kap * c0;
    if (BC != GMRF_BC_NEUMANN || xg > 0) r += c0 - src[sl * PW + c - 1];
    if (BC != GMRF_BC_NEUMANN || xg < nx - 1) r += c0 - src[sl * PW + c + 1];
    if (BC != GMRF_BC_NEUMANN || y > 0) r += c0 - src[ring(y - 1) * PW + c];
    if (BC != GMRF_BC_NEUMANN || y < ny - 1) r += c0 - src[ring(y + 1) * PW + c];
    return r;
  };
  // B on the lane's VX interior cells of row y from array src: 16-byte row
  // loads (centre, up, down), x neighbours by shuffle (the strip edges from
  // the halo columns); the same order of terms as bop.  A Neumann edge that
  // leaves the grid takes the centre value as its neighbour, so its term
  // (c - c) is exactly 0: the same sum as leaving the edge out, without a
  // test per cell.
  const bool nl = BC == GMRF_BC_NEUMANN && x0 + VX * lane == 0;
  const bool nr = BC == GMRF_BC_NEUMANN && x0 + VX * lane + VX == nx;
  auto bop_vec = [&](const T* src, int y, const T (&kap)[VX], T (&r)[VX]) {
    const int sl = ring(y), c0 = VX + VX * lane;
    T cc[VX], up[VX], dn[VX];
    ld16<T, VX>(src + sl * PW + c0, cc);
    ld16<T, VX>(src + ring(y - 1) * PW + c0, up);
    ld16<T, VX>(src + ring(y + 1) * PW + c0, dn);
    T lft = __shfl_up_sync(0xffffffffu, cc[VX - 1], 1);
    T rgt = __shfl_down_sync(0xffffffffu, cc[0], 1);
    if (lane == 0) lft = src[sl * PW + c0 - 1];
    if (lane == 31) rgt = src[sl * PW + c0 + VX];
    if (nl) lft = cc[0];
    if (nr) rgt = cc[VX - 1];
    if (BC == GMRF_BC_NEUMANN && y == 0) {
#pragma unroll
      for (int e = 0; e < VX; ++e) up[e] = cc[e];
    }
    if (BC == GMRF_BC_NEUMANN && y == ny - 1) {
#pragma unroll
      for (int e = 0; e < VX; ++e) dn[e] = cc[e];
    }
    if constexpr (sizeof(T) == 4) {
      // pairs of cells on paired FP32 instructions (kappa^2 c fused with the first difference)
#pragma unroll
      for (int e = 0; e < VX; e += 2) {
        const float2 c = make_float2(cc[e], cc[e + 1]);
        const float2 l = make_float2(e == 0 ? lft : cc[e - 1 < 0 ? 0 : e - 1], cc[e]);
        const float2 rr = make_float2(cc[e + 1], e + 1 == VX - 1 ? rgt : cc[e + 2 < VX ? e + 2 : VX - 1]);
        float2 t = x2_fma(make_float2(kap[e], kap[e + 1]), c, x2_sub(c, l));
        t = x2_add(t, x2_sub(c, rr));
        t = x2_add(t, x2_sub(c, make_float2(up[e], up[e + 1])));
        t = x2_add(t, x2_sub(c, make_float2(dn[e], dn[e + 1])));
        r[e] = t.x;
        r[e + 1] = t.y;
      }
    } else {
#pragma unroll
      for (int e = 0; e < VX; ++e) {
        const T l = e == 0 ? lft : cc[e - 1 < 0 ? 0 : e - 1];
        const T rr = e == VX - 1 ? rgt : cc[e + 1 < VX ? e + 1 : VX - 1];
        T t = kap[e] * cc[e];
        t += cc[e] - l;
        t += cc[e] - rr;
        t += cc[e] - up[e];
        t += cc[e] - dn[e];
        r[e] = t;
      }
    }
  };
  auto kap_vec = [&](int y, T (&kap)[VX]) {
    if (OP == GMRF_OP_SPDE_PLUS_DIAG || !kfield) {
#pragma unroll
      for (int e = 0; e < VX; ++e) kap[e] = kc;
    } else {
      float k[VX];
      ldk_s<VX>(kr + ring(y) * PW + VX + VX * lane, k);
#pragma unroll
      for (int e = 0; e < VX; ++e) kap[e] = (T)k[e];
    }
  };
  // g = B v on row y: the lane's VX cells, plus x0 - 1 (lane 0) and x0 + BX (lane 31)
  auto g_row = [&](int y) {
    const bool rin = (y >= 0 && y < ny) || BC == GMRF_BC_PERIODIC;
    const int sl = ring(y);
    T kap[VX], gv[VX];
    kap_vec(y, kap);
    bop_vec(vr, y, kap, gv);  // every warp lane takes part (shuffles)
    if (!rin) {
#pragma unroll
      for (int e = 0; e < VX; ++e) gv[e] = 0;
    }
    st16<T, VX>(gr + sl * PW + VX + VX * lane, gv);
    if (lane == 0 || lane == 31) {
      const int c = lane == 0 ? VX - 1 : VX + BX;
      const int xg = x0 - VX + c;
      const bool in = rin && ((xg >= 0 && xg < nx) || BC == GMRF_BC_PERIODIC);
      T g1 = 0;
      if (in) {
        const T k1 = (OP == GMRF_OP_SPDE_PLUS_DIAG || !kfield) ? kc : (T)kr[sl * PW + c];
        g1 = bop(vr, y, c, xg, k1);
      }
      gr[sl * PW + c] = g1;
    }
  };
  Dots<T> d;
  d.zero();
  Dot2x2 dd;  // FP32: the sums over pairs of cells on paired instructions
  dd.zero();
  // q on row y (< yb): the lane's VX cells; stores and dot products
  auto q_row = [&](int y) {
    const int sl = ring(y);
    const int c0 = VX + VX * lane;
    T q[VX], v[VX], kap[VX];
    kap_vec(y, kap);
    bop_vec(SQ ? gr : vr, y, kap, q);
    ld16<T, VX>(vr + sl * PW + c0, v);
    if (OP == GMRF_OP_SPDE_PLUS_DIAG && kfield) {
      float dk[VX];
      ldk_s<VX>(kr + sl * PW + c0, dk);
#pragma unroll
      for (int e = 0; e < VX; ++e) q[e] += (T)dk[e] * v[e];
    }
    if (STEP && j > 0) {
      T vp[VX];
      ld16<T, VX>(vpr + sl * PW + c0, vp);
#pragma unroll
      for (int e = 0; e < VX; ++e) q[e] -= bprev * vp[e];
    }
    const size_t i = (size_t)y * nx + x0 + VX * lane;
    st16<T, VX>(Wout + i, q);
    if (STEP) {
      st16<T, VX>(Vc + i, v);
      if (a.P.vb) {
        __nv_bfloat16* pb = vb_at(a.P, s, j, n, i);
        if (VX == 4) vb_store4(pb, (float)v[0], (float)v[1 % VX], (float)v[2 % VX], (float)v[3 % VX]);
        else vb_store2(pb, (float)v[0], (float)v[1 % VX]);
      }
      if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int e = 0; e < VX; e += 2) dd.add(make_float2(v[e], v[e + 1]), make_float2(q[e], q[e + 1]));
      } else {
#pragma unroll
        for (int e = 0; e < VX; ++e) d.add(v[e], q[e]);
      }
    }
  };

  // prologue: the rows above the chunk's first slab, then DEPTH slabs of copies
  if (w < 2 * H) copy_row(ya - H + w);
#pragma unroll
  for (int k = 0; k < DEPTH; ++k) {
    const int y = ya + 8 * k + H + w;
    if (y < yb + H) copy_row(y);
    cp_async_commit();
  }
  for (int y0 = ya; y0 < yb; y0 += 8) {
    cp_async_wait<DEPTH - 1>();  // this thread's copies of slab y0 have landed
    __syncthreads();
    if (y0 == ya && w < 2 * H) form_row(ya - H + w);
    if (y0 + H + w < yb + H) form_row(y0 + H + w);
    __syncthreads();
    {
      const int y = y0 + 8 * DEPTH + H + w;  // the slab DEPTH ahead, into slots no slab in flight reads
      if (y < yb + H) copy_row(y);
      cp_async_commit();
    }
    if (SQ) {
      const int g0 = y0 == ya ? ya - 1 : y0 + 1;
      const int g1 = min(y0 + 8, yb);
      for (int y = g0 + w; y <= g1; y += 8) g_row(y);
      __syncthreads();
    }
    {
      const int y = y0 + w;
      if (y < yb) q_row(y);
    }
  }
  cp_async_wait<0>();
  if (!STEP) return;
  if constexpr (sizeof(T) == 4) d = dd.merged();
  d = block_reduce(d, red);
  const int nblk = gridDim.x * gridDim.y;
  if (threadIdx.x == 0) a.partials[(size_t)s * nblk + blockIdx.x + gridDim.x * blockIdx.y] = d;
  if (last_block(a.counters, s, nblk, &s_int[3]))
    finish_step<T>(a.P, j, s, a.partials, nblk, a.st, a.alpha, a.beta, a.alpha_f, a.beta2_f, red, s_int, s_flt);
}

template <typename T, int OP, bool STEP>
constexpr size_t strip_smem_bytes() {
  constexpr int VX = strip_vx<T>(), BX = strip_bx<T>(), PW = BX + 2 * VX;
  return (size_t)SR * PW * sizeof(T) * (OP != GMRF_OP_SHIFTED_LAPLACIAN ? 2 : 1) +
         (STEP ? (size_t)SR * PW * sizeof(T) : 0) + (size_t)SR * PW * sizeof(float);
}

template <typename T>
int strip_ychunk(const Grid& g) {
  return g.ny >= 1024 ? 64 : 32;
}

template <typename T, int OP, int BC, bool STEP>
cudaError_t launch_bc(dim3 grd, const StencilArgs<T>& a, int yc, cudaStream_t s) {
  constexpr size_t sm = strip_smem_bytes<T, OP, STEP>();
  static std::atomic<bool> attr{false};  // several host threads may launch at once
  if (!attr.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(k_stencil2d_strip<T, OP, BC, STEP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr.store(true, std::memory_order_release);
  }
  k_stencil2d_strip<T, OP, BC, STEP><<<grd, SNT, sm, s>>>(a, yc);
  return cudaGetLastError();
}

template <typename T, bool STEP, int OP>
cudaError_t launch_op(const Grid& g, const StencilArgs<T>& a, int nvec, cudaStream_t s) {
  const int yc = strip_ychunk<T>(g);
  dim3 grd(g.nx / strip_bx<T>(), (g.ny + yc - 1) / yc, nvec);
  switch (g.bc) {
    case GMRF_BC_PERIODIC: return launch_bc<T, OP, GMRF_BC_PERIODIC, STEP>(grd, a, yc, s);
    case GMRF_BC_NEUMANN: return launch_bc<T, OP, GMRF_BC_NEUMANN, STEP>(grd, a, yc, s);
    default: return launch_bc<T, OP, GMRF_BC_DIRICHLET, STEP>(grd, a, yc, s);
  }
}

}  // namespace

bool stencil2d_strip_eligible(const Grid& g, bool fp64) {
  const int bx = fp64 ? strip_bx<double>() : strip_bx<float>();
  return g.dim == 2 && g.nx % bx == 0 && g.ny >= 4 && (int64_t)g.nx * g.ny >= 65536;
}

int stencil2d_strip_blocks_per_vector(const Grid& g, bool fp64) {
  const int bx = fp64 ? strip_bx<double>() : strip_bx<float>();
  const int yc = fp64 ? strip_ychunk<double>(g) : strip_ychunk<float>(g);
  return (g.nx / bx) * ((g.ny + yc - 1) / yc);
}

bool stencil2d_strip_pointers_ok(const void* win, const void* wout, const float* kappa2) {
  auto al = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
  return al(win) && al(wout) && al(kappa2);
}

template <typename T>
cudaError_t launch_stencil2d_strip(const Grid& g, const StencilArgs<T>& a, int nvec, bool step, cudaStream_t s) {
  if (g.op == GMRF_OP_SPDE_SQUARED)
    return step ? launch_op<T, true, GMRF_OP_SPDE_SQUARED>(g, a, nvec, s)
                : launch_op<T, false, GMRF_OP_SPDE_SQUARED>(g, a, nvec, s);
  if (g.op == GMRF_OP_SPDE_PLUS_DIAG)
    return step ? launch_op<T, true, GMRF_OP_SPDE_PLUS_DIAG>(g, a, nvec, s)
                : launch_op<T, false, GMRF_OP_SPDE_PLUS_DIAG>(g, a, nvec, s);
  return step ? launch_op<T, true, GMRF_OP_SHIFTED_LAPLACIAN>(g, a, nvec, s)
              : launch_op<T, false, GMRF_OP_SHIFTED_LAPLACIAN>(g, a, nvec, s);
}

template cudaError_t launch_stencil2d_strip<float>(const Grid&, const StencilArgs<float>&, int, bool, cudaStream_t);
template cudaError_t launch_stencil2d_strip<double>(const Grid&, const StencilArgs<double>&, int, bool, cudaStream_t);

}  // namespace gmrf
