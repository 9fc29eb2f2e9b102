// stencil3d_tma.cu -- the fused Lanczos step of Algorithm 1 with the 3-D
// 7-point lattice apply of Q (Section 2), staged through shared memory by the
// Tensor Memory Accelerator.
//
// Work unit ("item"): one 128 x 8 tile in x-y of one vector, marched over a
// chunk of z planes.  A persistent grid (resident blocks only) walks the items
// in order, so neighbouring tiles run side by side and share their halo rows
// in L2.  For each plane the producer thread issues three tiled bulk loads
// into a 4-deep ring of shared-memory stages, completing on one transaction
// barrier per stage:
//   q_{j-1} (W) and v_{j-1} (V ring) over the tile plus a halo of 1 row in y
//   and 4 columns in x (the x start is rounded to 16 bytes), and kappa^2 over
//   the tile.  Cells outside the grid arrive as zeros, which are the Dirichlet
//   values; zero-Neumann edges leaving the grid are skipped.
// Each thread owns 4 adjacent cells along x.  v_j = (q_{j-1} - alpha v_{j-1})
// / beta is formed from the staged values where it is read (own cells from
// the next plane, x neighbours by warp shuffles, y neighbours from the halo
// rows), q_j = Q v_j - beta_{j-1} v_{j-1} and v_j go to global memory with
// 16-byte stores, and the dot products v.q, q.q, v.v are accumulated per item
// (compensated FP32) for the step's alpha_j, beta_j (common.cuh).
//
// The partial sums of an item depend only on the grid, so a vector's result
// is the same in any batch.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"
#include "stencil_args.h"
#include "tma.cuh"

namespace gmrf {
namespace tma {

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}
}  // namespace

bool encode_f32(CUtensorMap* map, const void* base, int rank, const uint64_t* dims, const uint64_t* strides_bytes,
                const uint32_t* box) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || rank < 1 || rank > 5) return false;
  cuuint64_t d[5], st[4];
  cuuint32_t b[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    es[i] = 1;
    if (i + 1 < rank) st[i] = strides_bytes[i];
  }
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void*>(base), d, st, b, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tma

namespace {

constexpr int BX = 128;                // tile width (cells): 32 lanes x 4
constexpr int BY = 8;                  // tile height: one warp per row
constexpr int NT = 32 * BY;            // threads per block
constexpr int HX = 4;                  // x halo, rounded up to 16 bytes
constexpr int TWX = BX + 2 * HX;       // staged columns
constexpr int TWY = BY + 2;            // staged rows
constexpr int kStages = 4;             // planes resident or in flight per block
constexpr int kMinBlocks = 3;          // resident blocks per SM the kernel is built for
constexpr uint32_t kHaloBytes = TWX * TWY * 4;
constexpr uint32_t kKapBytes = BX * BY * 4;
constexpr uint32_t kHaloPitch = (kHaloBytes + 127) / 128 * 128;
constexpr uint32_t kStageBytes = 2 * kHaloPitch + kKapBytes;
constexpr size_t kSmemBytes = (size_t)kStages * kStageBytes;
static_assert(kStageBytes % 128 == 0, "stage alignment");

struct Maps {
  CUtensorMap w0;  // step: q ping-pong buffer 0 (apply: v), dims (nx, ny, nz, nvec), box (TWX, TWY, 1, 1)
  CUtensorMap w1;  // step: q ping-pong buffer 1
  CUtensorMap v;   // step: basis ring, dims (nx, ny, nz, nvec * nslots), box (TWX, TWY, 1, 1)
  CUtensorMap k;   // kappa^2, dims (nx, ny, nz), box (BX, BY, 1)
};

struct Items {
  int ntx, nty, nzc, zper, per_vec, total;
};

template <int BC, bool STEP>
__global__ void __launch_bounds__(NT, kMinBlocks)
    k_stencil3d_tma(StencilArgs<float> a, const __grid_constant__ Maps maps, Items it) {
  extern __shared__ __align__(128) unsigned char sbuf[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ Dots<float> red[NT / 32];
  __shared__ int s_int[4];
  __shared__ float s_flt[4];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
  if (tid == 0) {
#pragma unroll
    for (int b = 0; b < kStages; ++b) tma::mbar_init(&full[b], 1);
    tma::fence_barrier_init();
  }
  __syncthreads();
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t n = a.n, plane = (size_t)nx * ny;
  uint32_t ph = 0;       // parity of the next completion of each stage barrier
  uint32_t pending = 0;  // thread 0: stages with a load issued and not yet waited
  bool bad = false;      // this thread saw a wait run out

  for (int item = blockIdx.x; item < it.total; item += gridDim.x) {
    const int s = item / it.per_vec;
    const int li = item - s * it.per_vec;
    const int bx = li % it.ntx;
    const int by = (li / it.ntx) % it.nty;
    const int zc = li / (it.ntx * it.nty);
    int j = 0;
    __syncthreads();  // the previous item's stages and scratch are free
    if (STEP) {
      // a vector's state changes only after all of its items of this launch
      // are done, so every thread reads the same value
      if (a.st[s].status != VS_RUNNING) continue;
      j = a.st[s].m;
    }
    const int x0 = bx * BX, y0 = by * BY;
    const int z0 = zc * it.zper, z1 = min(nz, z0 + it.zper);
    const int P = z0 < z1 ? z1 - z0 + 2 : 0;  // planes z0 - 1 .. z1
    const CUtensorMap* wmap = (STEP && (j & 1)) ? &maps.w1 : &maps.w0;
    float* Wout = (STEP ? ((j & 1) ? a.W0 : a.W1) : a.Wout) + (size_t)s * n;
    float* Vc = nullptr;
    const bool use_vp = STEP && j > 0;
    int vrow = 0;
    float coef = 0.f, inv_b = 1.f, bprev = 0.f;
    if (STEP) {
      const size_t base = (size_t)s * a.P.nslots;
      Vc = a.V + (base + (size_t)(j % a.P.nslots)) * n;
      if (j == 0) {
        inv_b = (float)a.st[s].vscale;
      } else {
        vrow = (int)(base + (size_t)((j - 1) % a.P.nslots));
        const size_t mo = (size_t)s * a.P.m_max + (j - 1);
        coef = (float)a.alpha[mo];
        bprev = (float)a.beta[mo];
        inv_b = (float)a.st[s].vscale;
      }
    }
    // v_j from the staged q_{j-1} and v_{j-1}
    auto fv = [&](float w, float vp) -> float {
      if (!STEP) return w;
      if (j == 0) return w * inv_b;
      return __fmul_rn(__fmaf_rn(-coef, vp, w), inv_b);
    };
    auto issue = [&](int t) {  // thread 0: plane z0 - 1 + t into stage t % kStages
      const int b = t % kStages;
      unsigned char* sp = sbuf + (size_t)b * kStageBytes;
      const int z = z0 - 1 + t;
      const bool kap = a.kappa2 != nullptr && t > 0 && t < P - 1;
      const uint32_t bytes = kHaloBytes + (use_vp ? kHaloBytes : 0u) + (kap ? kKapBytes : 0u);
      tma::fence_proxy_async_smem();
      tma::mbar_arrive_expect_tx(&full[b], bytes);
      tma::load_4d(sp, wmap, &full[b], x0 - HX, y0 - 1, z, s);
      if (use_vp) tma::load_4d(sp + kHaloPitch, &maps.v, &full[b], x0 - HX, y0 - 1, z, vrow);
      if (kap) tma::load_3d(sp + 2 * kHaloPitch, &maps.k, &full[b], x0, y0, z);
      pending |= 1u << b;
    };
    auto wait_plane = [&](int t) -> const float* {
      const int b = t % kStages;
      if (!tma::mbar_wait(&full[b], (ph >> b) & 1u)) bad = true;
      ph ^= 1u << b;
      pending &= ~(1u << b);
      return reinterpret_cast<const float*>(sbuf + (size_t)b * kStageBytes);
    };
    const int gx = x0 + 4 * tx, gy = y0 + ty;
    const bool own = gx < nx && gy < ny;
    const int oc = (ty + 1) * TWX + HX + 4 * tx;  // first own cell in a staged halo tile
    constexpr int VOFF = kHaloPitch / 4;          // v_{j-1} tile offset (floats)
    constexpr int KOFF = 2 * kHaloPitch / 4;      // kappa^2 tile offset (floats)
    // v_j and v_{j-1} at the own cells of a staged plane
    auto own4 = [&](const float* sp, float* v, float* vp) {
      const float4 w4 = *reinterpret_cast<const float4*>(sp + oc);
      float4 p4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (use_vp) p4 = *reinterpret_cast<const float4*>(sp + VOFF + oc);
      vp[0] = p4.x; vp[1] = p4.y; vp[2] = p4.z; vp[3] = p4.w;
      v[0] = fv(w4.x, p4.x); v[1] = fv(w4.y, p4.y); v[2] = fv(w4.z, p4.z); v[3] = fv(w4.w, p4.w);
    };
    auto row4 = [&](const float* sp, int off, float* v) {
      const float4 w4 = *reinterpret_cast<const float4*>(sp + off);
      float4 p4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (use_vp) p4 = *reinterpret_cast<const float4*>(sp + VOFF + off);
      v[0] = fv(w4.x, p4.x); v[1] = fv(w4.y, p4.y); v[2] = fv(w4.z, p4.z); v[3] = fv(w4.w, p4.w);
    };
    auto cell = [&](const float* sp, int off) -> float { return fv(sp[off], use_vp ? sp[VOFF + off] : 0.f); };

    Dot2x2 dd;
    dd.zero();
    bool abort = false;
    if (P > 0) {
      if (tid == 0)
        for (int t = 0; t < kStages && t < P; ++t) issue(t);
      float vdn[4], vc[4], vup[4], vpc[4], vpu[4];
      own4(wait_plane(0), vdn, vpu);
      own4(wait_plane(1), vc, vpc);
      abort = __syncthreads_or(bad);
      if (!abort && tid == 0 && kStages < P) issue(kStages);
      for (int t = 1; t <= P - 2 && !abort; ++t) {
        own4(wait_plane(t + 1), vup, vpu);
        const float* sc = reinterpret_cast<const float*>(sbuf + (size_t)(t % kStages) * kStageBytes);
        const int z = z0 - 1 + t;
        float vl = __shfl_up_sync(0xffffffffu, vc[3], 1);
        float vr = __shfl_down_sync(0xffffffffu, vc[0], 1);
        if (tx == 0) vl = cell(sc, oc - 1);
        if (tx == 31) vr = cell(sc, oc + 4);
        float vs[4], vn[4];
        row4(sc, oc - TWX, vs);
        row4(sc, oc + TWX, vn);
        float kk[4];
        if (a.kappa2) {
          const float4 k4 = *reinterpret_cast<const float4*>(sc + KOFF + ty * BX + 4 * tx);
          kk[0] = k4.x; kk[1] = k4.y; kk[2] = k4.z; kk[3] = k4.w;
        } else {
          kk[0] = kk[1] = kk[2] = kk[3] = a.kappa2_const;
        }
        if (own && BC != GMRF_BC_NEUMANN) {
          // every edge exists: pairs of cells on paired FP32 instructions
          float qo[4];
#pragma unroll
          for (int e = 0; e < 4; e += 2) {
            const float2 c = make_float2(vc[e], vc[e + 1]);
            const float2 l = make_float2(e == 0 ? vl : vc[e - 1 < 0 ? 0 : e - 1], vc[e]);
            const float2 rr = make_float2(vc[e + 1], e == 2 ? vr : vc[e + 2 < 4 ? e + 2 : 3]);
            float2 t = x2_fma(make_float2(kk[e], kk[e + 1]), c, x2_sub(c, l));
            t = x2_add(t, x2_sub(c, rr));
            t = x2_add(t, x2_sub(c, make_float2(vs[e], vs[e + 1])));
            t = x2_add(t, x2_sub(c, make_float2(vn[e], vn[e + 1])));
            t = x2_add(t, x2_sub(c, make_float2(vdn[e], vdn[e + 1])));
            t = x2_add(t, x2_sub(c, make_float2(vup[e], vup[e + 1])));
            if (STEP && j > 0) t = x2_fma(make_float2(-bprev, -bprev), make_float2(vpc[e], vpc[e + 1]), t);
            qo[e] = t.x;
            qo[e + 1] = t.y;
          }
          if (STEP) {
            dd.add(make_float2(vc[0], vc[1]), make_float2(qo[0], qo[1]));
            dd.add(make_float2(vc[2], vc[3]), make_float2(qo[2], qo[3]));
          }
          const size_t i = (size_t)gx + (size_t)nx * gy + plane * z;
          *reinterpret_cast<float4*>(Wout + i) = make_float4(qo[0], qo[1], qo[2], qo[3]);
          if (STEP) {
            *reinterpret_cast<float4*>(Vc + i) = make_float4(vc[0], vc[1], vc[2], vc[3]);
            if (a.P.vb) vb_store4(vb_at(a.P, s, j, n, i), vc[0], vc[1], vc[2], vc[3]);
          }
        } else if (own) {
          float qo[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float c = vc[e];
            const float left = e == 0 ? vl : vc[e - 1];
            const float right = e == 3 ? vr : vc[e + 1];
            float r = kk[e] * c;
            if (BC != GMRF_BC_NEUMANN || gx + e > 0) r += c - left;
            if (BC != GMRF_BC_NEUMANN || gx + e < nx - 1) r += c - right;
            if (BC != GMRF_BC_NEUMANN || gy > 0) r += c - vs[e];
            if (BC != GMRF_BC_NEUMANN || gy < ny - 1) r += c - vn[e];
            if (BC != GMRF_BC_NEUMANN || z > 0) r += c - vdn[e];
            if (BC != GMRF_BC_NEUMANN || z < nz - 1) r += c - vup[e];
            if (STEP && j > 0) r -= bprev * vpc[e];
            qo[e] = r;
          }
          if (STEP) {
            dd.add(make_float2(vc[0], vc[1]), make_float2(qo[0], qo[1]));
            dd.add(make_float2(vc[2], vc[3]), make_float2(qo[2], qo[3]));
          }
          const size_t i = (size_t)gx + (size_t)nx * gy + plane * z;
          *reinterpret_cast<float4*>(Wout + i) = make_float4(qo[0], qo[1], qo[2], qo[3]);
          if (STEP) {
            *reinterpret_cast<float4*>(Vc + i) = make_float4(vc[0], vc[1], vc[2], vc[3]);
            if (a.P.vb) vb_store4(vb_at(a.P, s, j, n, i), vc[0], vc[1], vc[2], vc[3]);
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          vdn[e] = vc[e];
          vc[e] = vup[e];
          vpc[e] = vpu[e];
        }
        abort = __syncthreads_or(bad);  // every thread is done with stage t % kStages
        if (!abort && tid == 0 && t + kStages < P) issue(t + kStages);
      }
    }
    if (abort) {
      // let the copies still in flight land (bounded), record the time-out, leave
      if (tid == 0) {
        for (int b = 0; b < kStages; ++b)
          if (pending & (1u << b)) tma::mbar_wait(&full[b], (ph >> b) & 1u);
        if (STEP) atomicExch(&a.st[s].status, (int)GMRF_ERR_TIMEOUT);
      }
      return;
    }
    if (STEP) {
      const Dots<float> d = block_reduce(dd.merged(), red);
      if (tid == 0) a.partials[(size_t)s * it.per_vec + li] = d;
      if (last_block(a.counters, s, it.per_vec, &s_int[3]))
        finish_step<float>(a.P, j, s, a.partials, it.per_vec, a.st, a.alpha, a.beta, a.alpha_f, a.beta2_f, red,
                           s_int, s_flt);
    }
  }
}

Items make_items(const Grid& g, int nvec) {
  Items it;
  it.ntx = (g.nx + BX - 1) / BX;
  it.nty = (g.ny + BY - 1) / BY;
  // z chunks from the grid alone (so partial sums do not depend on the batch):
  // at least a wave of items per vector, chunks of at least 32 planes
  int c = 1;
  while (it.ntx * it.nty * c < 3 * 152 && g.nz / (2 * c) >= 32) c *= 2;
  it.zper = (g.nz + c - 1) / c;
  if (g.zchunk > 0) it.zper = g.zchunk < g.nz ? g.zchunk : g.nz;  // tuned
  it.nzc = (g.nz + it.zper - 1) / it.zper;
  it.per_vec = it.ntx * it.nty * it.nzc;
  it.total = it.per_vec * nvec;
  return it;
}

template <int BC, bool STEP>
cudaError_t launch_bc(const StencilArgs<float>& a, const Maps& maps, const Items& it, cudaStream_t s) {
  auto k = k_stencil3d_tma<BC, STEP>;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  static int resident = 0;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    int per_sm = 0, dev = 0, nsm = 0;
    if (attr_err == cudaSuccess) attr_err = cudaGetDevice(&dev);
    if (attr_err == cudaSuccess) attr_err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (attr_err == cudaSuccess)
      attr_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, kSmemBytes);
    resident = per_sm * nsm;
    if (attr_err == cudaSuccess && resident < 1) attr_err = cudaErrorInvalidConfiguration;
  });
  if (attr_err != cudaSuccess) return attr_err;
  const int grid = it.total < resident ? it.total : resident;
  if (grid < 1) return cudaSuccess;
  k<<<grid, dim3(32, BY), kSmemBytes, s>>>(a, maps, it);
  return cudaGetLastError();
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

bool stencil3d_tma_eligible(const Grid& g, bool fp64) {
  return !fp64 && g.dim == 3 && g.op == GMRF_OP_SHIFTED_LAPLACIAN && g.bc != GMRF_BC_PERIODIC && g.nx % 4 == 0 &&
         g.nx >= BX && g.ny >= 2 && g.nz >= 2;
}

int stencil3d_tma_items_per_vector(const Grid& g) { return make_items(g, 1).per_vec; }

cudaError_t launch_stencil3d_tma(const Grid& g, const StencilArgs<float>& a, int nvec, bool step, cudaStream_t s) {
  if (!stencil3d_tma_eligible(g, false)) return cudaErrorNotSupported;
  const uint64_t nx = g.nx, ny = g.ny, nz = g.nz;
  const uint64_t rowb = nx * 4, planeb = nx * ny * 4, volb = nx * ny * nz * 4;
  const uint64_t strides[3] = {rowb, planeb, volb};
  const uint32_t hbox[4] = {(uint32_t)TWX, (uint32_t)TWY, 1, 1};
  Maps maps;
  memset(&maps, 0, sizeof(maps));
  bool ok = true;
  if (step) {
    const uint64_t dw[4] = {nx, ny, nz, (uint64_t)nvec};
    const uint64_t dv[4] = {nx, ny, nz, (uint64_t)nvec * (uint64_t)a.P.nslots};
    ok = ok && tma::encode_f32(&maps.w0, a.W0, 4, dw, strides, hbox);
    ok = ok && tma::encode_f32(&maps.w1, a.W1, 4, dw, strides, hbox);
    ok = ok && tma::encode_f32(&maps.v, a.V, 4, dv, strides, hbox);
  } else {
    const uint64_t dw[4] = {nx, ny, nz, (uint64_t)nvec};
    ok = ok && tma::encode_f32(&maps.w0, a.Win, 4, dw, strides, hbox);
    maps.w1 = maps.w0;
    maps.v = maps.w0;
  }
  if (a.kappa2) {
    const uint64_t dk[3] = {nx, ny, nz};
    const uint32_t kbox[3] = {(uint32_t)BX, (uint32_t)BY, 1};
    ok = ok && tma::encode_f32(&maps.k, a.kappa2, 3, dk, strides, kbox);
  } else {
    maps.k = maps.w0;
  }
  if (!ok) return cudaErrorInvalidValue;
  const Items it = make_items(g, nvec);
  if (step) {
    return g.bc == GMRF_BC_NEUMANN ? launch_bc<GMRF_BC_NEUMANN, true>(a, maps, it, s)
                                   : launch_bc<GMRF_BC_DIRICHLET, true>(a, maps, it, s);
  }
  return g.bc == GMRF_BC_NEUMANN ? launch_bc<GMRF_BC_NEUMANN, false>(a, maps, it, s)
                                 : launch_bc<GMRF_BC_DIRICHLET, false>(a, maps, it, s);
}

bool stencil3d_tma_pointers_ok(const void* win, const void* wout, const float* kappa2) {
  return aligned16(win) && aligned16(wout) && (kappa2 == nullptr || aligned16(kappa2));
}

}  // namespace gmrf
