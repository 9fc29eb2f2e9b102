// precond_fast.cuh -- FP32 preconditioner transforms with warp-cooperative
// register FFTs (see precond.cu for the operator they implement).
//
// A line of L = 32 E complex values (E = 2..32) is split over the 32 lanes of
// a warp: lane l holds x[l + 32 r], r < E.  Lines shorter than 1024 complex go
// one per warp (E values per lane, lfft_*, 32-point stage split over lane
// groups).  Lines of 1024 (E = 32) use wfft_*, which can also take G = 32 / E
// lines per warp (32 values per lane): E-point DFTs in registers, twiddles
// W_L^{l k1}, one 32x33 shared-memory transpose, 32-point DFTs in registers;
// the result X[k1 + E k2] sits in lane (g, k1) register k2 ("digit-reversed"
// layout).  The inverse runs the same steps backwards and
// returns the strided layout, so a forward/inverse pair needs no extra
// reordering.  Real transforms of length N = 2L use the half-length packing
// of fft.cuh; the DCT-II packing u[m] = x[2m], u[N-1-m] = x[2m+1] is formed
// from float4 loads and one lane-swap shuffle.
//
// The 2-D spectrum is stored transposed (line kx holds all ky contiguously),
// so the column kernels read and write whole contiguous lines, and the row
// kernels stage their spectrum rows through a shared-memory tile and move it
// in 32-byte segments.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "fft.cuh"
#include "precond.h"
#include "precond_fast.h"
#include "trace.h"

namespace gmrf {
namespace fast {

static __constant__ float2 c_w32[32] = {
    {1.000000000e+00f, -0.000000000e+00f}, {9.807852804e-01f, -1.950903220e-01f},
    {9.238795325e-01f, -3.826834324e-01f}, {8.314696123e-01f, -5.555702330e-01f},
    {7.071067812e-01f, -7.071067812e-01f}, {5.555702330e-01f, -8.314696123e-01f},
    {3.826834324e-01f, -9.238795325e-01f}, {1.950903220e-01f, -9.807852804e-01f},
    {6.123233996e-17f, -1.000000000e+00f}, {-1.950903220e-01f, -9.807852804e-01f},
    {-3.826834324e-01f, -9.238795325e-01f}, {-5.555702330e-01f, -8.314696123e-01f},
    {-7.071067812e-01f, -7.071067812e-01f}, {-8.314696123e-01f, -5.555702330e-01f},
    {-9.238795325e-01f, -3.826834324e-01f}, {-9.807852804e-01f, -1.950903220e-01f},
    {-1.000000000e+00f, -1.224646799e-16f}, {-9.807852804e-01f, 1.950903220e-01f},
    {-9.238795325e-01f, 3.826834324e-01f}, {-8.314696123e-01f, 5.555702330e-01f},
    {-7.071067812e-01f, 7.071067812e-01f}, {-5.555702330e-01f, 8.314696123e-01f},
    {-3.826834324e-01f, 9.238795325e-01f}, {-1.950903220e-01f, 9.807852804e-01f},
    {-1.836970199e-16f, 1.000000000e+00f}, {1.950903220e-01f, 9.807852804e-01f},
    {3.826834324e-01f, 9.238795325e-01f}, {5.555702330e-01f, 8.314696123e-01f},
    {7.071067812e-01f, 7.071067812e-01f}, {8.314696123e-01f, 5.555702330e-01f},
    {9.238795325e-01f, 3.826834324e-01f}, {9.807852804e-01f, 1.950903220e-01f}
};

__host__ __device__ constexpr int brev_c(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
__host__ __device__ constexpr int ilog2_c(int v) { return v <= 1 ? 0 : 1 + ilog2_c(v >> 1); }

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return f2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return f2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return f2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 mulc2(float2 a, float2 b) { return f2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
__device__ __forceinline__ float2 conj2(float2 a) { return f2(a.x, -a.y); }
__device__ __forceinline__ float2 scl2(float2 a, float s) { return f2(a.x * s, a.y * s); }

// In-register radix-2 FFT of length M (<= 32): natural order in and out.
template <int M, bool INV>
__device__ __forceinline__ void reg_fft(float2* v) {
  constexpr int LM = ilog2_c(M);
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int j = brev_c(i, LM);
    if (j > i) {
      const float2 t = v[i];
      v[i] = v[j];
      v[j] = t;
    }
  }
#pragma unroll
  for (int h = 1; h < M; h <<= 1) {
#pragma unroll
    for (int i = 0; i < M; i += 2 * h) {
#pragma unroll
      for (int k = 0; k < h; ++k) {
        float2 w = c_w32[k * (32 / (2 * h))];
        if (INV) w.y = -w.y;
        const float2 t = (k == 0) ? v[i + k + h] : mul2(v[i + k + h], w);
        v[i + k + h] = sub2(v[i + k], t);
        v[i + k] = add2(v[i + k], t);
      }
    }
  }
}

// Forward: v[g*E + r] = x_g[lane + 32 r]  ->  v[k2] = X_g[k1 + E k2], g = lane / E, k1 = lane % E.
// tw[t] = exp(-2 pi i t / TN) with TN = tws * L.  sm: this warp's 32 x 33 scratch.
template <int LOGL>
__device__ __forceinline__ void wfft_fwd(float2 (&v)[32], float2* sm, const float2* __restrict__ tw, int tws) {
  constexpr int E = (1 << LOGL) / 32, G = 32 / E;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int g = 0; g < G; ++g) reg_fft<E, false>(v + g * E);
  if (E > 1) {
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
      for (int k1 = 1; k1 < E; ++k1) v[g * E + k1] = mul2(v[g * E + k1], tw[lane * k1 * tws]);
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 32; ++i) sm[i * 33 + lane] = v[i];
  __syncwarp();
#pragma unroll
  for (int l = 0; l < 32; ++l) v[l] = sm[lane * 33 + l];
  reg_fft<32, false>(v);
}

// Inverse (unnormalised): v[k2] = X_g[k1 + E k2]  ->  v[g*E + r] = L x_g[lane + 32 r].
template <int LOGL>
__device__ __forceinline__ void wfft_inv(float2 (&v)[32], float2* sm, const float2* __restrict__ tw, int tws) {
  constexpr int E = (1 << LOGL) / 32, G = 32 / E;
  const int lane = threadIdx.x & 31;
  const int k1 = lane % E;
  reg_fft<32, true>(v);
  if (E > 1) {
#pragma unroll
    for (int l = 1; l < 32; ++l) v[l] = mulc2(v[l], tw[l * k1 * tws]);
  }
  __syncwarp();
#pragma unroll
  for (int l = 0; l < 32; ++l) sm[lane * 33 + l] = v[l];
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = sm[i * 33 + lane];
#pragma unroll
  for (int g = 0; g < G; ++g) reg_fft<E, true>(v + g * E);
}

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return f2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// One line of L = 32 E complex values per warp, E per lane (E = 2 .. 16):
// L = E x 32 with each 32-point DFT split over S = 32 / E lanes.  Forward: in
// v[r] = z[lane + 32 r]; E-point DFTs over r, twiddles W_L^{lane k1}, an
// E x 33 shared transpose so that lane S k1 + h holds the entries l = S a + h
// of DFT k1, E-point DFTs over a, twiddles W_32^{h j}, and an S-point DFT over
// the lanes h (radix-2 stages by shuffle, decimation in frequency).  Out
// ("split layout"): lane S k1 + h, register j holds Z[k1 + E j + E^2 brev(h)].
// tw[t] = exp(-2 pi i t / TN), TN = tws * L; sc: this warp's E x 33 scratch.
template <int E>
__device__ __forceinline__ int split_index(int lane, int j) {
  constexpr int S = 32 / E, LS = ilog2_c(S);
  return lane / S + E * j + E * E * brev_c(lane % S, LS);
}

template <int E>
__device__ __forceinline__ void lfft_fwd(float2 (&v)[E], float2* sc, const float2* __restrict__ tw, int tws) {
  constexpr int S = 32 / E;
  const int lane = threadIdx.x & 31;
  reg_fft<E, false>(v);
#pragma unroll
  for (int k1 = 1; k1 < E; ++k1) v[k1] = mul2(v[k1], tw[lane * k1 * tws]);
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < E; ++k1) sc[k1 * 33 + lane] = v[k1];
  __syncwarp();
  const int k1 = lane / S, h = lane % S;
#pragma unroll
  for (int a = 0; a < E; ++a) v[a] = sc[k1 * 33 + S * a + h];
  reg_fft<E, false>(v);
  if (h) {
#pragma unroll
    for (int j = 1; j < E; ++j) v[j] = mul2(v[j], c_w32[S == 2 ? j : (h * j) & 31]);
  }
#pragma unroll
  for (int d = S / 2; d >= 1; d >>= 1) {
    const bool up = (h & d) != 0;
    const float2 w = c_w32[(h & (d - 1)) * (16 / d)];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const float2 t = shfl_xor2(v[j], d);
      if (d == 1) v[j] = up ? sub2(t, v[j]) : add2(v[j], t);  // twiddle 1
      else v[j] = up ? mul2(sub2(t, v[j]), w) : add2(v[j], t);
    }
  }
}

// Inverse (unnormalised) of lfft_fwd: split layout in, v[r] = L z[lane + 32 r] out.
template <int E>
__device__ __forceinline__ void lfft_inv(float2 (&v)[E], float2* sc, const float2* __restrict__ tw, int tws) {
  constexpr int S = 32 / E;
  const int lane = threadIdx.x & 31;
  const int k1 = lane / S, h = lane % S;
#pragma unroll
  for (int d = 1; d < S; d <<= 1) {
    const bool up = (h & d) != 0;
    const float2 w = c_w32[(h & (d - 1)) * (16 / d)];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const float2 t = shfl_xor2(v[j], d);
      if (d == 1) v[j] = up ? sub2(t, v[j]) : add2(v[j], t);  // twiddle 1
      else v[j] = up ? sub2(t, mulc2(v[j], w)) : add2(v[j], mulc2(t, w));
    }
  }
  if (h) {
#pragma unroll
    for (int j = 1; j < E; ++j) v[j] = mulc2(v[j], c_w32[S == 2 ? j : (h * j) & 31]);
  }
  reg_fft<E, true>(v);
  __syncwarp();
#pragma unroll
  for (int a = 0; a < E; ++a) sc[k1 * 33 + S * a + h] = v[a];
  __syncwarp();
#pragma unroll
  for (int k = 0; k < E; ++k) v[k] = sc[k * 33 + lane];
#pragma unroll
  for (int k = 1; k < E; ++k) v[k] = mulc2(v[k], tw[lane * k * tws]);
  reg_fft<E, true>(v);
}

enum { R_FWD = 0, R_INV = 1, R_MID = 2, R_MIDW = 3, R_MIDG = 4, R_LAST = 5 };

// Lines per warp and complex values per lane.  Lines of L < 1024 complex go
// one per warp with E = L / 32 values per lane (lfft_*), so that every line of
// a vector has its own warp; lines of L = 1024 put 32 values in each lane of
// one warp (wfft_*).
// COL: the column kernel, which keeps several lines per warp below L = 512
// (its DCT pair pass has L / 2 + 1 pairs, one lane-iteration too many for a
// single short line).
template <int LOGL, bool COL = false>
__host__ __device__ constexpr bool one_line() { return COL ? LOGL == 9 : (LOGL >= 6 && LOGL <= 9); }
template <int LOGL, bool COL = false>
__host__ __device__ constexpr int lpw() { return one_line<LOGL, COL>() ? 1 : 32 / ((1 << LOGL) / 32); }
template <int LOGL, bool COL = false>
__host__ __device__ constexpr int vpl() { return one_line<LOGL, COL>() ? (1 << LOGL) / 32 : 32; }
// per-warp shared scratch (float2): transposes, then one natural-order line per line of the warp
template <int LOGL, bool COL = false>
__host__ __device__ constexpr int scratch_f2() {
  return one_line<LOGL, COL>() ? ((1 << LOGL) / 32) * 33 : 32 * 33;
}

template <int KIND>
__host__ __device__ constexpr int seg_rows() { return KIND == GMRF_PREC_MIRROR ? 8 : 4; }
template <int KIND, int LOGL>
__host__ __device__ constexpr int rows_per_block() {
  return lpw<LOGL>() > seg_rows<KIND>() ? lpw<LOGL>() : seg_rows<KIND>();
}
template <int KIND, int LOGL>
__host__ __device__ constexpr int tile_pitch() {  // floats per tile row
  return KIND == GMRF_PREC_MIRROR ? 2 * (1 << LOGL) + 4 : 2 * (1 << LOGL) + 6;
}

// Copy `count` float2 from global memory to shared memory (all block threads).
__device__ __forceinline__ void stage_table(float2* dst, const float2* __restrict__ src, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = __ldg(src + i);
}
__device__ __forceinline__ void stage_table(float* dst, const float* __restrict__ src, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = __ldg(src + i);
}
__device__ __forceinline__ void stage_table(float4* dst, const float4* __restrict__ src, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = __ldg(src + i);
}

// warps per column block: with one line per warp, 8 lines share the staged tables
template <int LOGL>
__host__ __device__ constexpr int col_warps() { return one_line<LOGL, true>() ? 8 : 4; }

// Dynamic shared memory of the row kernel:
//   tile[RB][TP] floats | per-warp scratch [WPC][scratch_f2] float2 | twx[NX] |
//   MIRROR: pair planes [3][L/2 + 1] float4 (see pair_tab)
template <int KIND, int LOGL>
__host__ __device__ constexpr size_t row_smem_bytes() {
  return (size_t)rows_per_block<KIND, LOGL>() * tile_pitch<KIND, LOGL>() * sizeof(float) +
         (size_t)(rows_per_block<KIND, LOGL>() / lpw<LOGL>()) * scratch_f2<LOGL>() * sizeof(float2) +
         (size_t)2 * (1 << LOGL) * sizeof(float2) +
         (KIND == GMRF_PREC_MIRROR ? (size_t)3 * ((1 << LOGL) / 2 + 1) * sizeof(float4) : 0);
}
// Dynamic shared memory of the column kernel:
//   per-warp scratch [col_warps][scratch_f2] float2 | twy[ny] |
//   CIRCULANT: lamy[ny] floats;  MIRROR: pair records [(L/2 + 1) * 4] float4
template <int KIND, int LOGL>
__host__ __device__ constexpr size_t col_smem_bytes() {
  return (size_t)col_warps<LOGL>() * scratch_f2<LOGL, true>() * sizeof(float2) +
         (KIND == GMRF_PREC_CIRCULANT
              ? (size_t)(1 << LOGL) * (sizeof(float2) + sizeof(float))
              : (size_t)2 * (1 << LOGL) * sizeof(float2) + (size_t)((1 << LOGL) / 2 + 1) * 4 * sizeof(float4));
}

template <int KIND>
__device__ __forceinline__ bool edge_terms(int bc) {
  return KIND == GMRF_PREC_CIRCULANT ? bc != GMRF_BC_PERIODIC : bc != GMRF_BC_NEUMANN;
}
template <int KIND>
__device__ __forceinline__ float edge_val(int bc, float wi, float wp) {
  const float b = bc == GMRF_BC_PERIODIC ? (wi - wp) : (bc == GMRF_BC_DIRICHLET ? wi : 0.f);
  const float pr = KIND == GMRF_PREC_CIRCULANT ? (wi - wp) : 0.f;
  return b - pr;
}

// ----- row layout helpers.  A real row of NX = 2L values is held per lane as
// E float2 "pairs": CIRCULANT pair r = x[2m, 2m+1], m = lane + 32 r;
// MIRROR pairs 2r', 2r'+1 = x[4m .. 4m+3], m = lane + 32 r'.
template <int KIND, int E>
__device__ __forceinline__ size_t pair_off(int lane, int r) {
  if (KIND == GMRF_PREC_CIRCULANT) return (size_t)2 * (lane + 32 * r);
  return (size_t)4 * (lane + 32 * (r >> 1)) + 2 * (r & 1);
}

template <int KIND, int E>
__device__ __forceinline__ void load_row(float2* p, const float* __restrict__ src) {
  const int lane = threadIdx.x & 31;
  if (KIND == GMRF_PREC_CIRCULANT) {
#pragma unroll
    for (int r = 0; r < E; ++r) p[r] = *reinterpret_cast<const float2*>(src + 2 * (lane + 32 * r));
  } else {
#pragma unroll
    for (int r = 0; r < E / 2; ++r) {
      const float4 q = *reinterpret_cast<const float4*>(src + 4 * (lane + 32 * r));
      p[2 * r] = f2(q.x, q.y);
      p[2 * r + 1] = f2(q.z, q.w);
    }
  }
}
template <int KIND, int E>
__device__ __forceinline__ void store_row(const float2* p, float* __restrict__ dst) {
  const int lane = threadIdx.x & 31;
  if (KIND == GMRF_PREC_CIRCULANT) {
#pragma unroll
    for (int r = 0; r < E; ++r) *reinterpret_cast<float2*>(dst + 2 * (lane + 32 * r)) = p[r];
  } else {
#pragma unroll
    for (int r = 0; r < E / 2; ++r)
      *reinterpret_cast<float4*>(dst + 4 * (lane + 32 * r)) = make_float4(p[2 * r].x, p[2 * r].y, p[2 * r + 1].x, p[2 * r + 1].y);
  }
}
template <int KIND, int E>
__device__ __forceinline__ void store_row_bf16(const float2* p, __nv_bfloat16* dst) {
  const int lane = threadIdx.x & 31;
  if (KIND == GMRF_PREC_CIRCULANT) {
#pragma unroll
    for (int r = 0; r < E; ++r) vb_store2(dst + 2 * (lane + 32 * r), p[r].x, p[r].y);
  } else {
#pragma unroll
    for (int r = 0; r < E / 2; ++r)
      vb_store4(dst + 4 * (lane + 32 * r), p[2 * r].x, p[2 * r].y, p[2 * r + 1].x, p[2 * r + 1].y);
  }
}
// row pairs -> packed complex input of the half-length FFT (strided layout)
template <int KIND, int E>
__device__ __forceinline__ void pack_row(const float2* p, float2* v) {
  if (KIND == GMRF_PREC_CIRCULANT) {
#pragma unroll
    for (int r = 0; r < E; ++r) v[r] = p[r];
  } else {
    // z[m] = (x[4m], x[4m+2]); z[L-1-m] = (x[4m+3], x[4m+1]) belongs to lane 31-lane, register E-1-r
#pragma unroll
    for (int r = 0; r < E / 2; ++r) {
      v[r] = f2(p[2 * r].x, p[2 * r + 1].x);
      const float2 o = f2(p[2 * r + 1].y, p[2 * r].y);
      v[E - 1 - r] = f2(__shfl_xor_sync(0xffffffffu, o.x, 31), __shfl_xor_sync(0xffffffffu, o.y, 31));
    }
  }
}
// strided half-length FFT output z -> real row pairs
template <int KIND, int E>
__device__ __forceinline__ void unpack_row(const float2* v, float2* p) {
  if (KIND == GMRF_PREC_CIRCULANT) {
#pragma unroll
    for (int r = 0; r < E; ++r) p[r] = v[r];
  } else {
    // x[4m] = z[m].x, x[4m+2] = z[m].y, x[4m+1] = z[L-1-m].y, x[4m+3] = z[L-1-m].x
#pragma unroll
    for (int r = 0; r < E / 2; ++r) {
      const float2 a = v[r];
      const float2 b = f2(__shfl_xor_sync(0xffffffffu, v[E - 1 - r].x, 31),
                          __shfl_xor_sync(0xffffffffu, v[E - 1 - r].y, 31));
      p[2 * r] = f2(a.x, b.y);
      p[2 * r + 1] = f2(a.y, b.x);
    }
  }
}

// Twiddles and DCT factors of the pair (k, L-k) of a real line of N = 2L
// points.  MIRROR reads them from three planes of L/2 + 1 float4 (consecutive
// pairs contiguous, so a warp's load is conflict-free):
//   plane 0 {tw_k, tw_{L-k}}, plane 1 {d_k, d_{N-k}}, plane 2 {d_{L-k}, d_{N-L+k}}
// with tw_t = exp(-2 pi i t / N) and d_t = exp(-i pi t / (2N)).  CIRCULANT has
// only the twiddles, read from tw[].
struct PairTab {
  float2 twk, twkp, dk, dnk, dkp, dnkp;
};
template <int KIND, int L>
__device__ __forceinline__ PairTab pair_tab(int k, const float2* __restrict__ tw, const float4* __restrict__ pt) {
  PairTab t;
  if (KIND == GMRF_PREC_MIRROR) {
    constexpr int HP1 = L / 2 + 1;
    const float4 P0 = pt[k], P1 = pt[HP1 + k], P2 = pt[2 * HP1 + k];
    t.twk = f2(P0.x, P0.y); t.twkp = f2(P0.z, P0.w);
    t.dk = f2(P1.x, P1.y); t.dnk = f2(P1.z, P1.w);
    t.dkp = f2(P2.x, P2.y); t.dnkp = f2(P2.z, P2.w);
  } else {
    t.twk = tw[k];
    t.twkp = tw[(L - k) & (2 * L - 1)];
    t.dk = t.dnk = t.dkp = t.dnkp = f2(0.f, 0.f);
  }
  return t;
}

// Post-processing of one pair (k, L-k) of the half-length FFT output Z (natural
// order in sm line zl) into the spectrum of the real line: CIRCULANT writes
// X_k (complex) at out[k]; MIRROR writes the DCT-II coefficients C at outr[].
template <int KIND, int L>
__device__ __forceinline__ void post_pair(const float2* zl, int k, const float2* __restrict__ tw,
                                          const float4* __restrict__ pt, float2* outc, float* outr) {
  constexpr int N = 2 * L;
  const float2 zk = zl[k & (L - 1)];
  const float2 zr = zl[(L - k) & (L - 1)];
  if (k == 0) {
    const float x0 = zk.x + zk.y, xl = zk.x - zk.y;
    if (KIND == GMRF_PREC_CIRCULANT) {
      outc[0] = f2(x0, 0.f);
      outc[L] = f2(xl, 0.f);
    } else {
      outr[0] = x0;
      outr[L] = pt[2 * (L / 2 + 1)].x * xl;  // d_L
    }
    return;
  }
  const PairTab t = pair_tab<KIND, L>(k, tw, pt);
  const float2 zc = conj2(zr);
  const float2 d = mul2(t.twk, sub2(zk, zc));
  const float2 Xk = f2(0.5f * (zk.x + zc.x + d.y), 0.5f * (zk.y + zc.y - d.x));
  if (KIND == GMRF_PREC_CIRCULANT) outc[k] = Xk;
  else {
    outr[k] = mul2(t.dk, Xk).x;
    outr[N - k] = mulc2(t.dnk, Xk).x;
  }
  if (2 * k == L) return;
  const int kp = L - k;
  const float2 zkc = conj2(zk);
  const float2 d2 = mul2(t.twkp, sub2(zr, zkc));
  const float2 Xp = f2(0.5f * (zr.x + zkc.x + d2.y), 0.5f * (zr.y + zkc.y - d2.x));
  if (KIND == GMRF_PREC_CIRCULANT) outc[kp] = Xp;
  else {
    outr[kp] = mul2(t.dkp, Xp).x;
    outr[N - kp] = mulc2(t.dnkp, Xp).x;
  }
}

// Pre-processing of one pair (k, L-k): spectrum of a real line (CIRCULANT X,
// MIRROR C) -> Z' (natural order, written to zl) whose unnormalised inverse
// half-length FFT is the packed real line (times L).
template <int KIND, int L>
__device__ __forceinline__ void pre_pair(const float2* inc, const float* inr, int k, const float2* __restrict__ tw,
                                         const float4* __restrict__ pt, float2* zl) {
  constexpr int N = 2 * L;
  float2 Vk, Vp;
  const int kp = L - k;
  const PairTab t = pair_tab<KIND, L>(k, tw, pt);
  if (KIND == GMRF_PREC_CIRCULANT) {
    Vk = inc[k];
    Vp = inc[kp];
  } else {
    const float ck = inr[k], cnk = k == 0 ? 0.f : inr[N - k];
    const float cp = inr[kp], cnp = inr[N - kp];
    Vk = mulc2(f2(ck, -cnk), t.dk);
    Vp = mulc2(f2(cp, -cnp), t.dkp);
  }
  {
    const float2 c = conj2(Vp);
    const float2 E = scl2(add2(Vk, c), 0.5f);
    const float2 O = mulc2(scl2(sub2(Vk, c), 0.5f), t.twk);
    zl[k] = f2(E.x - O.y, E.y + O.x);
  }
  if (k == 0 || 2 * k == L) return;
  {
    const float2 c = conj2(Vk);
    const float2 E = scl2(add2(Vp, c), 0.5f);
    const float2 O = mulc2(scl2(sub2(Vp, c), 0.5f), t.twkp);
    zl[kp] = f2(E.x - O.y, E.y + O.x);
  }
}

__device__ __forceinline__ float kap(const Args& a, size_t i) { return a.kappa2 ? __ldg(a.kappa2 + i) : a.kappa2_const; }

template <int KIND, int E>
__device__ __forceinline__ void load_kap(const Args& a, size_t rowoff, float2* p) {
  if (a.kappa2) load_row<KIND, E>(p, a.kappa2 + rowoff);
  else {
#pragma unroll
    for (int r = 0; r < E; ++r) p[r] = f2(a.kappa2_const, a.kappa2_const);
  }
}

// ----------------------------------------------------------------- rows
// Tile <-> transposed spectrum T.  Tile row i (pitch TP floats) = spectrum of
// grid row y0 + i.  MIRROR: T[kx * ny + y] (reals); CIRCULANT:
// T[(kx * ny + y) complex].
template <int KIND, int LOGL>
__device__ __forceinline__ void tile_store_T(const Args& a, const float* tile, float* Tv, int y0) {
  constexpr int L = 1 << LOGL, RB = rows_per_block<KIND, LOGL>(), TP = tile_pitch<KIND, LOGL>();
  const int tid = threadIdx.x, nt = blockDim.x;
  if (KIND == GMRF_PREC_MIRROR) {
    constexpr int NX = 2 * L, Q = RB / 4;
    for (int idx = tid; idx < NX * Q; idx += nt) {
      const int kx = idx / Q, q = idx - kx * Q;
      const float4 o = make_float4(tile[(4 * q) * TP + kx], tile[(4 * q + 1) * TP + kx], tile[(4 * q + 2) * TP + kx],
                                   tile[(4 * q + 3) * TP + kx]);
      *reinterpret_cast<float4*>(Tv + (size_t)kx * a.ny + y0 + 4 * q) = o;
    }
  } else {
    constexpr int NC = L + 1, Q = RB / 2;
    for (int idx = tid; idx < NC * Q; idx += nt) {
      const int kx = idx / Q, q = idx - kx * Q;
      const float2 c0 = *reinterpret_cast<const float2*>(tile + (2 * q) * TP + 2 * kx);
      const float2 c1 = *reinterpret_cast<const float2*>(tile + (2 * q + 1) * TP + 2 * kx);
      *reinterpret_cast<float4*>(Tv + 2 * ((size_t)kx * a.ny + y0 + 2 * q)) = make_float4(c0.x, c0.y, c1.x, c1.y);
    }
  }
}
template <int KIND, int LOGL>
__device__ __forceinline__ void tile_load_T(const Args& a, float* tile, const float* Tv, int y0) {
  constexpr int L = 1 << LOGL, RB = rows_per_block<KIND, LOGL>(), TP = tile_pitch<KIND, LOGL>();
  const int tid = threadIdx.x, nt = blockDim.x;
  if (KIND == GMRF_PREC_MIRROR) {
    constexpr int NX = 2 * L, Q = RB / 4;
    for (int idx = tid; idx < NX * Q; idx += nt) {
      const int kx = idx / Q, q = idx - kx * Q;
      const float4 o = *reinterpret_cast<const float4*>(Tv + (size_t)kx * a.ny + y0 + 4 * q);
      tile[(4 * q) * TP + kx] = o.x;
      tile[(4 * q + 1) * TP + kx] = o.y;
      tile[(4 * q + 2) * TP + kx] = o.z;
      tile[(4 * q + 3) * TP + kx] = o.w;
    }
  } else {
    constexpr int NC = L + 1, Q = RB / 2;
    for (int idx = tid; idx < NC * Q; idx += nt) {
      const int kx = idx / Q, q = idx - kx * Q;
      const float4 o = *reinterpret_cast<const float4*>(Tv + 2 * ((size_t)kx * a.ny + y0 + 2 * q));
      *reinterpret_cast<float2*>(tile + (2 * q) * TP + 2 * kx) = f2(o.x, o.y);
      *reinterpret_cast<float2*>(tile + (2 * q + 1) * TP + 2 * kx) = f2(o.z, o.w);
    }
  }
}

// forward real transform of the warp's G rows held as pairs p[g][E]; spectrum
// rows written to the tile rows tr0 + g.
template <int KIND, int LOGL>
__device__ __forceinline__ void rows_forward(const Args& a, float2 (&p)[vpl<LOGL>()], float2* sm, float* tile,
                                             int tr0, const float2* twx, const float4* ptx) {
  constexpr int L = 1 << LOGL, E = L / 32, G = lpw<LOGL>(), TP = tile_pitch<KIND, LOGL>();
  const int lane = threadIdx.x & 31;
  float2 v[vpl<LOGL>()];
#pragma unroll
  for (int g = 0; g < G; ++g) pack_row<KIND, E>(p + g * E, v + g * E);
  if constexpr (one_line<LOGL>()) {
    lfft_fwd<E>(v, sm, twx, 2);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < E; ++j) sm[split_index<E>(lane, j)] = v[j];
  } else {
    wfft_fwd<LOGL>(v, sm, twx, 2);
    __syncwarp();
    const int g = lane / E, k1 = lane % E;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) sm[g * L + k1 + E * k2] = v[k2];
  }
  __syncwarp();
  // pairs (k, L - k), k = 0 .. L/2; the lane with k = 0 also takes the cheap
  // k = L/2 item, so the L/2 + 1 items fill whole lane-iterations
  constexpr int HP = L / 2;
  for (int idx = lane; idx < G * HP; idx += 32) {
    const int g = idx / HP, k = idx - g * HP;
    float* trow = tile + (tr0 + g) * TP;
    post_pair<KIND, L>(sm + g * L, k, twx, ptx, reinterpret_cast<float2*>(trow), trow);
    if (k == 0) post_pair<KIND, L>(sm + g * L, HP, twx, ptx, reinterpret_cast<float2*>(trow), trow);
  }
}

// inverse real transform: tile rows tr0 + g -> pairs p[g][E] (times L).
template <int KIND, int LOGL>
__device__ __forceinline__ void rows_inverse(const Args& a, float2 (&p)[vpl<LOGL>()], float2* sm, const float* tile,
                                             int tr0, const float2* twx, const float4* ptx) {
  constexpr int L = 1 << LOGL, E = L / 32, G = lpw<LOGL>(), TP = tile_pitch<KIND, LOGL>();
  const int lane = threadIdx.x & 31;
  constexpr int HP = L / 2;  // k = 0 and k = L/2 go to one lane (see rows_forward)
  __syncwarp();
  for (int idx = lane; idx < G * HP; idx += 32) {
    const int g = idx / HP, k = idx - g * HP;
    const float* trow = tile + (tr0 + g) * TP;
    pre_pair<KIND, L>(reinterpret_cast<const float2*>(trow), trow, k, twx, ptx, sm + g * L);
    if (k == 0) pre_pair<KIND, L>(reinterpret_cast<const float2*>(trow), trow, HP, twx, ptx, sm + g * L);
  }
  __syncwarp();
  float2 v[vpl<LOGL>()];
  if constexpr (one_line<LOGL>()) {
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = sm[split_index<E>(lane, j)];
    __syncwarp();
    lfft_inv<E>(v, sm, twx, 2);
  } else {
    const int g = lane / E, k1 = lane % E;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) v[k2] = sm[g * L + k1 + E * k2];
    wfft_inv<LOGL>(v, sm, twx, 2);
  }
#pragma unroll
  for (int g = 0; g < G; ++g) unpack_row<KIND, E>(v + g * E, p + g * E);
}

template <int KIND, int LOGL, int MODE>
__global__ void __launch_bounds__(32 * (rows_per_block<KIND, LOGL>() / lpw<LOGL>()), LOGL == 9 ? 1 : (LOGL == 8 ? 4 : 0))
    k_row(Args a) {
  constexpr int L = 1 << LOGL, E = L / 32, G = lpw<LOGL>(), NX = 2 * L;
  constexpr int RB = rows_per_block<KIND, LOGL>(), TP = tile_pitch<KIND, LOGL>();
  extern __shared__ __align__(16) float smf[];
  __shared__ Dots<float> red[8];
  __shared__ int s_int[4];
  __shared__ float s_flt[4];
  constexpr int WPC = RB / G;
  float* tile = smf;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* sm = reinterpret_cast<float2*>(smf + RB * TP) + warp * scratch_f2<LOGL>();
  float2* twx = reinterpret_cast<float2*>(smf + RB * TP) + WPC * scratch_f2<LOGL>();  // [NX] exp(-2 pi i t / NX)
  float4* ptx = reinterpret_cast<float4*>(twx + NX);  // MIRROR: 3 planes of NX/4 + 1 (see pair_tab)
  const int s = blockIdx.y;
  const bool step = (MODE == R_FWD || MODE == R_LAST || MODE == R_MID || MODE == R_MIDW || MODE == R_MIDG) &&
                    a.in == nullptr;
  int j = 0;
  if (step) {
    if (a.st[s].status != VS_RUNNING) return;
    j = a.st[s].m;
  }
  const int y0 = blockIdx.x * RB;
  const int tr0 = warp * G;       // first tile row of this warp
  const size_t n = a.n;
  float* Tv = a.T + (size_t)s * a.tstride;
  float2 p[vpl<LOGL>()];
  const size_t slot = (size_t)s * a.P.nslots;
  // the transform tables are staged behind the block's first global loads,
  // so that both latencies overlap (one barrier)
  auto stage_tables = [&]() {
    stage_table(twx, a.twx, NX);
    if (KIND == GMRF_PREC_MIRROR) stage_table(ptx, a.pairx, 3 * (NX / 4 + 1));
  };

  if (MODE == R_FWD) {
    const float* Win = a.in ? a.in + (size_t)s * n : (((j & 1) ? a.W1 : a.W0) + (size_t)s * n);
    float* Vc = a.in ? nullptr : a.V + (slot + (size_t)(j % a.P.nslots)) * n;
    const float* Vp = (!a.in && j > 0) ? a.V + (slot + (size_t)((j - 1) % a.P.nslots)) * n : nullptr;
    float coef = 0.f, inv_b = 1.f;
    if (!a.in) {
      if (j == 0) inv_b = (float)a.st[s].vscale;
      else {
        const size_t mo = (size_t)s * a.P.m_max + (j - 1);
        coef = (float)a.alpha[mo];
        inv_b = (float)a.st[s].vscale;
      }
    }
    float2 qv[vpl<LOGL>()];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const size_t ro = (size_t)(y0 + tr0 + g) * NX;
      load_row<KIND, E>(p + g * E, Win + ro);
      if (Vp) load_row<KIND, E>(qv + g * E, Vp + ro);
    }
    stage_tables();
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const size_t ro = (size_t)(y0 + tr0 + g) * NX;
      if (!a.in) {
        if (j > 0) {
          const float2* q = qv + g * E;
#pragma unroll
          for (int r = 0; r < E; ++r)
            p[g * E + r] = f2((p[g * E + r].x - coef * q[r].x) * inv_b, (p[g * E + r].y - coef * q[r].y) * inv_b);
        } else {
#pragma unroll
          for (int r = 0; r < E; ++r) p[g * E + r] = scl2(p[g * E + r], inv_b);
        }
        store_row<KIND, E>(p + g * E, Vc + ro);
        if (a.P.vb) store_row_bf16<KIND, E>(p + g * E, vb_at(a.P, s, j, n, ro));
      }
    }
    rows_forward<KIND, LOGL>(a, p, sm, tile, tr0, twx, ptx);
    __syncthreads();
    tile_store_T<KIND, LOGL>(a, tile, Tv, y0);
    return;
  }

  // inverse transform of the block's rows
  const float* vsrc = a.in ? a.in + (size_t)s * n : a.V + (slot + (size_t)(j % a.P.nslots)) * n;
  const float* gsrc = a.form == FORM_CTC ? a.G + (size_t)s * n : vsrc;
  // Rows of 1024 (one per warp, one block per SM at one vector): the arrays
  // the elementwise part reads after the inverse transform are loaded before
  // it, so that their latency overlaps the table staging and the transform
  // (pa, pb, pc: kappa^2 and v for R_MID; g, v and v_{j-1} for R_LAST).
  constexpr bool PF = LOGL == 9 && G == 1 && (MODE == R_MID || MODE == R_LAST);
  float2 pa[PF ? E : 1], pb[PF ? E : 1], pc[PF ? E : 1];
  if constexpr (PF) {
    const size_t ro = (size_t)(y0 + tr0) * NX;
    if (MODE == R_MID) {
      load_kap<KIND, E>(a, ro, pa);
      if (a.form == FORM_CTC) load_row<KIND, E>(pb, vsrc + ro);
    } else {
      load_row<KIND, E>(pa, gsrc + ro);
      if (!a.in) {
        load_row<KIND, E>(pb, vsrc + ro);
        if (j > 0) load_row<KIND, E>(pc, a.V + (slot + (size_t)((j - 1) % a.P.nslots)) * n + ro);
      }
    }
  }
  stage_tables();
  if (MODE != R_MIDG) tile_load_T<KIND, LOGL>(a, tile, Tv, y0);
  __syncthreads();
  if (MODE != R_MIDG) rows_inverse<KIND, LOGL>(a, p, sm, tile, tr0, twx, ptx);
  if (MODE == R_INV) {
#pragma unroll
    for (int g = 0; g < G; ++g) store_row<KIND, E>(p + g * E, a.out + (size_t)s * n + (size_t)(y0 + tr0 + g) * NX);
    return;
  }
  if (MODE == R_MIDW) {
    float* wg = a.Wg + (size_t)s * n;
#pragma unroll
    for (int g = 0; g < G; ++g) store_row<KIND, E>(p + g * E, wg + (size_t)(y0 + tr0 + g) * NX);
    return;
  }
  if (MODE == R_MID || MODE == R_MIDG) {
    // p holds w = B_bar^{-1} v (MID) or is loaded from the global w buffer
    // (MIDG, which also applies the y-boundary terms with the partner row).
    const float* wg = a.Wg + (size_t)s * n;
    const bool ex = edge_terms<KIND>(a.bc);
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int y = y0 + tr0 + g;
      const size_t ro = (size_t)y * NX;
      float2* w = p + g * E;
      if (MODE == R_MIDG) load_row<KIND, E>(w, wg + ro);
      const bool hy = MODE == R_MIDG && (y == 0 || y == a.ny - 1);
      const size_t rp = (size_t)((y == 0) ? a.ny - 1 : 0) * NX;
      // partner row's g (needed for the y-term of R g at this row)
      float2 gp[E];
      if (hy && a.form == FORM_CTC) {
        float wpf = 0.f, wpl = 0.f;
        float2 wp[E];
        load_row<KIND, E>(wp, wg + rp);
        if (ex) {
          wpl = __shfl_sync(0xffffffffu, wp[E - 1].y, 31);
          wpf = __shfl_sync(0xffffffffu, wp[0].x, 0);
        }
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const size_t o = rp + pair_off<KIND, E>(lane, i);
          const float2 kk = a.kappa2 ? *reinterpret_cast<const float2*>(a.kappa2 + o) : f2(a.kappa2_const, a.kappa2_const);
          const float2 vp = *reinterpret_cast<const float2*>(vsrc + o);
          float2 t = f2(vp.x + (kk.x - a.roff) * wp[i].x + edge_val<KIND>(a.bc, wp[i].x, w[i].x),
                        vp.y + (kk.y - a.roff) * wp[i].y + edge_val<KIND>(a.bc, wp[i].y, w[i].y));
          if (lane == 0 && i == 0) t.x += edge_val<KIND>(a.bc, wp[0].x, wpl);
          if (lane == 31 && i == E - 1) t.y += edge_val<KIND>(a.bc, wp[E - 1].y, wpf);
          gp[i] = t;
        }
      }
      float wf = 0.f, wl = 0.f;
      if (ex) {
        wl = __shfl_sync(0xffffffffu, w[E - 1].y, 31);
        wf = __shfl_sync(0xffffffffu, w[0].x, 0);
      }
      // rg = R w (in place), then g = v + rg (squared operator)
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const size_t o = ro + pair_off<KIND, E>(lane, i);
        float2 kk;
        if constexpr (PF) kk = pa[i];
        else kk = a.kappa2 ? *reinterpret_cast<const float2*>(a.kappa2 + o) : f2(a.kappa2_const, a.kappa2_const);
        float2 t = f2((kk.x - a.roff) * w[i].x, (kk.y - a.roff) * w[i].y);
        if (ex && lane == 0 && i == 0) t.x += edge_val<KIND>(a.bc, w[0].x, wl);
        if (ex && lane == 31 && i == E - 1) t.y += edge_val<KIND>(a.bc, w[E - 1].y, wf);
        if (hy) {
          // y partner of w: reload from the global w buffer
          const float2 wq = *reinterpret_cast<const float2*>(wg + rp + pair_off<KIND, E>(lane, i));
          t.x += edge_val<KIND>(a.bc, w[i].x, wq.x);
          t.y += edge_val<KIND>(a.bc, w[i].y, wq.y);
        }
        if (a.form == FORM_CTC) {
          float2 vv;
          if constexpr (PF) vv = pb[i];
          else vv = *reinterpret_cast<const float2*>(vsrc + o);
          t = add2(vv, t);
        }
        w[i] = t;
      }
      if (a.form == FORM_CTC) {
        store_row<KIND, E>(w, a.G + (size_t)s * n + ro);
        // r = R g (in place)
        float gf = 0.f, gl = 0.f;
        if (ex) {
          gl = __shfl_sync(0xffffffffu, w[E - 1].y, 31);
          gf = __shfl_sync(0xffffffffu, w[0].x, 0);
        }
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const size_t o = ro + pair_off<KIND, E>(lane, i);
          float2 kk;
          if constexpr (PF) kk = pa[i];
          else kk = a.kappa2 ? *reinterpret_cast<const float2*>(a.kappa2 + o) : f2(a.kappa2_const, a.kappa2_const);
          float2 t = f2((kk.x - a.roff) * w[i].x, (kk.y - a.roff) * w[i].y);
          if (ex && lane == 0 && i == 0) t.x += edge_val<KIND>(a.bc, w[0].x, gl);
          if (ex && lane == 31 && i == E - 1) t.y += edge_val<KIND>(a.bc, w[E - 1].y, gf);
          if (hy) {
            t.x += edge_val<KIND>(a.bc, w[i].x, gp[i].x);
            t.y += edge_val<KIND>(a.bc, w[i].y, gp[i].y);
          }
          w[i] = t;
        }
      }
    }
    __syncthreads();  // tile rows consumed by every warp before they are rewritten
    rows_forward<KIND, LOGL>(a, p, sm, tile, tr0, twx, ptx);
    __syncthreads();
    tile_store_T<KIND, LOGL>(a, tile, Tv, y0);
    return;
  }
  // R_LAST: A v = g + h
  if (a.in) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const size_t ro = (size_t)(y0 + tr0 + g) * NX;
      float2 gg[E];
      if constexpr (PF) {
#pragma unroll
        for (int i = 0; i < E; ++i) gg[i] = pa[i];
      } else {
        load_row<KIND, E>(gg, gsrc + ro);
      }
#pragma unroll
      for (int i = 0; i < E; ++i) gg[i] = add2(gg[i], p[g * E + i]);
      store_row<KIND, E>(gg, a.out + (size_t)s * n + ro);
    }
    return;
  }
  const float* Vp = j > 0 ? a.V + (slot + (size_t)((j - 1) % a.P.nslots)) * n : nullptr;
  const float bprev = j > 0 ? (float)a.beta[(size_t)s * a.P.m_max + (j - 1)] : 0.f;
  float* Wo = ((j & 1) ? a.W0 : a.W1) + (size_t)s * n;
  Dots<float> d;
  d.zero();
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const size_t ro = (size_t)(y0 + tr0 + g) * NX;
    float2 gg[E], vv[E], q[E];
    if constexpr (PF) {
#pragma unroll
      for (int i = 0; i < E; ++i) {
        gg[i] = pa[i];
        vv[i] = pb[i];
        q[i] = pc[i];
      }
    } else {
      load_row<KIND, E>(gg, gsrc + ro);
      load_row<KIND, E>(vv, vsrc + ro);
      if (j > 0) load_row<KIND, E>(q, Vp + ro);
    }
#pragma unroll
    for (int i = 0; i < E; ++i) {
      float2 t = add2(gg[i], p[g * E + i]);
      if (j > 0) t = f2(t.x - bprev * q[i].x, t.y - bprev * q[i].y);
      q[i] = t;
      d.add_dot2(vv[i].x, t.x);  // Dot2: 10 operations per product instead of 13
      d.add_dot2(vv[i].y, t.y);
    }
    store_row<KIND, E>(q, Wo + ro);
  }
  d = block_reduce(d, red);
  const int nblk = gridDim.x;
  if (threadIdx.x == 0) a.partials[(size_t)s * nblk + blockIdx.x] = d;
  if (last_block(a.counters, s, nblk, &s_int[3]))
    finish_step<float>(a.P, j, s, a.partials, nblk, a.st, a.alpha, a.beta, a.alpha_f, a.beta2_f, red, s_int, s_flt);
}

// ----------------------------------------------------------------- columns
// symbol of B_bar^{-p/2} (times the transform normalisation); cx = kappa_bar^2 + lambda_x
__device__ __forceinline__ float sym_l(const Args& a, float cx, float lam_y) {
  const float r = rsqrtf(cx + lam_y);  // lam^{-1/2}; lam^{-1} = r^2 (a few ulp, no division)
  return (a.power == 2 ? r * r : r) * a.dscale;
}
__device__ __forceinline__ float sym(const Args& a, float cx, const float* lamy, int ky) {
  return sym_l(a, cx, lamy[ky]);
}

template <int KIND, int LOGL>
__global__ void __launch_bounds__(32 * col_warps<LOGL>()) k_col(Args a, int step_mode) {
  constexpr int L = 1 << LOGL, E = L / 32, G = lpw<LOGL, true>(), VN = vpl<LOGL, true>();
  constexpr int NYc = KIND == GMRF_PREC_CIRCULANT ? L : 2 * L;  // ny
  extern __shared__ __align__(16) float smf[];
  const int s = blockIdx.y;
  if (step_mode && a.st[s].status != VS_RUNNING) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2* sm = reinterpret_cast<float2*>(smf) + warp * scratch_f2<LOGL, true>();
  // layout (must match col_smem_bytes): warp scratch | twy[ny] | CIRCULANT: lamy[ny]; MIRROR: pair records
  float2* twy = reinterpret_cast<float2*>(smf) + col_warps<LOGL>() * scratch_f2<LOGL, true>();
  float* lamy = reinterpret_cast<float*>(twy + NYc);
  float4* ptab = reinterpret_cast<float4*>(twy + NYc);  // NYc float2 keep it 16-byte aligned
  // the tables are staged after the warp's line loads are issued (one barrier)
  auto stage_tables = [&]() {
    stage_table(twy, a.twy, NYc);
    if (KIND == GMRF_PREC_MIRROR) stage_table(ptab, a.pairy, 4 * (L / 2 + 1));
    else stage_table(lamy, a.lamy, NYc);
    __syncthreads();
  };
  float* Tv = a.T + (size_t)s * a.tstride;
  const int line0 = (blockIdx.x * col_warps<LOGL>() + warp) * G;
  float2 v[VN];
  if (KIND == GMRF_PREC_CIRCULANT) {
    // complex lines kx = 0..nx/2 of length ny = L
    const int ncl = a.nx / 2 + 1;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int kx = line0 + g;
      const float2* src = reinterpret_cast<const float2*>(Tv) + (size_t)kx * L;
#pragma unroll
      for (int r = 0; r < E; ++r) v[g * E + r] = kx < ncl ? src[lane + 32 * r] : f2(0.f, 0.f);
    }
    stage_tables();
    if constexpr (one_line<LOGL, true>()) {
      lfft_fwd<E>(v, sm, twy, 1);
      if (line0 < ncl) {
        const float cx = a.kbar2 + __ldg(a.lamx + line0);
#pragma unroll
        for (int j = 0; j < E; ++j) v[j] = scl2(v[j], sym(a, cx, lamy, split_index<E>(lane, j)));
      }
      lfft_inv<E>(v, sm, twy, 1);
    } else {
      wfft_fwd<LOGL>(v, sm, twy, 1);
      {
        const int g = lane / E, k1 = lane % E, kx = line0 + g;
        if (kx < ncl) {
          const float cx = a.kbar2 + __ldg(a.lamx + kx);
#pragma unroll
          for (int k2 = 0; k2 < 32; ++k2) v[k2] = scl2(v[k2], sym(a, cx, lamy, k1 + E * k2));
        }
      }
      wfft_inv<LOGL>(v, sm, twy, 1);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int kx = line0 + g;
      if (kx < ncl) {
        float2* dst = reinterpret_cast<float2*>(Tv) + (size_t)kx * L;
#pragma unroll
        for (int r = 0; r < E; ++r) dst[lane + 32 * r] = v[g * E + r];
      }
    }
    return;
  }
  // MIRROR: real lines kx = 0..nx-1 of length ny = 2L (DCT-II, symbol, inverse)
  constexpr int NY = 2 * L;
  float2 p[VN];
#pragma unroll
  for (int g = 0; g < G; ++g) {
    if (line0 + g < a.nx) load_row<KIND, E>(p + g * E, Tv + (size_t)(line0 + g) * NY);
    else {
#pragma unroll
      for (int r = 0; r < E; ++r) p[g * E + r] = f2(0.f, 0.f);
    }
  }
  stage_tables();
#pragma unroll
  for (int g = 0; g < G; ++g) pack_row<KIND, E>(p + g * E, v + g * E);
  if constexpr (one_line<LOGL, true>()) {
    lfft_fwd<E>(v, sm, twy, 2);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < E; ++j) sm[split_index<E>(lane, j)] = v[j];
  } else {
    wfft_fwd<LOGL>(v, sm, twy, 2);
    __syncwarp();
    const int g = lane / E, k1 = lane % E;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) sm[g * L + k1 + E * k2] = v[k2];
  }
  float cxl[G];
#pragma unroll
  for (int g = 0; g < G; ++g) cxl[g] = line0 + g < a.nx ? a.kbar2 + __ldg(a.lamx + line0 + g) : 1.f;
  __syncwarp();
  // pairs (k, L - k), k = 0 .. L/2; the lane with k = 0 also takes k = L/2
  constexpr int HP = L / 2;
  auto pair = [&](int g, int k) {
    const int kx = line0 + g;
    float cx = cxl[0];
#pragma unroll
    for (int q = 1; q < G; ++q)
      if (g == q) cx = cxl[q];
    float C[4] = {0.f, 0.f, 0.f, 0.f};
    int nc = 0;
    float2* zl = sm + g * L;
    const bool live = kx < a.nx;
    // the pair's entries, one float4 from each of four planes (consecutive k are contiguous):
    // twiddles tw_k, tw_kp | DCT factors d_k, d_{NY-k} | d_kp, d_{NY-kp} | 4 lambda_y
    const float4 P0 = ptab[k], P1 = ptab[(HP + 1) + k], P2 = ptab[2 * (HP + 1) + k], P3 = ptab[3 * (HP + 1) + k];
    const float2 twk = f2(P0.x, P0.y), twkp = f2(P0.z, P0.w);
    const float2 dk = f2(P1.x, P1.y), dnk = f2(P1.z, P1.w), dkp = f2(P2.x, P2.y), dnkp = f2(P2.z, P2.w);
    const float lam[4] = {P3.x, P3.y, P3.z, P3.w};
    // DCT coefficients of this pair, scaled by the symbol
    {
      const float2 zk = zl[k & (L - 1)];
      const float2 zr = zl[(L - k) & (L - 1)];
      if (k == 0) {
        C[0] = zk.x + zk.y;
        C[1] = dkp.x * (zk.x - zk.y);  // d_L
        nc = 2;
      } else {
        const float2 zc = conj2(zr);
        const float2 d = mul2(twk, sub2(zk, zc));
        const float2 Xk = f2(0.5f * (zk.x + zc.x + d.y), 0.5f * (zk.y + zc.y - d.x));
        C[0] = mul2(dk, Xk).x;
        C[1] = mulc2(dnk, Xk).x;
        nc = 2;
        if (2 * k != L) {
          const float2 zkc = conj2(zk);
          const float2 d2 = mul2(twkp, sub2(zr, zkc));
          const float2 Xp = f2(0.5f * (zr.x + zkc.x + d2.y), 0.5f * (zr.y + zkc.y - d2.x));
          C[2] = mul2(dkp, Xp).x;
          C[3] = mulc2(dnkp, Xp).x;
          nc = 4;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (i < nc) C[i] = live ? C[i] * sym_l(a, cx, lam[i]) : 0.f;
    // inverse pre-processing of the same pair
    const int kp = L - k;
    float ck, cnk, cp, cnp;
    if (k == 0) { ck = C[0]; cnk = 0.f; cp = C[1]; cnp = C[1]; }
    else if (2 * k == L) { ck = C[0]; cnk = C[1]; cp = C[0]; cnp = C[1]; }
    else { ck = C[0]; cnk = C[1]; cp = C[2]; cnp = C[3]; }
    const float2 Vk = mulc2(f2(ck, -cnk), dk);
    const float2 Vp = mulc2(f2(cp, -cnp), dkp);
    {
      const float2 c = conj2(Vp);
      const float2 Ev = scl2(add2(Vk, c), 0.5f);
      const float2 O = mulc2(scl2(sub2(Vk, c), 0.5f), twk);
      zl[k] = f2(Ev.x - O.y, Ev.y + O.x);
    }
    if (k != 0 && 2 * k != L) {
      const float2 c = conj2(Vk);
      const float2 Ev = scl2(add2(Vp, c), 0.5f);
      const float2 O = mulc2(scl2(sub2(Vp, c), 0.5f), twkp);
      zl[kp] = f2(Ev.x - O.y, Ev.y + O.x);
    }
  };
  for (int idx = lane; idx < G * HP; idx += 32) {
    const int g = idx / HP, k = idx - g * HP;
    pair(g, k);
    if (k == 0) pair(g, HP);
  }
  __syncwarp();
  if constexpr (one_line<LOGL, true>()) {
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = sm[split_index<E>(lane, j)];
    __syncwarp();
    lfft_inv<E>(v, sm, twy, 2);
  } else {
    const int g = lane / E, k1 = lane % E;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) v[k2] = sm[g * L + k1 + E * k2];
    wfft_inv<LOGL>(v, sm, twy, 2);
  }
#pragma unroll
  for (int g = 0; g < G; ++g) unpack_row<KIND, E>(v + g * E, p + g * E);
#pragma unroll
  for (int g = 0; g < G; ++g)
    if (line0 + g < a.nx) store_row<KIND, E>(p + g * E, Tv + (size_t)(line0 + g) * NY);
}

}  // namespace fast
}  // namespace gmrf

namespace gmrf {
namespace fast {

// ----------------------------------------------------------------- launchers
template <int KIND, int LOGL, int MODE>
cudaError_t row_launch_t(const Args& a, int nvec, cudaStream_t s, int kc) {
  constexpr int G = lpw<LOGL>();
  constexpr int RB = rows_per_block<KIND, LOGL>(), TP = tile_pitch<KIND, LOGL>();
  constexpr int WPC = RB / G;
  const size_t sm = row_smem_bytes<KIND, LOGL>();
  static std::atomic<bool> attr{false};  // several host threads may launch at once
  if (!attr.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(k_row<KIND, LOGL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr.store(true, std::memory_order_release);
  }
  dim3 grd(a.ny / RB, nvec);
  trace_begin(kc, s);
  k_row<KIND, LOGL, MODE><<<grd, 32 * WPC, sm, s>>>(a);
  trace_end(kc, s);
  return cudaGetLastError();
}

template <int KIND, int MODE>
cudaError_t row_launch(const Args& a, int nvec, cudaStream_t s, int kc) {
  switch (a.nx) {
    case 128: return row_launch_t<KIND, 6, MODE>(a, nvec, s, kc);
    case 256: return row_launch_t<KIND, 7, MODE>(a, nvec, s, kc);
    case 512: return row_launch_t<KIND, 8, MODE>(a, nvec, s, kc);
    case 1024: return row_launch_t<KIND, 9, MODE>(a, nvec, s, kc);
    case 2048: return row_launch_t<KIND, 10, MODE>(a, nvec, s, kc);
    default: return cudaErrorInvalidValue;
  }
}

template <int KIND, int LOGL>
cudaError_t col_launch_t(const Args& a, int nvec, int step_mode, cudaStream_t s, int kc) {
  constexpr int G = lpw<LOGL, true>();
  const int nlines = KIND == GMRF_PREC_CIRCULANT ? a.nx / 2 + 1 : a.nx;
  const int per = col_warps<LOGL>() * G;
  const size_t sm = col_smem_bytes<KIND, LOGL>();
  static std::atomic<bool> attr{false};  // several host threads may launch at once
  if (!attr.load(std::memory_order_acquire)) {
    cudaError_t e = cudaFuncSetAttribute(k_col<KIND, LOGL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr.store(true, std::memory_order_release);
  }
  dim3 grd((nlines + per - 1) / per, nvec);
  trace_begin(kc, s);
  k_col<KIND, LOGL><<<grd, 32 * col_warps<LOGL>(), sm, s>>>(a, step_mode);
  trace_end(kc, s);
  return cudaGetLastError();
}

template <int KIND>
cudaError_t col_launch(const Args& a, int nvec, int step_mode, cudaStream_t s, int kc) {
  const int L = KIND == GMRF_PREC_CIRCULANT ? a.ny : a.ny / 2;
  switch (L) {
    case 64: return col_launch_t<KIND, 6>(a, nvec, step_mode, s, kc);
    case 128: return col_launch_t<KIND, 7>(a, nvec, step_mode, s, kc);
    case 256: return col_launch_t<KIND, 8>(a, nvec, step_mode, s, kc);
    case 512: return col_launch_t<KIND, 9>(a, nvec, step_mode, s, kc);
    case 1024: return col_launch_t<KIND, 10>(a, nvec, step_mode, s, kc);
    default: return cudaErrorInvalidValue;
  }
}

inline bool host_edge_terms(int kind, int bc) {
  return kind == GMRF_PREC_CIRCULANT ? bc != GMRF_BC_PERIODIC : bc != GMRF_BC_NEUMANN;
}

#define FAST_CK(x)                         \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return e_;      \
  } while (0)

// one preconditioned Lanczos step
template <int KIND>
cudaError_t step_k(const Args& a, int nvec, cudaStream_t s) {
  FAST_CK((row_launch<KIND, R_FWD>(a, nvec, s, KC_PRE_ROW_FWD)));
  FAST_CK((col_launch<KIND>(a, nvec, 1, s, KC_PRE_COL)));
  if (host_edge_terms(KIND, a.bc)) {
    FAST_CK((row_launch<KIND, R_MIDW>(a, nvec, s, KC_PRE_ROW_MID)));
    FAST_CK((row_launch<KIND, R_MIDG>(a, nvec, s, KC_PRE_ROW_MID)));
  } else {
    FAST_CK((row_launch<KIND, R_MID>(a, nvec, s, KC_PRE_ROW_MID)));
  }
  FAST_CK((col_launch<KIND>(a, nvec, 1, s, KC_PRE_COL)));
  FAST_CK((row_launch<KIND, R_LAST>(a, nvec, s, KC_PRE_ROW_LAST)));
  return cudaSuccess;
}

// out = B_bar^{-p/2} in
template <int KIND>
cudaError_t apply_k(const Args& a, int nvec, cudaStream_t s) {
  FAST_CK((row_launch<KIND, R_FWD>(a, nvec, s, KC_PRE_APPLY)));
  FAST_CK((col_launch<KIND>(a, nvec, 0, s, KC_PRE_APPLY)));
  FAST_CK((row_launch<KIND, R_INV>(a, nvec, s, KC_PRE_APPLY)));
  return cudaSuccess;
}

// out = A in
template <int KIND>
cudaError_t operator_k(const Args& a, int nvec, cudaStream_t s) {
  FAST_CK((row_launch<KIND, R_FWD>(a, nvec, s, KC_PRE_APPLY)));
  FAST_CK((col_launch<KIND>(a, nvec, 0, s, KC_PRE_APPLY)));
  if (host_edge_terms(KIND, a.bc)) {
    FAST_CK((row_launch<KIND, R_MIDW>(a, nvec, s, KC_PRE_APPLY)));
    FAST_CK((row_launch<KIND, R_MIDG>(a, nvec, s, KC_PRE_APPLY)));
  } else {
    FAST_CK((row_launch<KIND, R_MID>(a, nvec, s, KC_PRE_APPLY)));
  }
  FAST_CK((col_launch<KIND>(a, nvec, 0, s, KC_PRE_APPLY)));
  FAST_CK((row_launch<KIND, R_LAST>(a, nvec, s, KC_PRE_APPLY)));
  return cudaSuccess;
}

}  // namespace fast
}  // namespace gmrf
