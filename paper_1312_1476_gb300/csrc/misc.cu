// misc.cu -- noise generation (Algorithm 1, first step; Section 6 probes),
// Lanczos start-up (v_1 = z / ||z||), sample assembly x_m = ||z|| V_m y
// (Algorithm 1, last step) and small elementwise helpers.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>
#include <math.h>

#include "internal.h"

namespace gmrf {
namespace {

// Gaussian stream: group g of vector s -> counter (g, s, 0, 0); Box-Muller on
// (w0, w1) and (w2, w3), u = ((w >> 8) + 1/2) 2^-24.
template <typename T>
__global__ void k_rng_gauss(T* out, int64_t nvec, int64_t n, uint32_t k0, uint32_t k1, int64_t soff) {
  const int64_t ng = (n + 3) / 4;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nvec * ng;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx / ng, g = idx - s * ng;
    uint32_t c[4] = {(uint32_t)g, (uint32_t)(s + soff), 0u, 0u};
    philox4x32_10(c, k0, k1);
    T z[4];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      if (sizeof(T) == 4) {
        float ua = ((float)(c[2 * p] >> 8) + 0.5f) * 5.9604644775390625e-8f;
        float ub = ((float)(c[2 * p + 1] >> 8) + 0.5f) * 5.9604644775390625e-8f;
        float r = sqrtf(-2.0f * logf(ua));
        float sn, cs;
        sincospif(2.0f * ub, &sn, &cs);
        z[2 * p] = (T)(r * cs);
        z[2 * p + 1] = (T)(r * sn);
      } else {
        double ua = ((double)(c[2 * p] >> 8) + 0.5) * 5.9604644775390625e-8;
        double ub = ((double)(c[2 * p + 1] >> 8) + 0.5) * 5.9604644775390625e-8;
        double r = sqrt(-2.0 * log(ua));
        double sn, cs;
        sincospi(2.0 * ub, &sn, &cs);
        z[2 * p] = (T)(r * cs);
        z[2 * p + 1] = (T)(r * sn);
      }
    }
    T* o = out + s * n + 4 * g;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (4 * g + e < n) o[e] = z[e];
  }
}

__global__ void k_rng_words(uint32_t* out, int64_t nvec, int64_t n, uint32_t k0, uint32_t k1, int64_t soff) {
  const int64_t ng = (n + 3) / 4;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nvec * ng;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx / ng, g = idx - s * ng;
    uint32_t c[4] = {(uint32_t)g, (uint32_t)(s + soff), 0u, 0u};
    philox4x32_10(c, k0, k1);
    uint32_t* o = out + s * (4 * ng) + 4 * g;
    o[0] = c[0];
    o[1] = c[1];
    o[2] = c[2];
    o[3] = c[3];
  }
}

// Rademacher stream: element e of probe s is bit e%32 of word (e/32)%4 of
// Philox counter (e/128, s, 1, 0).  One thread per 32 elements.
template <typename T>
__global__ void k_rng_rademacher(T* out, int64_t nvec, int64_t n, uint32_t k0, uint32_t k1, int64_t soff) {
  const int64_t nw = (n + 31) / 32;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nvec * nw;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx / nw, w = idx - s * nw;
    uint32_t c[4] = {(uint32_t)(w / 4), (uint32_t)(s + soff), 1u, 0u};
    philox4x32_10(c, k0, k1);
    const uint32_t word = c[w & 3];
    T* o = out + s * n + 32 * w;
    for (int b = 0; b < 32 && 32 * w + b < n; ++b) o[b] = ((word >> b) & 1u) ? (T)1 : (T)-1;
  }
}

// Coloured Rademacher probes (Section 6.1): probe k = d * ncol + c is the
// Rademacher vector of draw d (the stream of k_rng_rademacher for vector d)
// restricted to colour class c of the distance-p lattice colouring
// colour(x, y, z) = ((z mod P) P + (y mod P)) P + (x mod P), P = p + 1.
template <typename T>
__global__ void k_rng_coloured(T* out, int64_t nvec, int64_t n, uint32_t k0, uint32_t k1, int64_t soff, int nx,
                               int ny, int P, int ncol) {
  const int64_t nw = (n + 31) / 32;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < nvec * nw;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx / nw, w = idx - s * nw;
    const int64_t k = s + soff;
    const int64_t d = k / ncol;
    const int c = (int)(k - d * ncol);
    uint32_t ctr[4] = {(uint32_t)(w / 4), (uint32_t)d, 1u, 0u};
    philox4x32_10(ctr, k0, k1);
    const uint32_t word = ctr[w & 3];
    T* o = out + s * n + 32 * w;
    for (int b = 0; b < 32 && 32 * w + b < n; ++b) {
      const int64_t i = 32 * w + b;
      const int64_t row = i / nx;
      const int x = (int)(i - row * nx);
      const int y = (int)(row % ny);
      const int z = (int)(row / ny);
      const int col = ((z % P) * P + (y % P)) * P + (x % P);
      o[b] = col != c ? (T)0 : (((word >> b) & 1u) ? (T)1 : (T)-1);
    }
  }
}

// ||z|| per vector and state reset.  grid (nblk, nvec).
template <typename T>
__global__ void k_init(const T* __restrict__ W, size_t n, VecState* st, Dots<T>* partials, unsigned* counters,
                       const int* m_min) {
  __shared__ Dots<T> red[8];
  __shared__ int s_flag;
  const int s = blockIdx.y;
  const T* z = W + (size_t)s * n;
  Dots<T> d;
  d.zero();
  // only ||z||^2 (the s3 slot) is used: one compensated sum per element
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(T) == 4) Dots<float>::dot2(d.s3, z[i], z[i]);
    else d.s3 = fma(z[i], z[i], d.s3);
  }
  d = block_reduce(d, red);
  const int nblk = gridDim.x;
  if (threadIdx.x == 0) partials[(size_t)s * nblk + blockIdx.x] = d;
  if (!last_block(counters, s, nblk, &s_flag)) return;
  Dots<T> acc;
  acc.zero();
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc.merge(partials[(size_t)s * nblk + b]);
  acc = block_reduce(acc, red);
  if (threadIdx.x == 0) {
    double s1, s2, s3;
    acc.get(s1, s2, s3);
    VecState v = {};
    v.znorm = sqrt(s3);
    v.vscale = v.znorm > 0.0 ? 1.0 / v.znorm : 0.0;
    v.m = 0;
    v.m_min = m_min ? m_min[s] : 0;
    if (!isfinite(v.znorm)) v.status = GMRF_ERR_NUMERIC;
    else if (v.znorm == 0.0) v.status = VS_DONE;
    else v.status = VS_RUNNING;
    st[s] = v;
  }
}

// x[s][i] = scale_s * sum_j V[s][j][i] y[s][j], scale_s = ||z_s|| * extra.
// FP32: y split into float hi + lo, compensated (Neumaier) accumulation.
// The basis is read in its storage type S (T, or bfloat16 for T = float).
// DUAL: in the same pass over V_m also x2[s][i] = ||z_s|| sum_j V[s][j][i]
// y2[s][j] (the CG iterate of the accuracy check), with the same arithmetic;
// x is computed exactly as without it.
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ double to_f(double v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// x_i += vv * y_j in a compensated (sum, error) pair
__device__ __forceinline__ void acc_comp(float vv, float yh, float yl, float& sum, float& comp) {
  const float t = __fmaf_rn(vv, yh, __fmul_rn(vv, yl));
  const float s2 = __fadd_rn(sum, t);
  comp = __fadd_rn(comp, fabsf(sum) >= fabsf(t) ? __fadd_rn(__fsub_rn(sum, s2), t) : __fadd_rn(__fsub_rn(t, s2), sum));
  sum = s2;
}

template <typename T, typename S = T, bool DUAL = false>
__global__ void k_assemble(const S* __restrict__ V, int nslots, size_t n, const VecState* st, const double* y,
                           int y_stride, double extra, T* x, const double* y2, T* x2) {
  extern __shared__ unsigned char smem_raw[];
  const int s = blockIdx.y;
  const VecState v = st[s];
  const int m = v.m;
  T* xo = x + (size_t)s * n;
  T* xo2 = DUAL ? x2 + (size_t)s * n : nullptr;
  const bool bad = !(v.status == VS_DONE || v.status == GMRF_ERR_NOT_CONVERGED);
  if (bad || m == 0) {
    const T fill = (bad && v.status != VS_DONE) ? (T)NAN : (T)0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
      xo[i] = fill;
      if (DUAL) xo2[i] = fill;
    }
    return;
  }
  const double scale = v.znorm * extra;
  const double* ys = y + (size_t)s * y_stride;
  const double* ys2 = DUAL ? y2 + (size_t)s * y_stride : nullptr;
  const S* Vs = V + (size_t)s * nslots * n;
  if (sizeof(T) == 4) {
    float* yh = (float*)smem_raw;
    float* yl = yh + m;
    float* y2h = yl + m;
    float* y2l = y2h + m;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const double yy = ys[j] * scale;
      const float h = (float)yy;
      yh[j] = h;
      yl[j] = (float)(yy - (double)h);
      if (DUAL) {
        const double y2v = ys2[j] * v.znorm;
        const float h2 = (float)y2v;
        y2h[j] = h2;
        y2l[j] = (float)(y2v - (double)h2);
      }
    }
    __syncthreads();
    // the order of the terms is j = 0 .. m-1
    if constexpr (std::is_same<S, __nv_bfloat16>::value) {
      // bfloat16 basis: half the bytes per load, so more loads in flight per
      // thread (the same arithmetic and order per element as below)
      for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float sum = 0.f, comp = 0.f, sum2 = 0.f, comp2 = 0.f;
#pragma unroll 8
        for (int j = 0; j < m; ++j) {
          const float vv = __bfloat162float(Vs[(size_t)j * n + i]);
          acc_comp(vv, yh[j], yl[j], sum, comp);
          if (DUAL) acc_comp(vv, y2h[j], y2l[j], sum2, comp2);
        }
        xo[i] = (T)__fadd_rn(sum, comp);
        if (DUAL) xo2[i] = (T)__fadd_rn(sum2, comp2);
      }
      return;
    }
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
      float sum = 0.f, comp = 0.f, sum2 = 0.f, comp2 = 0.f;
      for (int j = 0; j < m; ++j) {
        const float vv = (float)to_f(Vs[(size_t)j * n + i]);
        acc_comp(vv, yh[j], yl[j], sum, comp);
        if (DUAL) acc_comp(vv, y2h[j], y2l[j], sum2, comp2);
      }
      xo[i] = (T)__fadd_rn(sum, comp);
      if (DUAL) xo2[i] = (T)__fadd_rn(sum2, comp2);
    }
  } else {
    double* yd = (double*)smem_raw;
    double* yd2 = yd + m;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      yd[j] = ys[j] * scale;
      if (DUAL) yd2[j] = ys2[j] * v.znorm;
    }
    __syncthreads();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
      double sum = 0.0, sum2 = 0.0;
      for (int j = 0; j < m; ++j) {
        const double vv = (double)to_f(Vs[(size_t)j * n + i]);
        sum = fma(vv, yd[j], sum);
        if (DUAL) sum2 = fma(vv, yd2[j], sum2);
      }
      xo[i] = (T)sum;
      if (DUAL) xo2[i] = (T)sum2;
    }
  }
}

// ---- the FP32 assembly on paired FP32 instructions (x2_* in common.cuh):
// with two compensated accumulators per element the assembly is
// issue-bound, so k_assemble_pair runs two adjacent elements per thread.
// acc_comp on two elements: t = vv (yh + yl) as FMA(vv, yh, vv * yl), then
// (sum, comp) += t with the exact error of sum + t from TwoSum (Knuth).  The
// error of a floating-point sum is unique, so this gives bitwise the values
// of acc_comp's magnitude-ordered form.
__device__ __forceinline__ void acc_comp2(float2 vv, float2 yh, float2 yl, float2& sum, float2& comp) {
  const float2 t = x2_fma(vv, yh, x2_mul(vv, yl));
  const float2 s2 = x2_add(sum, t);
  const float2 bb = x2_sub(s2, sum);
  const float2 e = x2_add(x2_sub(sum, x2_sub(s2, bb)), x2_sub(t, bb));
  comp = x2_add(comp, e);
  sum = s2;
}

template <typename S>
__device__ __forceinline__ float2 load_pair(const S* p);
template <>
__device__ __forceinline__ float2 load_pair<float>(const float* p) {
  return *reinterpret_cast<const float2*>(p);
}
template <>
__device__ __forceinline__ float2 load_pair<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
}

// k_assemble for FP32 outputs and an even n: elements (2k, 2k + 1) per
// thread, coefficients staged as (yh, yh, yl, yl) per j; the same arithmetic,
// order and results as k_assemble.
template <typename S, bool DUAL>
__global__ void k_assemble_pair(const S* __restrict__ V, int nslots, size_t n, const VecState* st, const double* y,
                                int y_stride, double extra, float* x, const double* y2, float* x2) {
  extern __shared__ float4 c4[];
  const int s = blockIdx.y;
  const VecState v = st[s];
  const int m = v.m;
  float* xo = x + (size_t)s * n;
  float* xo2 = DUAL ? x2 + (size_t)s * n : nullptr;
  const size_t np = n / 2;
  const bool bad = !(v.status == VS_DONE || v.status == GMRF_ERR_NOT_CONVERGED);
  if (bad || m == 0) {
    const float fill = (bad && v.status != VS_DONE) ? NAN : 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
      xo[i] = fill;
      if (DUAL) xo2[i] = fill;
    }
    return;
  }
  const double scale = v.znorm * extra;
  const double* ys = y + (size_t)s * y_stride;
  const double* ys2 = DUAL ? y2 + (size_t)s * y_stride : nullptr;
  float4* c2 = c4 + m;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double yy = ys[j] * scale;
    const float h = (float)yy, l = (float)(yy - (double)h);
    c4[j] = make_float4(h, h, l, l);
    if (DUAL) {
      const double y2v = ys2[j] * v.znorm;
      const float h2 = (float)y2v, l2 = (float)(y2v - (double)h2);
      c2[j] = make_float4(h2, h2, l2, l2);
    }
  }
  __syncthreads();
  const S* Vs = V + (size_t)s * nslots * n;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < np; k += (size_t)gridDim.x * blockDim.x) {
    float2 sum = make_float2(0.f, 0.f), comp = sum, sum2 = sum, comp2 = sum;
    const S* p = Vs + 2 * k;
    int j = 0;
    // four basis loads in flight; the terms are still added in the order j = 0 .. m-1
    for (; j + 4 <= m; j += 4) {
      float2 vv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) vv[u] = load_pair<S>(p + (size_t)(j + u) * n);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 c = c4[j + u];
        acc_comp2(vv[u], make_float2(c.x, c.y), make_float2(c.z, c.w), sum, comp);
        if (DUAL) {
          const float4 d = c2[j + u];
          acc_comp2(vv[u], make_float2(d.x, d.y), make_float2(d.z, d.w), sum2, comp2);
        }
      }
    }
    for (; j < m; ++j) {
      const float2 vv = load_pair<S>(p + (size_t)j * n);
      const float4 c = c4[j];
      acc_comp2(vv, make_float2(c.x, c.y), make_float2(c.z, c.w), sum, comp);
      if (DUAL) {
        const float4 d = c2[j];
        acc_comp2(vv, make_float2(d.x, d.y), make_float2(d.z, d.w), sum2, comp2);
      }
    }
    reinterpret_cast<float2*>(xo)[k] = x2_add(sum, comp);
    if (DUAL) reinterpret_cast<float2*>(xo2)[k] = x2_add(sum2, comp2);
  }
}

// Two-pass sampling: x += scale_s y_j v_j for the basis vector v_j the step
// just formed (j = acc[s] if the step ran for vector s), with the arithmetic
// of k_assemble per element; with X2 also x2 += ||z_s|| y2_j v_j (the dual
// output of k_assemble).  acc[s] advances in the vector's last block, after
// every block has read it.
__device__ __forceinline__ void acc_pair(float vv, double yy, float* xh, float* xl, size_t i) {
  const float h = (float)yy;
  const float l = (float)(yy - (double)h);
  const float t = __fmaf_rn(vv, h, __fmul_rn(vv, l));
  const float sum = xh[i];
  const float s2 = __fadd_rn(sum, t);
  xl[i] = __fadd_rn(xl[i], fabsf(sum) >= fabsf(t) ? __fadd_rn(__fsub_rn(sum, s2), t) : __fadd_rn(__fsub_rn(t, s2), sum));
  xh[i] = s2;
}

template <typename T>
__global__ void k_accumulate(const T* __restrict__ V, int nslots, size_t n, const VecState* st, const double* y,
                             int m_max, double extra, void* X, int* acc, unsigned* counters, const double* y2,
                             void* X2) {
  __shared__ int s_flag;
  const int s = blockIdx.y;
  const VecState v = st[s];
  const int a = acc[s];
  const bool work = a < v.m;
  if (work) {
    const T* vj = V + ((size_t)s * nslots + (size_t)(a % nslots)) * n;
    const double yy = y[(size_t)s * m_max + a] * (v.znorm * extra);
    const double yy2 = X2 ? y2[(size_t)s * m_max + a] * v.znorm : 0.0;
    if (sizeof(T) == 4) {
      float* xh = (float*)X + (size_t)s * 2 * n;
      float* xl = xh + n;
      float* x2h = X2 ? (float*)X2 + (size_t)s * 2 * n : nullptr;
      float* x2l = x2h + n;
      for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float vv = (float)vj[i];
        acc_pair(vv, yy, xh, xl, i);
        if (X2) acc_pair(vv, yy2, x2h, x2l, i);
      }
    } else {
      double* xd = (double*)X + (size_t)s * n;
      double* xd2 = X2 ? (double*)X2 + (size_t)s * n : nullptr;
      for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        xd[i] = fma((double)vj[i], yy, xd[i]);
        if (X2) xd2[i] = fma((double)vj[i], yy2, xd2[i]);
      }
    }
  }
  if (last_block(counters, s, gridDim.x, &s_flag) && threadIdx.x == 0 && work) acc[s] = a + 1;
}

// x = sum + compensation (FP32) or the FP64 sum; failures filled as k_assemble does.
template <typename T>
__global__ void k_accumulate_finish(const void* X, size_t n, const VecState* st, T* x) {
  const int s = blockIdx.y;
  const VecState v = st[s];
  T* xo = x + (size_t)s * n;
  const bool bad = !(v.status == VS_DONE || v.status == GMRF_ERR_NOT_CONVERGED);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    if (bad || v.m == 0) {
      xo[i] = (bad && v.status != VS_DONE) ? (T)NAN : (T)0;
    } else if (sizeof(T) == 4) {
      const float* xh = (const float*)X + (size_t)s * 2 * n;
      xo[i] = (T)__fadd_rn(xh[i], xh[n + i]);
    } else {
      xo[i] = (T)((const double*)X)[(size_t)s * n + i];
    }
  }
}

// Condition of the device-side Lanczos loop (a CUDA graph WHILE node): the
// body runs again while some vector is still iterating and the iteration count
// is below `limit` (a bound the loop never needs: every vector stops by m_max).
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const VecState* st, int nvec, int* ctr, int limit) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < nvec; s += blockDim.x)
    if (st[s].status == VS_RUNNING) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int n = *ctr + 1;
    *ctr = n;
    cudaGraphSetConditional(h, (any && n < limit) ? 1u : 0u);
  }
}

// r = z - r in place (the residual from A u in r), elementwise in the type of r.
template <typename Z, typename R>
__global__ void k_resid_form(const Z* __restrict__ z, R* r, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    r[i] = (R)((double)z[i] - (double)r[i]);
}

// Partial sums of r.r, r.t, t.t per vector, grid (nblk, nvec); the block
// tree and the order of the partials depend only on n.  FP64 vectors sum in
// FP64; FP32 vectors sum in Dot2 form (exact products, pair sums) on the FP32
// pipe, each thread's sums finished in FP64.
template <typename R>
__global__ void k_dots3_partial(const R* __restrict__ r, const R* __restrict__ t, size_t n, Dots<double>* part) {
  __shared__ Dots<double> red[8];
  const int s = blockIdx.y;
  const R* rs = r + (size_t)s * n;
  const R* ts = t + (size_t)s * n;
  Dots<double> d;
  d.zero();
  if constexpr (sizeof(R) == 4) {
    df rr = {0.f, 0.f}, rt = {0.f, 0.f}, tt = {0.f, 0.f};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
      const float a = rs[i], b = ts[i];
      Dots<float>::dot2(rr, a, a);
      Dots<float>::dot2(rt, a, b);
      Dots<float>::dot2(tt, b, b);
    }
    d.s1 = df_to_double(rr);
    d.s2 = df_to_double(rt);
    d.s3 = df_to_double(tt);
  } else {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
      const double a = (double)rs[i], b = (double)ts[i];
      d.s1 = fma(a, a, d.s1);
      d.s2 = fma(a, b, d.s2);
      d.s3 = fma(b, b, d.s3);
    }
  }
  d = block_reduce(d, red);
  if (threadIdx.x == 0) part[(size_t)s * gridDim.x + blockIdx.x] = d;
}

__global__ void k_dots3_final(const Dots<double>* part, int nblk, double* out) {
  __shared__ Dots<double> red[8];
  const int s = blockIdx.x;
  Dots<double> d;
  d.zero();
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) d.merge(part[(size_t)s * nblk + b]);
  d = block_reduce(d, red);
  if (threadIdx.x == 0) {
    out[3 * s] = d.s1;
    out[3 * s + 1] = d.s2;
    out[3 * s + 2] = d.s3;
  }
}

template <typename T>
__global__ void k_scale(T* x, size_t count, T a) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    x[i] *= a;
}

// Coefficient-field checks and mean log: counts of negative / non-finite
// entries and of zeros, and sum of log kappa^2 over the positive entries
// (compensated FP32).  Each block reduces a contiguous chunk into part[b];
// k_field_final sums the parts in a fixed order.
constexpr int kFieldBlocks = 256;
__global__ void k_field_stats(const float* k, size_t n, Dots<float>* part) {
  __shared__ Dots<float> red[8];
  Dots<float> d;  // s1 = sum log, s2 = #bad, s3 = #zero (as compensated sums)
  d.zero();
  const size_t per = (n + gridDim.x - 1) / gridDim.x;
  const size_t lo = per * blockIdx.x, hi = min(n, lo + per);
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const float v = k[i];
    if (!(v >= 0.f) || !isfinite(v)) d.s2 = df_add(d.s2, df{1.f, 0.f});
    else if (v == 0.f) d.s3 = df_add(d.s3, df{1.f, 0.f});
    else d.s1 = df_add(d.s1, df{logf(v), 0.f});
  }
  d = block_reduce(d, red);
  if (threadIdx.x == 0) part[blockIdx.x] = d;
}
__global__ void k_field_final(const Dots<float>* part, int np, double* out4) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Dots<float> d;
  d.zero();
  for (int b = 0; b < np; ++b) d.merge(part[b]);
  double a, b2, c;
  d.get(a, b2, c);
  out4[0] = b2;
  out4[1] = c;
  out4[2] = a;
  out4[3] = 0.0;
}

int grid_for(size_t work, int threads) {
  size_t b = (work + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_rng(int kind, bool fp64, int64_t nvec, int64_t n, uint64_t seed, int64_t soff, void* out,
                       cudaStream_t s) {
  const uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  if (kind == 0) {
    const int grid = grid_for((size_t)nvec * ((n + 3) / 4), 256);
    if (fp64) k_rng_gauss<double><<<grid, 256, 0, s>>>((double*)out, nvec, n, k0, k1, soff);
    else k_rng_gauss<float><<<grid, 256, 0, s>>>((float*)out, nvec, n, k0, k1, soff);
  } else if (kind == 1) {
    const int grid = grid_for((size_t)nvec * ((n + 31) / 32), 256);
    if (fp64) k_rng_rademacher<double><<<grid, 256, 0, s>>>((double*)out, nvec, n, k0, k1, soff);
    else k_rng_rademacher<float><<<grid, 256, 0, s>>>((float*)out, nvec, n, k0, k1, soff);
  } else {
    const int grid = grid_for((size_t)nvec * ((n + 3) / 4), 256);
    k_rng_words<<<grid, 256, 0, s>>>((uint32_t*)out, nvec, n, k0, k1, soff);
  }
  return cudaGetLastError();
}

cudaError_t launch_rng_coloured(bool fp64, int64_t nvec, int64_t n, uint64_t seed, int64_t soff, int nx, int ny,
                                int P, int ncol, void* out, cudaStream_t s) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const int grid = grid_for((size_t)nvec * ((n + 31) / 32), 256);
  if (fp64) k_rng_coloured<double><<<grid, 256, 0, s>>>((double*)out, nvec, n, k0, k1, soff, nx, ny, P, ncol);
  else k_rng_coloured<float><<<grid, 256, 0, s>>>((float*)out, nvec, n, k0, k1, soff, nx, ny, P, ncol);
  return cudaGetLastError();
}

cudaError_t launch_field_stats(const float* k, size_t n, double* out4, cudaStream_t s) {
  Dots<float>* part = reinterpret_cast<Dots<float>*>(out4 + 4);
  k_field_stats<<<kFieldBlocks, 256, 0, s>>>(k, n, part);
  k_field_final<<<1, 32, 0, s>>>(part, kFieldBlocks, out4);
  return cudaGetLastError();
}

cudaError_t launch_lanczos_init(bool fp64, size_t n, const LanczosBufs& b, cudaStream_t s) {
  int nblk = (int)((n + 255) / 256);
  if (nblk > 256) nblk = 256;
  dim3 grd(nblk, b.nvec);
  if (fp64)
    k_init<double><<<grd, 256, 0, s>>>((const double*)b.W[0], n, b.st, (Dots<double>*)b.partials, b.counters,
                                       b.m_min);
  else
    k_init<float><<<grd, 256, 0, s>>>((const float*)b.W[0], n, b.st, (Dots<float>*)b.partials, b.counters,
                                      b.m_min);
  return cudaGetLastError();
}

template <typename T, typename S, bool DUAL>
static void assemble_one(const S* V, int nslots, size_t n, const LanczosBufs& b, const double* y, int y_stride,
                         double extra, T* x, const double* y2, T* x2, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    // even n (8-byte aligned pairs in every basis slot) and staged coefficients within 200 KB
    const size_t smp = (size_t)b.m_max * sizeof(float4) * (DUAL ? 2 : 1);
    if (n % 2 == 0 && smp <= 200 * 1024 && ((uintptr_t)x & 7) == 0 && (!DUAL || ((uintptr_t)x2 & 7) == 0)) {
      int nb = (int)((n / 2 + 255) / 256);
      if (nb > 2048) nb = 2048;
      if (smp > 48 * 1024)
        cudaFuncSetAttribute(k_assemble_pair<S, DUAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
      k_assemble_pair<S, DUAL><<<dim3(nb, b.nvec), 256, smp, s>>>(V, nslots, n, b.st, y, y_stride, extra, x, y2, x2);
      return;
    }
  }
  int nblk = (int)((n + 255) / 256);
  if (nblk > 2048) nblk = 2048;
  dim3 grd(nblk, b.nvec);
  const size_t sm = (size_t)b.m_max * 8 * (DUAL ? 2 : 1);
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_assemble<T, S, DUAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_assemble<T, S, DUAL><<<grd, 256, sm, s>>>(V, nslots, n, b.st, y, y_stride, extra, x, y2, x2);
}

template <bool DUAL>
static cudaError_t assemble_dispatch(bool fp64, size_t n, const LanczosBufs& b, const double* y, int y_stride,
                                     double extra_scale, void* x, const double* y2, void* x2, cudaStream_t s) {
  if (fp64)
    assemble_one<double, double, DUAL>((const double*)b.V, b.nslots, n, b, y, y_stride, extra_scale, (double*)x, y2,
                                       (double*)x2, s);
  else if (b.Vb)  // bfloat16 basis copy: m_max + 1 slots per vector
    assemble_one<float, __nv_bfloat16, DUAL>(b.Vb, b.m_max + 1, n, b, y, y_stride, extra_scale, (float*)x, y2,
                                             (float*)x2, s);
  else
    assemble_one<float, float, DUAL>((const float*)b.V, b.nslots, n, b, y, y_stride, extra_scale, (float*)x, y2,
                                     (float*)x2, s);
  return cudaGetLastError();
}

cudaError_t launch_assemble(bool fp64, size_t n, const LanczosBufs& b, const double* y, int y_stride,
                            double extra_scale, void* x, cudaStream_t s) {
  return assemble_dispatch<false>(fp64, n, b, y, y_stride, extra_scale, x, nullptr, nullptr, s);
}

cudaError_t launch_assemble_dual(bool fp64, size_t n, const LanczosBufs& b, const double* y, int y_stride,
                                 double extra_scale, void* x, const double* y2, void* x2, cudaStream_t s) {
  return assemble_dispatch<true>(fp64, n, b, y, y_stride, extra_scale, x, y2, x2, s);
}

cudaError_t launch_accumulate(bool fp64, size_t n, const LanczosBufs& b, cudaStream_t s) {
  int nblk = (int)((n + 255) / 256);
  if (nblk > 2048) nblk = 2048;
  dim3 grd(nblk, b.nvec);
  if (fp64)
    k_accumulate<double><<<grd, 256, 0, s>>>((const double*)b.V, b.nslots, n, b.st, b.y, b.m_max, b.xscale, b.Xacc,
                                             b.acc, b.counters, b.y2, b.Xacc2);
  else
    k_accumulate<float><<<grd, 256, 0, s>>>((const float*)b.V, b.nslots, n, b.st, b.y, b.m_max, b.xscale, b.Xacc,
                                            b.acc, b.counters, b.y2, b.Xacc2);
  return cudaGetLastError();
}

cudaError_t launch_accumulate_finish(bool fp64, size_t n, const LanczosBufs& b, const void* X, void* x,
                                     cudaStream_t s) {
  int nblk = (int)((n + 255) / 256);
  if (nblk > 2048) nblk = 2048;
  dim3 grd(nblk, b.nvec);
  if (fp64) k_accumulate_finish<double><<<grd, 256, 0, s>>>(X, n, b.st, (double*)x);
  else k_accumulate_finish<float><<<grd, 256, 0, s>>>(X, n, b.st, (float*)x);
  return cudaGetLastError();
}

cudaError_t launch_resid_form(bool z64, const void* z, bool r64, void* r, size_t count, cudaStream_t s) {
  const int grid = grid_for(count, 256);
  if (z64 && r64) k_resid_form<double, double><<<grid, 256, 0, s>>>((const double*)z, (double*)r, count);
  else if (!z64 && r64) k_resid_form<float, double><<<grid, 256, 0, s>>>((const float*)z, (double*)r, count);
  else if (!z64 && !r64) k_resid_form<float, float><<<grid, 256, 0, s>>>((const float*)z, (float*)r, count);
  else k_resid_form<double, float><<<grid, 256, 0, s>>>((const double*)z, (float*)r, count);
  return cudaGetLastError();
}

cudaError_t launch_dots3(bool r64, const void* r, const void* t, size_t n, int nvec, void* part, double* out,
                         cudaStream_t s) {
  dim3 grd(kResidBlocks, nvec);
  if (r64) k_dots3_partial<double><<<grd, 256, 0, s>>>((const double*)r, (const double*)t, n, (Dots<double>*)part);
  else k_dots3_partial<float><<<grd, 256, 0, s>>>((const float*)r, (const float*)t, n, (Dots<double>*)part);
  k_dots3_final<<<nvec, 256, 0, s>>>((const Dots<double>*)part, kResidBlocks, out);
  return cudaGetLastError();
}

cudaError_t launch_dots3_final(const void* part, int nvec, double* out, cudaStream_t s) {
  k_dots3_final<<<nvec, 256, 0, s>>>((const Dots<double>*)part, kResidBlocks, out);
  return cudaGetLastError();
}

const void* loop_cond_kernel() { return (const void*)k_loop_cond; }

cudaError_t launch_loop_cond(cudaGraphConditionalHandle h, const VecState* st, int nvec, int* ctr, int limit,
                             cudaStream_t s) {
  k_loop_cond<<<1, 256, 0, s>>>(h, st, nvec, ctr, limit);
  return cudaGetLastError();
}

cudaError_t launch_scale(bool fp64, void* x, size_t count, double a, cudaStream_t s) {
  const int grid = grid_for(count, 256);
  if (fp64) k_scale<double><<<grid, 256, 0, s>>>((double*)x, count, a);
  else k_scale<float><<<grid, 256, 0, s>>>((float*)x, count, (float)a);
  return cudaGetLastError();
}

}  // namespace gmrf
