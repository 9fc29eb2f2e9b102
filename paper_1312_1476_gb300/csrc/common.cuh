// common.cuh -- device helpers shared by the Lanczos kernels.
//
// * compensated FP32 ("double-float") sums for the dot products of the
//   Lanczos recurrence: GB300's FP64 rate is a small fraction of its FP32
//   rate, so every per-element and per-warp reduction of the FP32 path runs
//   on pairs of floats and only the final per-vector sums are FP64;
// * the per-vector iteration state and the end-of-step logic shared by the
//   stencil and the preconditioned step kernels: alpha_j, beta_j
//   (Algorithm 1), the LDL^T recurrence of T_m, and the stopping rule built
//   on the a-posteriori bound of Theorem 1 (eq. krylov_bound);
// * Philox-4x32-10 (Salmon et al., SC'11) for z and the Rademacher probes.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gmrf.h"

namespace gmrf {

// ----------------------------------------------------------------- status codes
enum : int { VS_RUNNING = 1, VS_DONE = 0 };  // other values: negative gmrf error codes

// --------------------------------------------------------- compensated float sums
struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}
// exact product a*b as an unevaluated pair
__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ df df_shfl_down(df v, int off) {
  return {__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off)};
}
__device__ __forceinline__ double df_to_double(df v) { return (double)v.hi + (double)v.lo; }

// Accumulator of the three dot products of one Lanczos step:
//   s1 = v_j . q, s2 = q . q, s3 = v_j . v_j  (all for one vector).
template <typename T>
struct Dots;

template <>
struct Dots<float> {
  df s1, s2, s3;
  __device__ __forceinline__ void zero() { s1 = s2 = s3 = {0.f, 0.f}; }
  __device__ __forceinline__ void add(float v, float q) {
    s1 = df_add(s1, two_prod(v, q));
    s2 = df_add(s2, two_prod(q, q));
    s3 = df_add(s3, two_prod(v, v));
  }
  // Dot2 of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 2005): exact product
  // (TwoProd), TwoSum into hi, the rounding errors summed into lo without
  // renormalising; as accurate as summing in twice the working precision.
  __device__ __forceinline__ static void dot2(df& a, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float pe = __fmaf_rn(x, y, -p);
    const df t = two_sum(a.hi, p);
    a.hi = t.hi;
    a.lo = __fadd_rn(a.lo, __fadd_rn(t.lo, pe));
  }
  __device__ __forceinline__ void add_dot2(float v, float q) {
    dot2(s1, v, q);
    dot2(s2, q, q);
    dot2(s3, v, v);
  }
  __device__ __forceinline__ void merge(const Dots& o) {
    s1 = df_add(s1, o.s1);
    s2 = df_add(s2, o.s2);
    s3 = df_add(s3, o.s3);
  }
  __device__ __forceinline__ Dots shfl_down(int off) const {
    Dots r;
    r.s1 = df_shfl_down(s1, off);
    r.s2 = df_shfl_down(s2, off);
    r.s3 = df_shfl_down(s3, off);
    return r;
  }
  __device__ __forceinline__ void get(double& a, double& b, double& c) const {
    a = df_to_double(s1);
    b = df_to_double(s2);
    c = df_to_double(s3);
  }
};

// ---- paired FP32 arithmetic (Blackwell f32x2): one issue slot for two
// lane-wise FP32 operations, each with the IEEE round-to-nearest result of
// the scalar operation.
__device__ __forceinline__ unsigned long long x2_pk(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 x2_upk(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 x2_add(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x2_pk(a)), "l"(x2_pk(b)));
  return x2_upk(d);
}
__device__ __forceinline__ float2 x2_sub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x2_pk(a)), "l"(x2_pk(b)));
  return x2_upk(d);
}
__device__ __forceinline__ float2 x2_mul(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x2_pk(a)), "l"(x2_pk(b)));
  return x2_upk(d);
}
__device__ __forceinline__ float2 x2_fma(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(x2_pk(a)), "l"(x2_pk(b)), "l"(x2_pk(c)));
  return x2_upk(d);
}

// The three sums of Dots<float> in Dot2 form over pairs of elements, on the
// paired instructions: two accumulators per sum (the pair's halves), merged
// into a Dots<float> at the end.  Per pair and sum: the product and its
// exact error (TwoProd by FMA), TwoSum into hi, the errors summed into lo.
struct Dot2x2 {
  float2 h1, l1, h2, l2, h3, l3;  // v.q, q.q, v.v
  __device__ __forceinline__ void zero() { h1 = l1 = h2 = l2 = h3 = l3 = make_float2(0.f, 0.f); }
  // (h, l) += x * y; xn = -x
  __device__ __forceinline__ static void acc(float2& h, float2& l, float2 x, float2 xn, float2 y) {
    const float2 p = x2_mul(x, y);
    const float2 pen = x2_fma(xn, y, p);  // p - x y = -(rounding error of p), exact
    const float2 s = x2_add(h, p);
    const float2 bb = x2_sub(s, h);
    const float2 e = x2_add(x2_sub(h, x2_sub(s, bb)), x2_sub(p, bb));
    l = x2_add(l, x2_sub(e, pen));
    h = s;
  }
  __device__ __forceinline__ void add(float2 v, float2 q) {
    const float2 vn = make_float2(-v.x, -v.y), qn = make_float2(-q.x, -q.y);
    acc(h1, l1, v, vn, q);
    acc(h2, l2, q, qn, q);
    acc(h3, l3, v, vn, v);
  }
  __device__ __forceinline__ Dots<float> merged() const {
    Dots<float> d;
    d.s1 = df_add({h1.x, l1.x}, {h1.y, l1.y});
    d.s2 = df_add({h2.x, l2.x}, {h2.y, l2.y});
    d.s3 = df_add({h3.x, l3.x}, {h3.y, l3.y});
    return d;
  }
};

template <>
struct Dots<double> {
  double s1, s2, s3;
  __device__ __forceinline__ void zero() { s1 = s2 = s3 = 0.0; }
  __device__ __forceinline__ void add(double v, double q) {
    s1 = fma(v, q, s1);
    s2 = fma(q, q, s2);
    s3 = fma(v, v, s3);
  }
  __device__ __forceinline__ void merge(const Dots& o) {
    s1 += o.s1;
    s2 += o.s2;
    s3 += o.s3;
  }
  __device__ __forceinline__ Dots shfl_down(int off) const {
    Dots r;
    r.s1 = __shfl_down_sync(0xffffffffu, s1, off);
    r.s2 = __shfl_down_sync(0xffffffffu, s2, off);
    r.s3 = __shfl_down_sync(0xffffffffu, s3, off);
    return r;
  }
  __device__ __forceinline__ void get(double& a, double& b, double& c) const {
    a = s1;
    b = s2;
    c = s3;
  }
};

// Fixed-order block reduction (result valid in thread 0).  `scratch` must
// hold blockDim/32 entries.  The tree depends only on the block shape.
template <typename A>
__device__ __forceinline__ A block_reduce(A v, A* scratch) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nwarps = (blockDim.x * blockDim.y * blockDim.z) >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v.merge(v.shfl_down(off));
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  if (warp == 0) {
    A w;
    if (lane < nwarps) w = scratch[lane];
    else w.zero();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) w.merge(w.shfl_down(off));
    v = w;
  }
  __syncthreads();
  return v;
}

// ------------------------------------------------------------- iteration state
// One record per vector (sample z or probe v) of a Lanczos batch.
struct VecState {
  int status;     // VS_RUNNING, VS_DONE or a negative gmrf error code
  int m;          // completed steps = number of alpha values
  int m_min;      // the stopping rule may end the iteration only once m >= m_min (0: any m)
  int pad_;
  double znorm;   // ||z||
  double d_prev;  // 1 / d_{m-1}, the reciprocal of the LDL^T pivot d_{m-1} of T_m
  double u_prev;  // u_{m-1} = (L^{-1} e_1)_{m-1}
  double energy;  // e_1^T T_m^{-1} e_1 = sum_i u_i^2 / d_i
  double theta;   // smallest Ritz value theta_min (upper estimate)
  double err_est; // relative Theorem 1 estimate at m
  double amax;    // max |alpha_i|
  double bmax;    // max beta_i
  double beta_last;  // beta_{m-1}
  double vscale;     // 1 / ||z|| at m = 0, then 1 / beta_{m-1}: the scale of v_m (one division per step)
};

// Loop-invariant parameters of the Lanczos steps.  The step index j (the
// basis vector v_j formed in the step, 0-based) is not a parameter: every
// step kernel reads it from its vector's state (VecState.m = completed
// steps), so one captured CUDA graph of c steps can be replayed.
struct StepParams {
  int m_max;      // largest subspace size
  int nslots;     // ring size of the stored basis (m_max + 1, or 2 when V_m is not kept)
  int solve;      // 1: the iteration solves A u = z (stopping rule on the CG residual), 0: sampling / quadrature
  double tol;     // stopping tolerance on the relative estimate
  double bd_tol;  // breakdown threshold relative to ||T_m||
  // bfloat16 copy of the basis for the assembly only ([nvec][m_max + 1][n]),
  // or null.  When set, the FP32 ring above holds just v_{j-1}, v_j (nslots 2),
  // so the recurrence itself is the same as with an FP32 basis.
  __nv_bfloat16* vb;
};

// Stores of v_j into the bfloat16 basis copy (round to nearest even).
__device__ __forceinline__ __nv_bfloat16* vb_at(const StepParams& P, int s, int j, size_t n, size_t i) {
  return P.vb + ((size_t)s * (size_t)(P.m_max + 1) + (size_t)j) * n + i;
}
__device__ __forceinline__ void vb_store1(__nv_bfloat16* p, float a) { *p = __float2bfloat16_rn(a); }
__device__ __forceinline__ void vb_store2(__nv_bfloat16* p, float a, float b) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
}
__device__ __forceinline__ void vb_store4(__nv_bfloat16* p, float a, float b, float c, float d) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  uint2 u;
  u.x = *reinterpret_cast<const unsigned*>(&lo);
  u.y = *reinterpret_cast<const unsigned*>(&hi);
  *reinterpret_cast<uint2*>(p) = u;
}

// Count of eigenvalues of T_m below sigma (Sturm sequence of the LDL^T pivots
// of T_m - sigma I), in FP32 on float copies of alpha and beta^2.
__device__ __forceinline__ int sturm_count(const float* __restrict__ af, const float* __restrict__ b2f, int m,
                                           float sigma) {
  int cnt = 0;
  float d = 1.f;
  for (int i = 0; i < m; ++i) {
    float a = af[i] - sigma;
    d = (i == 0) ? a : a - __fdividef(b2f[i - 1], d);
    if (fabsf(d) < 1e-30f) d = -1e-30f;
    cnt += (d < 0.f);
  }
  return cnt;
}

// Smallest eigenvalue of T_m by multisection over the block's threads on a
// geometric grid below `hi` (an upper bound).  All threads of the block call
// it; the result is returned to every thread.  Relative resolution after two
// rounds with 256+ threads is ~1e-4, ample for the bound's lambda_min^{-1/2}.
__device__ __noinline__ static double smallest_ritz(const float* af, const float* b2f, int m, double hi_in, int* s_int,
                                float* s_flt) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  float hi = (float)(hi_in * 1.0001) + 1e-30f;
  float lo = hi * 1e-8f;
  for (int round = 0; round < 8; ++round) {
    // points p_t = lo * (hi/lo)^((t+1)/nt), t = 0..nt-1 ; p_{nt-1} = hi
    float lr = __logf(hi / lo);
    float p = lo * __expf(lr * (float)(tid + 1) / (float)nt);
    if (tid == nt - 1) p = hi;
    int c = sturm_count(af, b2f, m, p);
    if (tid == 0) s_int[0] = nt;  // first index with count >= 1
    __syncthreads();
    if (c >= 1) atomicMin(&s_int[0], tid);
    int c_lo = (tid == 0) ? sturm_count(af, b2f, m, lo) : 0;
    __syncthreads();
    if (tid == 0) {
      int t = s_int[0];
      float nlo = lo, nhi = hi;
      int again = 0;
      if (c_lo >= 1) {          // theta_min below lo: move the window down
        nhi = lo;
        nlo = lo * 1e-8f;
        again = (nlo > 1e-35f) ? 2 : 3;
      } else if (t == nt) {     // hi was not an upper bound: widen up
        nlo = hi;
        nhi = hi * 1e4f;
        again = 2;
      } else {
        nhi = lo * __expf(lr * (float)(t + 1) / (float)nt);
        if (t == nt - 1) nhi = hi;
        nlo = (t == 0) ? lo : lo * __expf(lr * (float)t / (float)nt);
        again = (round == 0) ? 1 : 0;  // two refinement rounds
      }
      s_flt[0] = nlo;
      s_flt[1] = nhi;
      s_int[1] = again;
    }
    __syncthreads();
    lo = s_flt[0];
    hi = s_flt[1];
    int again = s_int[1];
    __syncthreads();
    if (again == 0 || again == 3) break;
  }
  return (double)hi;
}

// End of a Lanczos step for vector s, run by the last block of that vector
// (every thread of the block calls it).  Sums the per-block partial dot
// products in a fixed order, forms alpha_j and beta_j, advances the LDL^T
// recurrence of T_m and applies the stopping rule:
//   est = theta_min^{-1/2} ||r_m|| / ||x_m||,
//   ||r_m|| / ||z|| = beta_{m-1} |u_{m-1} / d_{m-1}|,  ||x_m|| / ||z|| = sqrt(e_1^T T_m^{-1} e_1).
// beta_j^2 comes from the three sums (one pass over the vectors), or, when
// b2_direct >= 0, is b2_direct = ||q_j - alpha_j v_j||^2 summed by a caller
// that holds both vectors (a second pass; exact also when beta_j << ||q_j||,
// where the one-pass form cancels to rounding noise).
template <typename T>
__device__ static void finish_step(const StepParams& P, int j, int s, const Dots<T>* __restrict__ partials, int nblk,
                            VecState* __restrict__ st, double* __restrict__ alpha, double* __restrict__ beta,
                            float* __restrict__ alpha_f, float* __restrict__ beta2_f, Dots<T>* red_scratch,
                            int* s_int, float* s_flt, double b2_direct = -1.0) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  Dots<T> acc;
  acc.zero();
  for (int b = tid; b < nblk; b += nt) acc.merge(partials[(size_t)s * nblk + b]);
  acc = block_reduce(acc, red_scratch);
  __shared__ int s_need_theta;
  __shared__ double s_theta_hi, s_pfac;
  const size_t mo = (size_t)s * P.m_max;
  if (tid == 0) {
    double s1, s2, s3;
    acc.get(s1, s2, s3);
    VecState v = st[s];
    double a = s1;
    double b2 = b2_direct >= 0.0 ? b2_direct : s2 - 2.0 * a * s1 + a * a * s3;
    double b = b2 > 0.0 ? sqrt(b2) : 0.0;
    alpha[mo + j] = a;
    beta[mo + j] = b;
    alpha_f[mo + j] = (float)a;
    beta2_f[mo + j] = (float)(b * b);
    // LDL^T of T_m: d_0 = a_0, d_j = a_j - b_{j-1}^2 / d_{j-1}; u_0 = 1, u_j = -(b_{j-1}/d_{j-1}) u_{j-1}.
    // The state keeps 1 / d_{j-1}, so that the step's FP64 chain holds one
    // division (1 / d_j) and one for 1 / beta_j: GB300's FP64 divisions and
    // square roots are slow, and this tail runs between every two steps.
    double d, u;
    if (j == 0) {
      d = a;
      u = 1.0;
      v.energy = 0.0;
      v.amax = 0.0;
      v.bmax = 0.0;
      v.theta = a;
    } else {
      const double r = v.beta_last * v.d_prev;  // b_{j-1} / d_{j-1}
      d = a - v.beta_last * r;
      u = -r * v.u_prev;
    }
    v.m = j + 1;
    v.beta_last = b;
    v.vscale = b > 0.0 ? 1.0 / b : 0.0;
    v.amax = fmax(v.amax, fabs(a));
    v.bmax = fmax(v.bmax, b);
    int need = 0;
    if (!(isfinite(a) && isfinite(b) && isfinite(d))) {
      v.status = GMRF_ERR_NUMERIC;
    } else if (d <= 0.0 || a <= 0.0) {
      v.status = GMRF_ERR_NOT_SPD;
    } else {
      const double dinv = 1.0 / d;
      v.energy += u * u * dinv;
      v.d_prev = dinv;
      v.u_prev = u;
      const double rres = b * fabs(u) * dinv;          // ||r_m|| / ||z||
      double pfac = rres * rsqrt(v.energy);             // ||r_m|| / ||x_m||
      if (b <= P.bd_tol * (v.amax + v.bmax)) {
        v.status = VS_DONE;  // invariant Krylov subspace: x_m is exact
        v.err_est = 0.0;
        need = !P.solve;     // theta still wanted for the T_m function of a sample
      } else if (P.solve) {
        // linear solve: x_m = ||z|| V_m T_m^{-1} e_1 is the CG iterate, with
        // relative residual ||r_m|| / ||z|| = beta_m |e_m^T T_m^{-1} e_1|
        v.err_est = rres;
        if (rres <= P.tol) v.status = VS_DONE;
        else if (j + 1 >= P.m_max) v.status = GMRF_ERR_NOT_CONVERGED;
      } else {
        double est_lb = pfac * rsqrt(v.theta);  // theta >= theta_min(T_m): a lower bound of est
        v.err_est = est_lb;
        if (est_lb <= P.tol || j + 1 >= P.m_max) need = 1;
      }
      s_pfac = pfac;
    }
    s_need_theta = need;
    s_theta_hi = v.theta;
    st[s] = v;
  }
  __syncthreads();
  if (s_need_theta) {
    double th = smallest_ritz(alpha_f + mo, beta2_f + mo, j + 1, s_theta_hi, s_int, s_flt);
    if (tid == 0) {
      VecState v = st[s];
      v.theta = th;
      if (v.status == VS_RUNNING) {
        double est = s_pfac * rsqrt(th);
        v.err_est = est;
        if (est <= P.tol && j + 1 >= v.m_min) v.status = VS_DONE;
        else if (j + 1 >= P.m_max) v.status = GMRF_ERR_NOT_CONVERGED;
      }
      st[s] = v;
    }
  }
}

// Last-block election: returns true in every thread of the block that is the
// last of the `nblk` blocks of vector s to finish (counter reset by it).
__device__ __forceinline__ bool last_block(unsigned* counter, int s, int nblk, int* s_flag) {
  __threadfence();
  __syncthreads();
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  if (tid == 0) {
    unsigned t = atomicAdd(&counter[s], 1u);
    int last = (t == (unsigned)(nblk - 1));
    if (last) counter[s] = 0u;
    *s_flag = last;
  }
  __syncthreads();
  if (*s_flag) __threadfence();
  return *s_flag != 0;
}

// ------------------------------------------------------------------- Philox
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t lo0 = 0xD2511F53u * c[0];
    uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
    uint32_t lo1 = 0xCD9E8D57u * c[2];
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

}  // namespace gmrf
