// tridiag.cu -- functions of the small Lanczos matrix T_m, in FP64.
//
// Sample (Algorithm 1, last step): y = T_m^{-1/2} e_1.  The algorithm's
// caption notes that the square root of T_m may be replaced by a rational
// approximation; this library uses one.  From
//   t^{-1/2} = (2/pi) int_0^inf ds / (t + s^2) = (2/pi) int_R e^u / (t + e^{2u}) du,
// whose integrand is sech(u - log(t)/2) / (2 sqrt t), the trapezoid rule with
// step h on [u_lo, u_hi] gives
//   T^{-1/2} e_1 ~= sum_k (2h/pi) e^{u_k} (T + e^{2u_k} I)^{-1} e_1,
// a sum of shifted SPD tridiagonal solves (Thomas algorithm, one pole per
// thread).  Discretisation error ~ 4 exp(-pi^2 / h) and truncation error
// ~ (2/pi) exp(-pad) relative, with the window covering
// [log(theta_min)/2 - pad, log(theta_max)/2 + pad]; theta_min comes from the
// Sturm multisection of the stopping rule, theta_max from Gershgorin.
//
// Log det (Section 6, Gauss quadrature e_1^T log(T_m) e_1): from
//   log t = int_0^inf (1/(1+s) - 1/(t+s)) ds = int_R (e^u/(1+e^u) - e^u/(t+e^u)) du
// the trapezoid rule gives
//   e_1^T log(T) e_1 ~= sum_k h e^{u_k} (1/(1+e^{u_k}) - [(T + e^{u_k} I)^{-1}]_{11}),
// with [(T + sI)^{-1}]_{11} = 1 / d~_1 from the backward continued fraction
// d~_m = a_m + s, d~_i = a_i + s - b_i^2 / d~_{i+1}.  Error ~ exp(-2 pi^2 / h).
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"

namespace gmrf {
namespace {

constexpr double kPi = 3.14159265358979323846;

struct DMax {
  double v;
  __device__ void zero() { v = 0.0; }
  __device__ void merge(const DMax& o) { v = fmax(v, o.v); }
  __device__ DMax shfl_down(int off) const { return {__shfl_down_sync(0xffffffffu, v, off)}; }
};
struct DSum {
  double v;
  __device__ void zero() { v = 0.0; }
  __device__ void merge(const DSum& o) { v += o.v; }
  __device__ DSum shfl_down(int off) const { return {__shfl_down_sync(0xffffffffu, v, off)}; }
};

__device__ __forceinline__ bool usable(const VecState& v) {
  return (v.status == VS_DONE || v.status == GMRF_ERR_NOT_CONVERGED) && v.m >= 1;
}

// Node window per vector.  kind 0: inverse square root; kind 1: log.
__global__ void k_nodes(const VecState* st, const double* alpha, const double* beta, int m_max, int kind, bool fp64,
                        TmNodes* nodes) {
  __shared__ DMax red[8];
  const int s = blockIdx.x;
  const VecState v = st[s];
  TmNodes out = {0.0, 1.0, 0, 0};
  if (!usable(v)) {
    if (threadIdx.x == 0) nodes[s] = out;
    return;
  }
  const int m = v.m;
  const double* a = alpha + (size_t)s * m_max;
  const double* b = beta + (size_t)s * m_max;
  DMax g;
  g.zero();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double r = a[i];
    if (i > 0) r += fabs(b[i - 1]);
    if (i < m - 1) r += fabs(b[i]);
    g.v = fmax(g.v, r);
  }
  g = block_reduce(g, red);
  if (threadIdx.x == 0) {
    const double tmax = 2.0 * g.v;
    const double tmin = 0.5 * v.theta;
    double eps, h, pad, lo, hi;
    if (kind == 0) {
      eps = fp64 ? 1e-15 : 1e-11;
      h = kPi * kPi / log(4.0 / eps);
      pad = log(2.0 / (kPi * eps));
      lo = 0.5 * log(tmin) - pad;
      hi = 0.5 * log(tmax) + pad;
    } else {
      eps = fp64 ? 1e-16 : 1e-12;
      h = 2.0 * kPi * kPi / log(1.0 / eps);
      pad = log(1.0 / eps) + 2.0;
      lo = log(tmin) - pad;
      hi = log(tmax) + pad;
    }
    if (!(tmin > 0.0) || !(tmax > 0.0) || !isfinite(lo) || !isfinite(hi)) {
      nodes[s] = out;  // L = 0: no usable window (reported through the vector's status)
      return;
    }
    int L = (int)ceil((hi - lo) / h) + 1;
    if (L > kMaxNodes) {
      L = kMaxNodes;
      h = (hi - lo) / (L - 1);
    }
    out.s_lo = lo;
    out.h = h;
    out.L = L;
    nodes[s] = out;
  }
}

// One pole per thread: D[s][i][k] = w_k ((T + sigma_k I)^{-1} e_1)_i, with the
// Thomas sweep's c'_i kept in C[s][i][k].  Layout k-fastest for coalescing.
__global__ void k_poles(const VecState* st, const double* alpha, const double* beta, int m_max, const TmNodes* nodes,
                        double* C, double* D) {
  const int s = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const VecState v = st[s];
  const TmNodes nd = nodes[s];
  if (!usable(v) || k >= nd.L) return;
  const int m = v.m;
  const double* a = alpha + (size_t)s * m_max;
  const double* b = beta + (size_t)s * m_max;
  const double u = nd.s_lo + nd.h * k;
  const double sigma = exp(2.0 * u);
  const double w = (2.0 * nd.h / kPi) * exp(u);
  const size_t base = (size_t)s * m_max * kMaxNodes;
  // forward sweep: c'_i = b_i / den_i, d'_i = (rhs_i - b_{i-1} d'_{i-1}) / den_i
  double cp = 0.0, dp = 0.0;
  for (int i = 0; i < m; ++i) {
    const double den = (a[i] + sigma) - (i > 0 ? b[i - 1] * cp : 0.0);
    const double rden = 1.0 / den;
    const double rhs = (i == 0) ? 1.0 : 0.0;
    dp = (rhs - (i > 0 ? b[i - 1] * dp : 0.0)) * rden;
    cp = (i < m - 1) ? b[i] * rden : 0.0;
    C[base + (size_t)i * kMaxNodes + k] = cp;
    D[base + (size_t)i * kMaxNodes + k] = dp;
  }
  // back substitution x_{m-1} = d'_{m-1}, x_i = d'_i - c'_i x_{i+1}
  double x = 0.0;
  for (int i = m - 1; i >= 0; --i) {
    const size_t o = base + (size_t)i * kMaxNodes + k;
    x = D[o] - C[o] * x;
    D[o] = w * x;
  }
}

// y[s][i] = sum_k D[s][i][k] in a fixed order; one warp per component i.
__global__ void k_pole_sum(const VecState* st, int m_max, const TmNodes* nodes, const double* D, double* y) {
  const int s = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + warp;
  const VecState v = st[s];
  const TmNodes nd = nodes[s];
  if (i >= m_max) return;
  if (!usable(v) || i >= v.m) {
    if (lane == 0) y[(size_t)s * m_max + i] = 0.0;
    return;
  }
  const double* row = D + (size_t)s * m_max * kMaxNodes + (size_t)i * kMaxNodes;
  double acc = 0.0;
  for (int k = lane; k < nd.L; k += 32) acc += row[k];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if (lane == 0) y[(size_t)s * m_max + i] = acc;
}

// q[s] = ||v||^2 e_1^T log(T_m) e_1.
__global__ void k_log(const VecState* st, const double* alpha, const double* beta, int m_max, const TmNodes* nodes,
                      double* q) {
  __shared__ DSum red[8];
  const int s = blockIdx.x;
  const VecState v = st[s];
  const TmNodes nd = nodes[s];
  if (!usable(v)) {
    if (threadIdx.x == 0) q[s] = (v.status == VS_DONE) ? 0.0 : NAN;
    return;
  }
  const int m = v.m;
  const double* a = alpha + (size_t)s * m_max;
  const double* b = beta + (size_t)s * m_max;
  DSum acc;
  acc.zero();
  for (int k = threadIdx.x; k < nd.L; k += blockDim.x) {
    const double u = nd.s_lo + nd.h * k;
    const double t = exp(u);
    double dt = a[m - 1] + t;
    for (int i = m - 2; i >= 0; --i) dt = (a[i] + t) - b[i] * b[i] / dt;
    acc.v += nd.h * t * (1.0 / (1.0 + t) - 1.0 / dt);
  }
  acc = block_reduce(acc, red);
  if (threadIdx.x == 0) q[s] = v.znorm * v.znorm * acc.v;
}

// Estimate and standard error over ng = nq / group draws, draw d being the sum
// of q[d * group .. d * group + group - 1] (group > 1: the colour classes of
// the coloured estimator, Section 6.1).
__global__ void k_logdet_reduce(const double* q, int nq, int group, double shift, double* out) {
  __shared__ DSum red[8];
  const int ng = nq / group;
  DSum s1;
  s1.zero();
  for (int d = threadIdx.x; d < ng; d += blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < group; ++c) t += q[(size_t)d * group + c];
    s1.v += t;
  }
  s1 = block_reduce(s1, red);
  __shared__ double mean;
  if (threadIdx.x == 0) mean = s1.v / ng;
  __syncthreads();
  DSum s2;
  s2.zero();
  for (int d = threadIdx.x; d < ng; d += blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < group; ++c) t += q[(size_t)d * group + c];
    s2.v += (t - mean) * (t - mean);
  }
  s2 = block_reduce(s2, red);
  if (threadIdx.x == 0) {
    out[0] = mean + shift;
    out[1] = ng > 1 ? sqrt(s2.v / (ng - 1) / ng) : NAN;
  }
}

// y = T_m^{-1} e_1 (the CG coefficients of a linear solve) by the LDL^T
// factorisation that the stopping rule also runs: d_0 = a_0,
// d_i = a_i - b_{i-1}^2 / d_{i-1}, l_i = b_{i-1} / d_{i-1}; L w = e_1 gives
// w_i = -l_i w_{i-1}; then y = L^{-T} D^{-1} w.  One thread per vector.
__global__ void k_tm_inv(const VecState* st, const double* alpha, const double* beta, int m_max, int nvec,
                         double* dwork, double* y) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nvec) return;
  const VecState v = st[s];
  if (!usable(v)) return;
  const int m = v.m;
  const double* a = alpha + (size_t)s * m_max;
  const double* b = beta + (size_t)s * m_max;
  double* d = dwork + (size_t)s * m_max;
  double* ys = y + (size_t)s * m_max;
  // d[] keeps the reciprocal pivots 1 / d_i: one FP64 division per row (the
  // chain is serial, and GB300's FP64 divisions are slow)
  double dinv = 1.0 / a[0], w = 1.0;
  d[0] = dinv;
  ys[0] = w * dinv;  // z_i = w_i / d_i
  for (int i = 1; i < m; ++i) {
    const double l = b[i - 1] * dinv;
    const double dp = a[i] - l * b[i - 1];
    w = -l * w;
    dinv = 1.0 / dp;
    d[i] = dinv;
    ys[i] = w * dinv;
  }
  for (int i = m - 2; i >= 0; --i) ys[i] -= (b[i] * d[i]) * ys[i + 1];  // y_i = z_i - l_{i+1} y_{i+1}
}

}  // namespace

cudaError_t launch_tm_inv(const LanczosBufs& b, double* dwork, double* y, cudaStream_t s) {
  k_tm_inv<<<(b.nvec + 31) / 32, 32, 0, s>>>(b.st, b.alpha, b.beta, b.m_max, b.nvec, dwork, y);
  return cudaGetLastError();
}

cudaError_t launch_tm_inv_sqrt(const LanczosBufs& b, bool fp64, TmNodes* nodes, double* scratch, double* y,
                               cudaStream_t s) {
  k_nodes<<<b.nvec, 256, 0, s>>>(b.st, b.alpha, b.beta, b.m_max, 0, fp64, nodes);
  double* C = scratch;
  double* D = scratch + (size_t)b.nvec * b.m_max * kMaxNodes;
  dim3 g1((kMaxNodes + 63) / 64, b.nvec);
  k_poles<<<g1, 64, 0, s>>>(b.st, b.alpha, b.beta, b.m_max, nodes, C, D);
  dim3 g2((b.m_max + 7) / 8, b.nvec);
  k_pole_sum<<<g2, 256, 0, s>>>(b.st, b.m_max, nodes, D, y);
  return cudaGetLastError();
}

cudaError_t launch_tm_log(const LanczosBufs& b, bool fp64, TmNodes* nodes, double* q, cudaStream_t s) {
  k_nodes<<<b.nvec, 256, 0, s>>>(b.st, b.alpha, b.beta, b.m_max, 1, fp64, nodes);
  k_log<<<b.nvec, 256, 0, s>>>(b.st, b.alpha, b.beta, b.m_max, nodes, q);
  return cudaGetLastError();
}

cudaError_t launch_logdet_reduce(const double* q, int nq, int group, double shift, double* out, cudaStream_t s) {
  k_logdet_reduce<<<1, 256, 0, s>>>(q, nq, group, shift, out);
  return cudaGetLastError();
}

}  // namespace gmrf
