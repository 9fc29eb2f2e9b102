// sparse.cu -- general sparse precision matrices Q (CSR) with an optional
// incomplete-Cholesky preconditioner M = F F^T (Section 5.2, Figure 3;
// Proposition 1 with this F):
//     x = F^{-T} A^{-1/2} z,   A = F^{-1} Q F^{-T},
//     log det Q = log det A + 2 sum_i log F_ii   (Section 6.2).
//
// Host side: validation of the CSR input, the threshold incomplete Cholesky
// factorisation (gmrf_ichol), and the level schedules of the two triangular
// solves.  Device side: one thread block per vector, whose working vectors
// stay in shared memory for a whole Lanczos step:
//     v_j formed from q_{j-1}, v_{j-1} (as in the lattice steps), stored;
//     t = F^{-T} v_j     backward substitution, level by level, in place
//                        (a group of lanes per row, sized to the rows);
//     u = Q t            CSR rows, Q read through L2 (shared by all blocks);
//     u := F^{-1} u      forward substitution, level by level, in place;
//     q_j = u - beta_{j-1} v_{j-1} -> W_out, the three dot products,
// then alpha_j = v_j . q_j, beta_j = ||q_j - alpha_j v_j|| (a second pass over
// the vectors in shared memory, exact also where A is close to the identity)
// and the stopping rule (finish_step, common.cuh) in the same block.  Rows of one level depend only on rows of earlier levels, so
// the threads of the block solve them in parallel with one barrier per level.
// Without F the step is u = Q v_j.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "internal.h"

namespace gmrf {

struct SparseOp {
  int n = 0;
  bool has_f = false;
  bool fp64 = false;
  // device arrays (T = float or double values)
  int* q_ptr = nullptr;  // Q: [n + 1], [nnz] columns, [nnz] values
  int* q_col = nullptr;
  void* q_val = nullptr;
  // The two substitutions, each with its rows stored in level order (entry r
  // of the order is row rows[r]): row pointers [n + 1], columns and values of
  // the off-diagonal entries, and 1 / F_ii [n], all indexed by r, so a row's
  // pointers load without going through its row index first.
  //   forward  (F^{-1}):  the strictly lower part of F by rows
  //   backward (F^{-T}):  the strictly upper part of F^T by rows (F by columns)
  int* l_ptr = nullptr;
  int* l_col = nullptr;
  void* l_val = nullptr;
  void* l_dinv = nullptr;
  int* u_ptr = nullptr;
  int* u_col = nullptr;
  void* u_val = nullptr;
  void* u_dinv = nullptr;
  int* lev_f = nullptr;     // rows in forward-solve level order [n]
  int* lev_f_ptr = nullptr; // [nlev_f + 1]
  int* lev_b = nullptr;     // rows in backward-solve level order [n]
  int* lev_b_ptr = nullptr; // [nlev_b + 1]
  int nlev_f = 0, nlev_b = 0;
  int gs = 1;               // lanes per row in the triangular solves
  size_t smem = 0;          // dynamic shared memory of the kernels
};

namespace {

constexpr int kSpThreads = 256;

// ------------------------------------------------------------------ host: CSR
struct HostCsr {
  int64_t n;
  const int64_t* ptr;
  const int32_t* col;
  const double* val;
};

// Structural checks: pointers monotone from 0, columns in range, no
// duplicate column within a row, finite values.
bool csr_wellformed(const HostCsr& a) {
  if (!a.ptr || !a.col || !a.val || a.n < 1 || a.ptr[0] != 0) return false;
  std::vector<int64_t> stamp((size_t)a.n, -1);
  for (int64_t i = 0; i < a.n; ++i) {
    if (a.ptr[i + 1] < a.ptr[i]) return false;
    for (int64_t e = a.ptr[i]; e < a.ptr[i + 1]; ++e) {
      const int64_t c = a.col[e];
      if (c < 0 || c >= a.n || stamp[(size_t)c] == i || !std::isfinite(a.val[e])) return false;
      stamp[(size_t)c] = i;
    }
  }
  return a.ptr[a.n] < ((int64_t)1 << 31);
}

// Rows with their entries sorted by column (for lookups).
struct SortedRows {
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  explicit SortedRows(const HostCsr& a) : ptr(a.ptr, a.ptr + a.n + 1), col((size_t)a.ptr[a.n]), val((size_t)a.ptr[a.n]) {
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t i = 0; i < a.n; ++i) {
      row.clear();
      for (int64_t e = a.ptr[i]; e < a.ptr[i + 1]; ++e) row.emplace_back(a.col[e], a.val[e]);
      std::sort(row.begin(), row.end(), [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
        return x.first < y.first;
      });
      for (size_t k = 0; k < row.size(); ++k) {
        col[(size_t)a.ptr[i] + k] = row[k].first;
        val[(size_t)a.ptr[i] + k] = row[k].second;
      }
    }
  }
  // value at (i, j), or 0 with *found = false
  double at(int64_t i, int32_t j, bool* found) const {
    const int32_t* b = col.data() + ptr[(size_t)i];
    const int32_t* e = col.data() + ptr[(size_t)i + 1];
    const int32_t* it = std::lower_bound(b, e, j);
    *found = it != e && *it == j;
    return *found ? val[(size_t)(it - col.data())] : 0.0;
  }
};

// Q symmetric (exact value equality) with a positive diagonal.
bool csr_symmetric_posdiag(const HostCsr& a, const SortedRows& r) {
  for (int64_t i = 0; i < a.n; ++i) {
    bool has_diag = false;
    for (int64_t e = r.ptr[(size_t)i]; e < r.ptr[(size_t)i + 1]; ++e) {
      const int32_t j = r.col[(size_t)e];
      if (j == i) {
        if (!(r.val[(size_t)e] > 0.0)) return false;
        has_diag = true;
        continue;
      }
      bool found = false;
      const double v = r.at(j, (int32_t)i, &found);
      if (!found || v != r.val[(size_t)e]) return false;
    }
    if (!has_diag) return false;
  }
  return true;
}

// Threshold incomplete Cholesky of A' = Q + shift diag(Q), left-looking by
// columns (the rule is stated with gmrf_ichol in include/gmrf.h).  Columns of
// F are kept as (row, value) lists in ascending row order; for column j the
// columns k < j with F_jk != 0 are found through per-column cursors (`next`)
// linked into the list of the row their next entry lies in.
struct IcholResult {
  std::vector<std::vector<std::pair<int32_t, double>>> cols;  // strictly lower entries of column j
  std::vector<double> diag;
  int64_t fail_col = -1;
};

bool ichol_columns(const SortedRows& r, int64_t n, double droptol, double shift, IcholResult& out) {
  out.cols.assign((size_t)n, {});
  out.diag.assign((size_t)n, 0.0);
  std::vector<double> w((size_t)n, 0.0);
  std::vector<int64_t> touched_at((size_t)n, -1), in_a((size_t)n, -1);
  std::vector<int32_t> touched;
  std::vector<size_t> next((size_t)n, 0);
  std::vector<int64_t> head((size_t)n, -1), link((size_t)n, -1);  // lists of columns by next row
  const bool ic0 = droptol < 0.0;
  for (int64_t j = 0; j < n; ++j) {
    touched.clear();
    double norm1 = 0.0;
    // column j of A' below and on the diagonal = row j of A' at columns >= j (symmetry)
    for (int64_t e = r.ptr[(size_t)j]; e < r.ptr[(size_t)j + 1]; ++e) {
      const int32_t i = r.col[(size_t)e];
      if (i < j) continue;
      double v = r.val[(size_t)e];
      if (i == j) v += shift * v;
      w[(size_t)i] = v;
      touched_at[(size_t)i] = j;
      if (v != 0.0) in_a[(size_t)i] = j;  // Q's pattern (explicit zeros excluded)
      touched.push_back(i);
      norm1 += std::fabs(v);
    }
    // w -= F[j:, k] F_jk for every column k < j with F_jk != 0
    for (int64_t k = head[(size_t)j]; k >= 0;) {
      const int64_t knext = link[(size_t)k];
      const auto& ck = out.cols[(size_t)k];
      const size_t p0 = next[(size_t)k];  // ck[p0].first == j
      const double fjk = ck[p0].second;
      for (size_t p = p0; p < ck.size(); ++p) {
        const int32_t i = ck[p].first;
        if (touched_at[(size_t)i] != j) {
          touched_at[(size_t)i] = j;
          w[(size_t)i] = 0.0;
          touched.push_back(i);
        }
        w[(size_t)i] -= ck[p].second * fjk;
      }
      // advance column k's cursor past row j and relink it
      next[(size_t)k] = p0 + 1;
      if (p0 + 1 < ck.size()) {
        const int32_t rnext = ck[p0 + 1].first;
        link[(size_t)k] = head[(size_t)rnext];
        head[(size_t)rnext] = k;
      }
      k = knext;
    }
    head[(size_t)j] = -1;
    const double pivot = w[(size_t)j];
    if (!(pivot > 0.0) || !std::isfinite(pivot)) {
      out.fail_col = j;
      return false;
    }
    const double d = std::sqrt(pivot);
    out.diag[(size_t)j] = d;
    std::sort(touched.begin(), touched.end());
    auto& cj = out.cols[(size_t)j];
    const double thr = ic0 ? 0.0 : droptol * norm1;
    for (int32_t i : touched) {
      if (i == j) continue;
      const double wi = w[(size_t)i];
      // exact zeros (a cancelled update, an explicit zero of Q) are not stored
      const bool keep = wi != 0.0 && (ic0 ? (in_a[(size_t)i] == j) : !(std::fabs(wi) < thr));
      if (keep) cj.emplace_back(i, wi / d);
    }
    if (!cj.empty()) {
      next[(size_t)j] = 0;
      const int32_t r0 = cj[0].first;
      link[(size_t)j] = head[(size_t)r0];
      head[(size_t)r0] = j;
    }
  }
  return true;
}

// ------------------------------------------------------------------ device
template <typename T>
struct SpArgs {
  int n;
  const int* qp;
  const int* qc;
  const T* qv;
  const int* lp;
  const int* lc;
  const T* lv;
  const T* ldi;
  const int* up;
  const int* uc;
  const T* uv;
  const T* udi;
  const int* lf;
  const int* lfp;
  int nlf;
  const int* lb;
  const int* lbp;
  int nlb;
  int has_f;
  int gs;  // lanes per row in the triangular solves: a power of two <= 32
};

// One level-scheduled substitution in place: x_i := (x_i - sum_e val_e x_col_e) * (1 / d_i)
// for the rows of each level in turn (the reciprocal pivots are stored).  A group of gs lanes (aligned within a
// warp) takes one row, its lanes striding over the row's entries, and the
// group sums by shuffles; the block's groups take the level's rows in rounds.
// The round loop depends only on the level, so every lane of a warp reaches
// the shuffles (inactive groups add zeros).
template <typename T>
__device__ __forceinline__ void tri_solve(const SpArgs<T>& a, const int* __restrict__ rows,
                                          const int* __restrict__ lptr, int nlev, const int* __restrict__ rp,
                                          const int* __restrict__ col, const T* __restrict__ val,
                                          const T* __restrict__ dinv, T* x) {
  const int gs = a.gs;
  const int grp = (int)threadIdx.x / gs, sub = (int)threadIdx.x & (gs - 1);
  const int ngrp = (int)blockDim.x / gs;
  for (int l = 0; l < nlev; ++l) {
    const int r0 = __ldg(lptr + l), r1 = __ldg(lptr + l + 1);
    for (int base = r0; base < r1; base += ngrp) {
      const int r = base + grp;
      int i = 0;
      T acc = 0;
      if (r < r1) {
        i = __ldg(rows + r);
        const int e1 = __ldg(rp + r + 1);
        for (int e = __ldg(rp + r) + sub; e < e1; e += gs) acc += __ldg(val + e) * x[__ldg(col + e)];
      }
      for (int off = gs >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (r < r1 && sub == 0) x[i] = (x[i] - acc) * __ldg(dinv + r);
    }
    __syncthreads();
  }
}

// x := F^{-1} x  (forward substitution)
template <typename T>
__device__ __forceinline__ void lower_solve(const SpArgs<T>& a, T* x) {
  tri_solve(a, a.lf, a.lfp, a.nlf, a.lp, a.lc, a.lv, a.ldi, x);
}

// x := F^{-T} x  (backward substitution)
template <typename T>
__device__ __forceinline__ void upper_solve(const SpArgs<T>& a, T* x) {
  tri_solve(a, a.lb, a.lbp, a.nlb, a.up, a.uc, a.uv, a.udi, x);
}

// y = Q x for all rows (x, y in shared memory; y written, no barrier)
template <typename T>
__device__ __forceinline__ void spmv(const SpArgs<T>& a, const T* x, T* y) {
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
    T acc = 0;
    for (int e = __ldg(a.qp + i); e < __ldg(a.qp + i + 1); ++e) acc += __ldg(a.qv + e) * x[__ldg(a.qc + e)];
    y[i] = acc;
  }
}

template <typename T>
struct SpStep {
  T* W0;
  T* W1;
  T* V;
  StepParams P;
  VecState* st;
  double* alpha;
  double* beta;
  float* alpha_f;
  float* beta2_f;
  Dots<T>* partials;
};

// One Lanczos step (Algorithm 1) on A (or Q without F) for vector blockIdx.x.
template <typename T>
__global__ void __launch_bounds__(kSpThreads) k_sparse_step(SpArgs<T> a, SpStep<T> b) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ Dots<T> red[kSpThreads / 32];
  __shared__ int s_int[4];
  __shared__ float s_flt[4];
  const int s = blockIdx.x;
  if (b.st[s].status != VS_RUNNING) return;
  const int j = b.st[s].m;
  const int n = a.n;
  T* sv = reinterpret_cast<T*>(smraw);  // v_j
  T* sw = sv + n;                       // t = F^{-T} v_j
  T* su = sw + n;                       // u = Q t, then F^{-1} u
  const size_t nn = (size_t)n;
  const T* Win = ((j & 1) ? b.W1 : b.W0) + (size_t)s * nn;
  T* Wout = ((j & 1) ? b.W0 : b.W1) + (size_t)s * nn;
  const size_t base = (size_t)s * b.P.nslots;
  T* Vc = b.V + (base + (size_t)(j % b.P.nslots)) * nn;
  const T* Vp = j > 0 ? b.V + (base + (size_t)((j - 1) % b.P.nslots)) * nn : nullptr;
  T coef = 0, bprev = 0;
  const T inv_b = (T)b.st[s].vscale;
  if (j > 0) {
    const size_t mo = (size_t)s * b.P.m_max + (j - 1);
    coef = (T)b.alpha[mo];
    bprev = (T)b.beta[mo];
  }
  // v_j = (q_{j-1} - alpha_{j-1} v_{j-1}) / beta_{j-1}   (v_0 = z / ||z||)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const T w = Win[i];
    const T v = j == 0 ? w * inv_b : (w - coef * Vp[i]) * inv_b;
    sv[i] = v;
    sw[i] = v;
    Vc[i] = v;
  }
  __syncthreads();
  if (a.has_f) {
    upper_solve(a, sw);
    spmv(a, sw, su);
    __syncthreads();
    lower_solve(a, su);
  } else {
    spmv(a, sv, su);
    __syncthreads();
  }
  // q_j = A v_j - beta_{j-1} v_{j-1} (kept in su), dot products
  Dots<T> d;
  d.zero();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const T v = sv[i];
    const T q = j > 0 ? su[i] - bprev * Vp[i] : su[i];
    su[i] = q;
    Wout[i] = q;
    d.add(v, q);
  }
  d = block_reduce(d, red);
  __shared__ double s_alpha, s_b2;
  if (threadIdx.x == 0) {
    b.partials[s] = d;
    double a1, a2, a3;
    d.get(a1, a2, a3);
    s_alpha = a1;
  }
  __syncthreads();
  // beta_j^2 = ||q_j - alpha_j v_j||^2 from the two vectors in shared memory
  const T al = (T)s_alpha;
  Dots<T> e;
  e.zero();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const T r = su[i] - al * sv[i];
    e.add(r, r);
  }
  e = block_reduce(e, red);
  if (threadIdx.x == 0) {
    double r1, r2, r3;
    e.get(r1, r2, r3);
    s_b2 = r2;
  }
  __syncthreads();
  finish_step<T>(b.P, j, s, b.partials, 1, b.st, b.alpha, b.beta, b.alpha_f, b.beta2_f, red, s_int, s_flt, s_b2);
}

// Plain applies on nvec vectors: mode 0 y = Q v, 1 y = A v, 2 y = F^{-T} v,
// 3 y = F^{-1} v.
template <typename T>
__global__ void __launch_bounds__(kSpThreads) k_sparse_ops(SpArgs<T> a, int mode, const T* in, T* out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n = a.n;
  T* sx = reinterpret_cast<T*>(smraw);
  T* sy = sx + n;
  const T* x = in + (size_t)blockIdx.x * n;
  T* y = out + (size_t)blockIdx.x * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sx[i] = x[i];
  __syncthreads();
  T* res = sx;
  if (mode == 0) {
    spmv(a, sx, sy);
    res = sy;
  } else if (mode == 1) {
    upper_solve(a, sx);
    spmv(a, sx, sy);
    __syncthreads();
    lower_solve(a, sy);
    res = sy;
  } else if (mode == 2) {
    upper_solve(a, sx);
  } else {
    lower_solve(a, sx);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = res[i];
}

template <typename T>
SpArgs<T> sp_args(const SparseOp& S) {
  SpArgs<T> a{};
  a.n = S.n;
  a.qp = S.q_ptr;
  a.qc = S.q_col;
  a.qv = (const T*)S.q_val;
  a.lp = S.l_ptr;
  a.lc = S.l_col;
  a.lv = (const T*)S.l_val;
  a.ldi = (const T*)S.l_dinv;
  a.up = S.u_ptr;
  a.uc = S.u_col;
  a.uv = (const T*)S.u_val;
  a.udi = (const T*)S.u_dinv;
  a.lf = S.lev_f;
  a.lfp = S.lev_f_ptr;
  a.nlf = S.nlev_f;
  a.lb = S.lev_b;
  a.lbp = S.lev_b_ptr;
  a.nlb = S.nlev_b;
  a.has_f = S.has_f ? 1 : 0;
  a.gs = S.gs;
  return a;
}

int optin_smem() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 48 * 1024;
  }
  return v;
}

// Raises the dynamic shared memory limit of a kernel to everything its static
// shared memory leaves of the opt-in limit; returns that amount (0 on error).
template <typename K>
size_t raise_smem(K kernel) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int avail = optin_smem() - (int)fa.sharedSizeBytes;
  if (avail <= 0 || cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, avail) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (size_t)avail;
}

// Done once per precision, at problem creation (outside any stream capture):
// the dynamic shared memory both kernels may use.
template <typename T>
size_t kernels_smem_limit() {
  static const size_t lim = std::min(raise_smem(k_sparse_step<T>), raise_smem(k_sparse_ops<T>));
  return lim;
}

template <typename T>
cudaError_t sparse_step_t(const SparseOp& S, const LanczosBufs& lb, const StepParams& P, cudaStream_t s) {
  SpStep<T> b{};
  b.W0 = (T*)lb.W[0];
  b.W1 = (T*)lb.W[1];
  b.V = (T*)lb.V;
  b.P = P;
  b.st = lb.st;
  b.alpha = lb.alpha;
  b.beta = lb.beta;
  b.alpha_f = lb.alpha_f;
  b.beta2_f = lb.beta2_f;
  b.partials = (Dots<T>*)lb.partials;
  k_sparse_step<T><<<lb.nvec, kSpThreads, S.smem, s>>>(sp_args<T>(S), b);
  return cudaGetLastError();
}

template <typename T>
cudaError_t sparse_ops_t(const SparseOp& S, int mode, const void* in, void* out, int nvec, cudaStream_t s) {
  k_sparse_ops<T><<<nvec, kSpThreads, S.smem, s>>>(sp_args<T>(S), mode, (const T*)in, (T*)out);
  return cudaGetLastError();
}

// Level of every row: forward (row i after the rows k < i it reads) or
// backward (row i after the rows k > i it reads); rows grouped by level.
void levels(int n, const std::vector<int>& ptr, const std::vector<int>& col, bool forward, std::vector<int>& rows,
            std::vector<int>& lptr) {
  std::vector<int> lev((size_t)n, 0);
  int nlev = 0;
  for (int t = 0; t < n; ++t) {
    const int i = forward ? t : n - 1 - t;
    int l = 0;
    for (int e = ptr[(size_t)i]; e < ptr[(size_t)i + 1]; ++e) l = std::max(l, lev[(size_t)col[(size_t)e]] + 1);
    lev[(size_t)i] = l;
    nlev = std::max(nlev, l + 1);
  }
  lptr.assign((size_t)nlev + 1, 0);
  for (int i = 0; i < n; ++i) ++lptr[(size_t)lev[(size_t)i] + 1];
  for (int l = 0; l < nlev; ++l) lptr[(size_t)l + 1] += lptr[(size_t)l];
  rows.assign((size_t)n, 0);
  std::vector<int> fill(lptr.begin(), lptr.end() - 1);
  for (int i = 0; i < n; ++i) rows[(size_t)fill[(size_t)lev[(size_t)i]]++] = i;
}

template <typename T>
int upload(void** dst, const std::vector<double>& v, cudaStream_t s) {
  std::vector<T> h(v.begin(), v.end());
  if (h.empty()) h.push_back(T(0));
  if (cudaMallocAsync(dst, h.size() * sizeof(T), s) != cudaSuccess) return GMRF_ERR_OOM;
  if (cudaMemcpyAsync(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return GMRF_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? GMRF_OK : GMRF_ERR_CUDA;
}
int upload_i(int** dst, const std::vector<int>& v, cudaStream_t s) {
  std::vector<int> h(v);
  if (h.empty()) h.push_back(0);
  if (cudaMallocAsync((void**)dst, h.size() * sizeof(int), s) != cudaSuccess) return GMRF_ERR_OOM;
  if (cudaMemcpyAsync(*dst, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return GMRF_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? GMRF_OK : GMRF_ERR_CUDA;
}

}  // namespace

int sparse_create(SparseOp** out, const gmrf_sparse_desc* d, bool fp64, cudaStream_t s, double* logdet_f) {
  *out = nullptr;
  const HostCsr q{d->n, d->rowptr, d->colind, d->val};
  if (d->n < 1 || d->n > (int64_t)1 << 30 || !csr_wellformed(q)) return GMRF_ERR_INVALID;
  const SortedRows qr(q);
  if (!csr_symmetric_posdiag(q, qr)) return GMRF_ERR_INVALID;
  const int n = (int)d->n;
  const bool has_f = d->f_rowptr != nullptr;
  std::vector<int> lp((size_t)n + 1, 0), lc, up((size_t)n + 1, 0), uc;
  std::vector<double> lv, uv, dg((size_t)n, 0.0);
  double ld = 0.0;
  if (has_f) {
    const HostCsr f{d->n, d->f_rowptr, d->f_colind, d->f_val};
    if (!csr_wellformed(f)) return GMRF_ERR_INVALID;
    // F: lower triangular with a positive diagonal in every row
    std::vector<int> cnt_u((size_t)n, 0);
    for (int i = 0; i < n; ++i) {
      bool has_diag = false;
      for (int64_t e = f.ptr[i]; e < f.ptr[i + 1]; ++e) {
        const int c = f.col[e];
        if (c > i) return GMRF_ERR_INVALID;
        if (c == i) {
          if (!(f.val[e] > 0.0)) return GMRF_ERR_INVALID;
          dg[(size_t)i] = f.val[e];
          has_diag = true;
        } else {
          lc.push_back(c);
          lv.push_back(f.val[e]);
          ++cnt_u[(size_t)c];
        }
      }
      if (!has_diag) return GMRF_ERR_INVALID;
      lp[(size_t)i + 1] = (int)lc.size();
      ld += 2.0 * std::log(dg[(size_t)i]);
    }
    // F^T by rows: row c of F^T holds F_ic for i > c
    for (int c = 0; c < n; ++c) up[(size_t)c + 1] = up[(size_t)c] + cnt_u[(size_t)c];
    uc.resize(lc.size());
    uv.resize(lc.size());
    std::vector<int> fill(up.begin(), up.end() - 1);
    for (int i = 0; i < n; ++i)
      for (int e = lp[(size_t)i]; e < lp[(size_t)i + 1]; ++e) {
        const int c = lc[(size_t)e];
        uc[(size_t)fill[(size_t)c]] = i;
        uv[(size_t)fill[(size_t)c]++] = lv[(size_t)e];
      }
  }
  const size_t es = fp64 ? sizeof(double) : sizeof(float);
  const size_t smem = 3 * (size_t)n * es;
  const size_t lim = fp64 ? kernels_smem_limit<double>() : kernels_smem_limit<float>();
  if (lim == 0) return GMRF_ERR_CUDA;
  if (smem + 2048 > lim) return GMRF_ERR_UNSUPPORTED;
  SparseOp* S = new (std::nothrow) SparseOp();
  if (!S) return GMRF_ERR_OOM;
  S->n = n;
  S->has_f = has_f;
  S->fp64 = fp64;
  S->smem = smem;
  auto fail = [&](int r) {
    sparse_free(S, s);
    return r;
  };
  std::vector<int> qp((size_t)n + 1), qc((size_t)q.ptr[n]);
  for (int i = 0; i <= n; ++i) qp[(size_t)i] = (int)qr.ptr[(size_t)i];
  for (size_t e = 0; e < qc.size(); ++e) qc[e] = qr.col[e];
  int r = upload_i(&S->q_ptr, qp, s);
  if (r == GMRF_OK) r = upload_i(&S->q_col, qc, s);
  if (r == GMRF_OK) r = fp64 ? upload<double>(&S->q_val, qr.val, s) : upload<float>(&S->q_val, qr.val, s);
  if (r == GMRF_OK && has_f) {
    std::vector<int> rf, pf, rb, pb;
    levels(n, lp, lc, true, rf, pf);
    levels(n, up, uc, false, rb, pb);
    S->nlev_f = (int)pf.size() - 1;
    S->nlev_b = (int)pb.size() - 1;
    // lanes per row: the power of two at or above the mean off-diagonal row length (1 .. 32)
    const double mean_row = (double)lc.size() / (double)n;
    while (S->gs < 32 && S->gs < mean_row) S->gs *= 2;
    // rows in level order: pointers, entries and 1 / F_ii indexed by the position r
    auto by_level = [&](const std::vector<int>& rows, const std::vector<int>& ptr, const std::vector<int>& col,
                        const std::vector<double>& val, std::vector<int>& optr, std::vector<int>& ocol,
                        std::vector<double>& oval, std::vector<double>& odinv) {
      optr.assign((size_t)n + 1, 0);
      ocol.clear();
      oval.clear();
      odinv.assign((size_t)n, 0.0);
      for (int q = 0; q < n; ++q) {
        const int i = rows[(size_t)q];
        for (int e = ptr[(size_t)i]; e < ptr[(size_t)i + 1]; ++e) {
          ocol.push_back(col[(size_t)e]);
          oval.push_back(val[(size_t)e]);
        }
        optr[(size_t)q + 1] = (int)ocol.size();
        odinv[(size_t)q] = 1.0 / dg[(size_t)i];
      }
    };
    std::vector<int> lp2, lc2, up2, uc2;
    std::vector<double> lv2, ld2, uv2, ud2;
    by_level(rf, lp, lc, lv, lp2, lc2, lv2, ld2);
    by_level(rb, up, uc, uv, up2, uc2, uv2, ud2);
    r = upload_i(&S->l_ptr, lp2, s);
    if (r == GMRF_OK) r = upload_i(&S->l_col, lc2, s);
    if (r == GMRF_OK) r = upload_i(&S->u_ptr, up2, s);
    if (r == GMRF_OK) r = upload_i(&S->u_col, uc2, s);
    if (r == GMRF_OK) r = upload_i(&S->lev_f, rf, s);
    if (r == GMRF_OK) r = upload_i(&S->lev_f_ptr, pf, s);
    if (r == GMRF_OK) r = upload_i(&S->lev_b, rb, s);
    if (r == GMRF_OK) r = upload_i(&S->lev_b_ptr, pb, s);
    if (r == GMRF_OK) {
      if (fp64) {
        r = upload<double>(&S->l_val, lv2, s);
        if (r == GMRF_OK) r = upload<double>(&S->u_val, uv2, s);
        if (r == GMRF_OK) r = upload<double>(&S->l_dinv, ld2, s);
        if (r == GMRF_OK) r = upload<double>(&S->u_dinv, ud2, s);
      } else {
        r = upload<float>(&S->l_val, lv2, s);
        if (r == GMRF_OK) r = upload<float>(&S->u_val, uv2, s);
        if (r == GMRF_OK) r = upload<float>(&S->l_dinv, ld2, s);
        if (r == GMRF_OK) r = upload<float>(&S->u_dinv, ud2, s);
      }
    }
  }
  if (r != GMRF_OK) {
    cudaGetLastError();
    return fail(r);
  }
  *logdet_f = ld;
  *out = S;
  return GMRF_OK;
}

void sparse_free(SparseOp* S, cudaStream_t s) {
  if (!S) return;
  void* ps[] = {S->q_ptr, S->q_col, S->q_val, S->l_ptr,  S->l_col,  S->l_val,     S->l_dinv,    S->u_ptr,
                S->u_col, S->u_val, S->u_dinv, S->lev_f, S->lev_f_ptr, S->lev_b, S->lev_b_ptr};
  for (void* p : ps)
    if (p) cudaFreeAsync(p, s);
  cudaGetLastError();
  delete S;
}

bool sparse_has_factor(const SparseOp* S) { return S && S->has_f; }
int sparse_size(const SparseOp* S) { return S ? S->n : 0; }

cudaError_t launch_sparse_step(const SparseOp& S, const LanczosBufs& b, const StepParams& P, cudaStream_t s) {
  return S.fp64 ? sparse_step_t<double>(S, b, P, s) : sparse_step_t<float>(S, b, P, s);
}

cudaError_t launch_sparse_ops(const SparseOp& S, int mode, const void* in, void* out, int nvec, cudaStream_t s) {
  if (mode < 0 || mode > 3 || (mode > 0 && !S.has_f)) return cudaErrorInvalidValue;
  return S.fp64 ? sparse_ops_t<double>(S, mode, in, out, nvec, s) : sparse_ops_t<float>(S, mode, in, out, nvec, s);
}

}  // namespace gmrf

extern "C" int gmrf_ichol(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val, double droptol,
                          double shift, int64_t cap, int64_t* f_rowptr, int32_t* f_colind, double* f_val,
                          int64_t* f_nnz) {
  using namespace gmrf;
  if (!f_nnz) return GMRF_ERR_INVALID;
  if (std::isnan(droptol) || !(shift >= 0.0) || !std::isfinite(shift)) return GMRF_ERR_INVALID;
  const HostCsr q{n, rowptr, colind, val};
  if (n < 1 || n > (int64_t)1 << 30 || !csr_wellformed(q)) return GMRF_ERR_INVALID;
  try {
    const SortedRows qr(q);
    if (!csr_symmetric_posdiag(q, qr)) return GMRF_ERR_INVALID;
    IcholResult res;
    if (!ichol_columns(qr, n, droptol, shift, res)) {
      *f_nnz = res.fail_col;
      return GMRF_ERR_NOT_SPD;
    }
    // rows of F: strictly lower entries (from the columns, in ascending column order), then the diagonal
    std::vector<int64_t> cnt((size_t)n + 1, 0);
    for (int64_t j = 0; j < n; ++j)
      for (const auto& e : res.cols[(size_t)j]) ++cnt[(size_t)e.first + 1];
    for (int64_t i = 0; i < n; ++i) cnt[(size_t)i + 1] += cnt[(size_t)i] + 1;  // + the diagonal of row i
    const int64_t nnz = cnt[(size_t)n];
    *f_nnz = nnz;
    if (f_rowptr)
      for (int64_t i = 0; i <= n; ++i) f_rowptr[i] = cnt[(size_t)i];
    if (!f_colind || !f_val) return GMRF_OK;
    if (cap < nnz) return GMRF_ERR_INVALID;
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t j = 0; j < n; ++j)
      for (const auto& e : res.cols[(size_t)j]) {
        const int64_t at = fill[(size_t)e.first]++;
        f_colind[at] = (int32_t)j;
        f_val[at] = e.second;
      }
    for (int64_t i = 0; i < n; ++i) {
      f_colind[fill[(size_t)i]] = (int32_t)i;
      f_val[fill[(size_t)i]] = res.diag[(size_t)i];
    }
  } catch (const std::bad_alloc&) {
    return GMRF_ERR_OOM;
  }
  return GMRF_OK;
}
