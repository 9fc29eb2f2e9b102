// precond.cu -- Proposition 1 with the constant-coefficient preconditioner of
// Section 5.1, applied by 2-D fast transforms in shared memory.
//
// M = tau B_bar^p, B_bar = kappa_bar^2 I + L_prec.  CIRCULANT: L_prec is the
// torus Laplacian (block circulant, 2-D real FFT).  MIRROR: L_prec is the
// cell-centred Neumann Laplacian = the torus Laplacian of the mirror-extended
// grid restricted to even vectors (2-D DCT-II, computed by Makhoul's
// reordering and a real FFT).  F = M^{1/2} (symmetric), so Proposition 1
// reads x = M^{-1/2} u with u ~ N(0, A^{-1}), A = M^{-1/2} Q M^{-1/2}.
//
// With Q = tau B^p, B = K + L_bc, and R = B - B_bar (diagonal
// kappa^2 - kappa_bar^2 plus the edge terms where L_bc and L_prec differ on
// the boundary), the preconditioned operator is applied as
//   p = 2:  A v = g + B_bar^{-1} (R g),   g = v + R (B_bar^{-1} v)   (A = C^T C, C = I + R B_bar^{-1})
//   p = 1:  A v = v + P (R (P v)),       P = B_bar^{-1/2}
// which is the same matrix as M^{-1/2} Q M^{-1/2}; each fast solve acts on a
// vector of the size of the correction, so FP32 rounding stays relative to
// ||v|| instead of being amplified by the spread of the preconditioner's
// spectrum.
//
// One preconditioned Lanczos step = 5 kernels:
//   row-forward (forms v_j, stores it) -> column (fwd * symbol * inv)
//   -> row-mid (inverse rows, g, R g, forward rows) -> column
//   -> row-last (inverse rows, A v_j, q_j, dot products, alpha/beta, stopping rule).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <atomic>
#include <vector>

#include "fft.cuh"
#include "precond.h"
#include "precond_fast.h"
#include "trace.h"

namespace gmrf {
namespace {

// M_MID does the middle pass in one kernel (no y-boundary terms of R);
// with them, M_MIDW writes w = B_bar^{-1} v of its rows to a global buffer and
// M_MIDG reads w of its rows and of their y-partners from it, so no block
// reads spectrum rows that another block of the same launch rewrites.
enum { M_FWD_PLAIN = 0, M_FWD_FORM = 1, M_INV_PLAIN = 2, M_MID = 3, M_LAST = 4, M_LAST_PLAIN = 5, M_MIDW = 6,
       M_MIDG = 7 };

template <typename R>
struct PArgs {
  typedef typename Cplx<R>::T C;
  int nx, ny, lognx, logny, power, bc, rb, cw;
  int form;        // FORM_SHIFT / FORM_CTC / FORM_DIAG
  R kbar2, dscale;
  R roff;          // R = K - roff (kappa_bar^2; 0 for FORM_DIAG, where K is the diagonal D)
  const R* lamx;
  const R* lamy;
  const C* twx;
  const C* twy;
  const C* dctx;
  const C* dcty;
  R* S;
  size_t sstride;  // per-vector stride of S in R units
  R* G;            // per-vector stride n
  R* Wg;           // w rows between M_MIDW and M_MIDG, per-vector stride n
  const R* in;     // plain input rows (FWD_PLAIN, MID/LAST_PLAIN v)
  R* out;          // plain output rows
  const float* kappa2;
  R kappa2_const;
  size_t n;
  // Lanczos: q ping-pong, W[j & 1] holds q_{j-1}, W[(j+1) & 1] receives q_j
  R* W0;
  R* W1;
  R* V;
  StepParams P;
  VecState* st;
  double* alpha;
  double* beta;
  float* alpha_f;
  float* beta2_f;
  Dots<R>* partials;
  unsigned* counters;
};

// Spectral row pitch (R units): CIRCULANT nx/2+1 complex, MIRROR nx reals.
template <int KIND>
__host__ __device__ __forceinline__ int spitch(int nx) {
  return KIND == GMRF_PREC_CIRCULANT ? nx + 2 : nx;
}

// Edge term of R at a boundary side: (L_bc - L_prec) for one missing/extra edge.
template <typename R, int KIND>
__device__ __forceinline__ R edge_term(int bc, R wi, R wp) {
  R b = bc == GMRF_BC_PERIODIC ? (wi - wp) : (bc == GMRF_BC_DIRICHLET ? wi : (R)0);
  R pr = KIND == GMRF_PREC_CIRCULANT ? (wi - wp) : (R)0;
  return b - pr;
}
template <int KIND>
__device__ __forceinline__ bool has_edge_terms(int bc) {
  return KIND == GMRF_PREC_CIRCULANT ? bc != GMRF_BC_PERIODIC : bc != GMRF_BC_NEUMANN;
}

// ---- row transforms on lines in shared memory (pitch PL reals per line)
// Forward: real lines in X (nl lines) -> S rows (rows[l]), Y scratch.  Mirror
// reorders X into Y first.  Clobbers X and Y.
template <typename R, int KIND>
__device__ void row_forward(const PArgs<R>& a, R* X, R* Y, int PL, int nl, const int* rows, R* Sv) {
  typedef typename Cplx<R>::T C;
  const int tid = block_tid(), nt = block_nt();
  const int nx = a.nx, half = nx >> 1;
  R* src = X;
  R* tmp = Y;
  if (KIND == GMRF_PREC_MIRROR) {
    for (int idx = tid; idx < nl * half; idx += nt) {
      const int l = idx / half, m = idx - l * half;
      Y[l * PL + m] = X[l * PL + 2 * m];
      Y[l * PL + nx - 1 - m] = X[l * PL + 2 * m + 1];
    }
    __syncthreads();
    src = Y;
    tmp = X;
  }
  C* Z = smem_fft<C>((C*)src, (C*)tmp, a.lognx - 1, nl, PL / 2, a.twx, nx, false);
  const int sp = spitch<KIND>(nx);
  for (int idx = tid; idx < nl * (half + 1); idx += nt) {
    const int l = idx / (half + 1), k = idx - l * (half + 1);
    const C zk = Z[l * (PL / 2) + (k & (half - 1))];
    const C zr = cconj(Z[l * (PL / 2) + ((half - k) & (half - 1))]);
    const C w = a.twx[k];
    const C dd = cmul(w, csub(zk, zr));
    C X_k = cmk<C>((R)0.5 * (zk.x + zr.x + dd.y), (R)0.5 * (zk.y + zr.y - dd.x));
    R* srow = Sv + (size_t)rows[l] * sp;
    if (KIND == GMRF_PREC_CIRCULANT) {
      ((C*)srow)[k] = X_k;
    } else {
      const C e = cmul(a.dctx[k], X_k);
      srow[k] = e.x;
      if (k > 0 && k < half) srow[nx - k] = cmulc(a.dctx[nx - k], X_k).x;
    }
  }
  __syncthreads();
}

// Inverse: S rows (rows[l]) -> real lines; B2 holds the half spectrum, the
// half-length inverse FFT ping-pongs between A and B.  Returns the buffer with
// the real result (A or B, or for MIRROR the one not holding u).
template <typename R, int KIND>
__device__ R* row_inverse(const PArgs<R>& a, R* A, R* B, R* B2, int PL, int nl, const int* rows, const R* Sv) {
  typedef typename Cplx<R>::T C;
  const int tid = block_tid(), nt = block_nt();
  const int nx = a.nx, half = nx >> 1;
  const int sp = spitch<KIND>(nx);
  C* H = (C*)B2;
  for (int idx = tid; idx < nl * (half + 1); idx += nt) {
    const int l = idx / (half + 1), k = idx - l * (half + 1);
    const R* srow = Sv + (size_t)rows[l] * sp;
    C v;
    if (KIND == GMRF_PREC_CIRCULANT) {
      v = ((const C*)srow)[k];
    } else {
      const R ck = srow[k];
      const R cnk = k == 0 ? (R)0 : srow[nx - k];
      v = cmulc(cmk<C>(ck, -cnk), a.dctx[k]);  // e^{+i pi k/(2N)} (C_k - i C_{N-k})
    }
    H[l * (PL / 2) + k] = v;
  }
  __syncthreads();
  C* Zin = (C*)A;
  for (int idx = tid; idx < nl * half; idx += nt) {
    const int l = idx / half, k = idx - l * half;
    const C xk = H[l * (PL / 2) + k];
    const C xr = cconj(H[l * (PL / 2) + half - k]);
    const C E = cmk<C>((R)0.5 * (xk.x + xr.x), (R)0.5 * (xk.y + xr.y));
    const C O = cmulc(cmk<C>((R)0.5 * (xk.x - xr.x), (R)0.5 * (xk.y - xr.y)), a.twx[k]);
    Zin[l * (PL / 2) + k] = cmk<C>(E.x - O.y, E.y + O.x);
  }
  __syncthreads();
  C* z = smem_fft<C>(Zin, (C*)B, a.lognx - 1, nl, PL / 2, a.twx, nx, true);
  R* u = (R*)z;
  if (KIND == GMRF_PREC_CIRCULANT) return u;
  R* x = (u == A) ? B : A;
  for (int idx = tid; idx < nl * half; idx += nt) {
    const int l = idx / half, m = idx - l * half;
    x[l * PL + 2 * m] = u[l * PL + m];
    x[l * PL + 2 * m + 1] = u[l * PL + nx - 1 - m];
  }
  __syncthreads();
  return x;
}

template <typename R>
__device__ __forceinline__ R kap(const PArgs<R>& a, size_t i) {
  return a.kappa2 ? (R)__ldg(a.kappa2 + i) : a.kappa2_const;
}

// (R w) at cell (x, row) where w lines are in Wl (line index li), partner row
// line index lp (or -1 when the row has no y partner edge term).
template <typename R, int KIND>
__device__ __forceinline__ R apply_R(const PArgs<R>& a, const R* Wl, int PL, int li, int lp, int x, int row) {
  const R wi = Wl[li * PL + x];
  R r = (kap(a, (size_t)row * a.nx + x) - a.roff) * wi;
  if (has_edge_terms<KIND>(a.bc)) {
    if (x == 0) r += edge_term<R, KIND>(a.bc, wi, Wl[li * PL + a.nx - 1]);
    if (x == a.nx - 1) r += edge_term<R, KIND>(a.bc, wi, Wl[li * PL]);
    if (lp >= 0) r += edge_term<R, KIND>(a.bc, wi, Wl[lp * PL + x]);
  }
  return r;
}

template <typename R, int KIND, int MODE>
__global__ void __launch_bounds__(256) k_prow(PArgs<R> a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int rows[20];
  __shared__ int partner[20];
  __shared__ Dots<R> red[8];
  __shared__ int s_int[4];
  __shared__ float s_flt[4];
  typedef typename Cplx<R>::T C;
  const int s = blockIdx.y;
  const bool step = (MODE == M_FWD_FORM || MODE == M_LAST ||
                     ((MODE == M_MID || MODE == M_MIDW || MODE == M_MIDG) && a.in == nullptr));
  int j = 0;
  if (step) {
    if (a.st[s].status != VS_RUNNING) return;
    j = a.st[s].m;  // step index: completed steps of this vector
  }
  const int tid = block_tid(), nt = block_nt();
  const int nx = a.nx, ny = a.ny, rb = a.rb;
  const int PL = nx + 2;
  const int y0 = blockIdx.x * rb;
  // line list: own rows, then y-partners of row 0 / row ny-1 when needed
  int nl = rb;
  if (tid == 0) {
    for (int l = 0; l < rb; ++l) {
      rows[l] = y0 + l;
      partner[l] = -1;
    }
    if ((MODE == M_MID || MODE == M_MIDG) && has_edge_terms<KIND>(a.bc)) {
      int extra = rb;
      const bool has0 = y0 == 0, hasN = y0 + rb == ny;
      if (has0) {
        if (hasN) partner[0] = rb - 1;
        else {
          rows[extra] = ny - 1;
          partner[extra] = 0;
          partner[0] = extra;
          ++extra;
        }
      }
      if (hasN) {
        if (has0) partner[rb - 1] = 0;
        else {
          rows[extra] = 0;
          partner[extra] = rb - 1;
          partner[rb - 1] = extra;
          ++extra;
        }
      }
      rows[19] = extra;
    } else {
      rows[19] = rb;
    }
  }
  __syncthreads();
  nl = rows[19];
  // staged lines: the block's rows, plus the two y-partner rows when R has edge terms
  const int LMAX = rb + (has_edge_terms<KIND>(a.bc) ? 2 : 0);
  R* B0 = (R*)smraw;
  R* B1 = B0 + (size_t)LMAX * PL;
  R* B2 = B1 + (size_t)LMAX * PL;
  R* GL = B2 + (size_t)LMAX * PL;
  R* Sv = a.S + (size_t)s * a.sstride;
  const size_t n = a.n;

  if (MODE == M_FWD_PLAIN || MODE == M_FWD_FORM) {
    const R* Win = nullptr;
    const R* Vp = nullptr;
    R* Vc = nullptr;
    R coef = 0, inv_b = 1;
    if (MODE == M_FWD_FORM) {
      const size_t base = (size_t)s * a.P.nslots;
      Win = ((j & 1) ? a.W1 : a.W0) + (size_t)s * n;
      Vc = a.V + (base + (size_t)(j % a.P.nslots)) * n;
      if (j == 0) {
        inv_b = (R)a.st[s].vscale;
      } else {
        Vp = a.V + (base + (size_t)((j - 1) % a.P.nslots)) * n;
        const size_t mo = (size_t)s * a.P.m_max + (j - 1);
        coef = (R)a.alpha[mo];
        inv_b = (R)a.st[s].vscale;
      }
    } else {
      Win = a.in + (size_t)s * n;
    }
    for (int idx = tid; idx < rb * nx; idx += nt) {
      const int l = idx / nx, x = idx - l * nx;
      const size_t i = (size_t)(y0 + l) * nx + x;
      R v = Win[i];
      if (MODE == M_FWD_FORM) {
        v = (j == 0) ? v * inv_b : (v - coef * Vp[i]) * inv_b;
        Vc[i] = v;
        if (a.P.vb) vb_store1(vb_at(a.P, s, j, n, i), (float)v);
      }
      B0[l * PL + x] = v;
    }
    __syncthreads();
    row_forward<R, KIND>(a, B0, B1, PL, rb, rows, Sv);
    return;
  }

  R* W = B0;
  if (MODE == M_MIDG) {
    // w of the block's rows and their y-partners, written by M_MIDW
    const R* wg = a.Wg + (size_t)s * n;
    for (int idx = tid; idx < nl * nx; idx += nt) {
      const int l = idx / nx, x = idx - l * nx;
      B0[l * PL + x] = wg[(size_t)rows[l] * nx + x];
    }
    __syncthreads();
  } else {
    W = row_inverse<R, KIND>(a, B0, B1, B2, PL, nl, rows, Sv);
  }
  if (MODE == M_MIDW) {
    R* wg = a.Wg + (size_t)s * n;
    for (int idx = tid; idx < rb * nx; idx += nt) {
      const int l = idx / nx, x = idx - l * nx;
      wg[(size_t)(y0 + l) * nx + x] = W[l * PL + x];
    }
    return;
  }

  if (MODE == M_INV_PLAIN) {
    R* o = a.out + (size_t)s * n;
    for (int idx = tid; idx < rb * nx; idx += nt) {
      const int l = idx / nx, x = idx - l * nx;
      o[(size_t)(y0 + l) * nx + x] = W[l * PL + x];
    }
    return;
  }

  // v: the caller's input (plain operator) or the basis vector v_j (step)
  const R* vsrc = a.in ? a.in + (size_t)s * n : a.V + ((size_t)s * a.P.nslots + (size_t)(j % a.P.nslots)) * n;

  if (MODE == M_MID || MODE == M_MIDG) {
    R* F = B2;                     // r lines (forward-transform input)
    R* T2 = (W == B0) ? B1 : B0;   // scratch for the forward transform
    R* base = W;                   // lines R is applied to
    if (a.form == FORM_CTC) {
      // g = v + R w on all lines (partners included)
      for (int idx = tid; idx < nl * nx; idx += nt) {
        const int l = idx / nx, x = idx - l * nx;
        const int row = rows[l];
        GL[l * PL + x] = vsrc[(size_t)row * nx + x] + apply_R<R, KIND>(a, W, PL, l, partner[l], x, row);
      }
      __syncthreads();
      base = GL;
      R* g = a.G + (size_t)s * n;
      for (int idx = tid; idx < rb * nx; idx += nt) {
        const int l = idx / nx, x = idx - l * nx;
        g[(size_t)(y0 + l) * nx + x] = GL[l * PL + x];
      }
    }
    for (int idx = tid; idx < rb * nx; idx += nt) {
      const int l = idx / nx, x = idx - l * nx;
      F[l * PL + x] = apply_R<R, KIND>(a, base, PL, l, partner[l], x, y0 + l);
    }
    __syncthreads();
    row_forward<R, KIND>(a, F, T2, PL, rb, rows, Sv);
    return;
  }

  // M_LAST / M_LAST_PLAIN: A v = g + h
  const R* gsrc = (a.form == FORM_CTC) ? (const R*)(a.G + (size_t)s * n) : vsrc;
  Dots<R> d;
  d.zero();
  if (MODE == M_LAST_PLAIN) {
    R* o = a.out + (size_t)s * n;
    for (int idx = tid; idx < rb * nx; idx += nt) {
      const int l = idx / nx, x = idx - l * nx;
      const size_t i = (size_t)(y0 + l) * nx + x;
      o[i] = gsrc[i] + W[l * PL + x];
    }
    return;
  }
  {
    const size_t base = (size_t)s * a.P.nslots;
    const R* Vc = a.V + (base + (size_t)(j % a.P.nslots)) * n;
    const R* Vp = j > 0 ? a.V + (base + (size_t)((j - 1) % a.P.nslots)) * n : nullptr;
    const R bprev = j > 0 ? (R)a.beta[(size_t)s * a.P.m_max + (j - 1)] : (R)0;
    R* Wo = ((j & 1) ? a.W0 : a.W1) + (size_t)s * n;
    for (int idx = tid; idx < rb * nx; idx += nt) {
      const int l = idx / nx, x = idx - l * nx;
      const size_t i = (size_t)(y0 + l) * nx + x;
      const R v = Vc[i];
      R q = gsrc[i] + W[l * PL + x];
      if (j > 0) q -= bprev * Vp[i];
      Wo[i] = q;
      d.add(v, q);
    }
  }
  d = block_reduce(d, red);
  const int nblk = gridDim.x;
  if (tid == 0) a.partials[(size_t)s * nblk + blockIdx.x] = d;
  if (last_block(a.counters, s, nblk, &s_int[3]))
    finish_step<R>(a.P, j, s, a.partials, nblk, a.st, a.alpha, a.beta, a.alpha_f, a.beta2_f, red, s_int, s_flt);
}

// Column pass: forward transform along y, multiply by the symbol of
// B_bar^{-p/2} (times the transform normalisation), inverse transform.
template <typename R>
__device__ __forceinline__ R symbol(const PArgs<R>& a, int kx, int ky) {
  const R lam = a.kbar2 + a.lamx[kx] + a.lamy[ky];
  return (a.power == 2 ? (R)1 / lam : (R)1 / sqrt(lam)) * a.dscale;
}

template <typename R, int KIND>
__global__ void __launch_bounds__(256) k_pcol(PArgs<R> a, int step_mode) {
  extern __shared__ __align__(16) unsigned char smraw[];
  typedef typename Cplx<R>::T C;
  const int s = blockIdx.y;
  if (step_mode && a.st[s].status != VS_RUNNING) return;
  const int tid = block_tid(), nt = block_nt();
  const int nx = a.nx, ny = a.ny, cw = a.cw;
  const int c0 = blockIdx.x * cw;
  R* Sv = a.S + (size_t)s * a.sstride;
  if (KIND == GMRF_PREC_CIRCULANT) {
    const int ncx = nx / 2 + 1;
    const int P = ny + 1;  // complex pitch (bank-conflict padding)
    C* A = (C*)smraw;
    C* B = A + (size_t)cw * P;
    C* Srow = (C*)Sv;
    for (int idx = tid; idx < cw * ny; idx += nt) {
      const int ky = idx / cw, c = idx - ky * cw;
      const int kx = c0 + c;
      A[c * P + ky] = kx < ncx ? Srow[(size_t)ky * ncx + kx] : cmk<C>((R)0, (R)0);
    }
    __syncthreads();
    C* F = smem_fft<C>(A, B, a.logny, cw, P, a.twy, ny, false);
    for (int idx = tid; idx < cw * ny; idx += nt) {
      const int c = idx / ny, ky = idx - c * ny;
      const int kx = c0 + c;
      if (kx < ncx) {
        const R d = symbol(a, kx, ky);
        C v = F[c * P + ky];
        F[c * P + ky] = cmk<C>(v.x * d, v.y * d);
      }
    }
    __syncthreads();
    C* G = smem_fft<C>(F, F == A ? B : A, a.logny, cw, P, a.twy, ny, true);
    for (int idx = tid; idx < cw * ny; idx += nt) {
      const int ky = idx / cw, c = idx - ky * cw;
      const int kx = c0 + c;
      if (kx < ncx) Srow[(size_t)ky * ncx + kx] = G[c * P + ky];
    }
    return;
  }
  // MIRROR: real DCT-II columns
  const int P = ny + 2;  // reals per line (complex pitch ny/2 + 1)
  const int half = ny >> 1;
  R* X = (R*)smraw;
  R* Y = X + (size_t)cw * P;
  R* Z2 = Y + (size_t)cw * P;
  for (int idx = tid; idx < cw * ny; idx += nt) {
    const int ky = idx / cw, c = idx - ky * cw;
    X[c * P + ky] = Sv[(size_t)ky * nx + c0 + c];
  }
  __syncthreads();
  for (int idx = tid; idx < cw * half; idx += nt) {
    const int c = idx / half, m = idx - c * half;
    Y[c * P + m] = X[c * P + 2 * m];
    Y[c * P + ny - 1 - m] = X[c * P + 2 * m + 1];
  }
  __syncthreads();
  C* Z = smem_fft<C>((C*)Y, (C*)X, a.logny - 1, cw, P / 2, a.twy, ny, false);
  // DCT coefficients C[k] into Z2, times the symbol
  for (int idx = tid; idx < cw * (half + 1); idx += nt) {
    const int c = idx / (half + 1), k = idx - c * (half + 1);
    const C zk = Z[c * (P / 2) + (k & (half - 1))];
    const C zr = cconj(Z[c * (P / 2) + ((half - k) & (half - 1))]);
    const C dd = cmul(a.twy[k], csub(zk, zr));
    const C U = cmk<C>((R)0.5 * (zk.x + zr.x + dd.y), (R)0.5 * (zk.y + zr.y - dd.x));
    const int kx = c0 + c;
    Z2[c * P + k] = cmul(a.dcty[k], U).x * symbol(a, kx, k);
    if (k > 0 && k < half) Z2[c * P + ny - k] = cmulc(a.dcty[ny - k], U).x * symbol(a, kx, ny - k);
  }
  __syncthreads();
  // inverse: V[k] = e^{+i pi k/(2N)} (C_k - i C_{N-k}) -> half spectrum in X (complex)
  C* H = (C*)X;
  for (int idx = tid; idx < cw * (half + 1); idx += nt) {
    const int c = idx / (half + 1), k = idx - c * (half + 1);
    const R ck = Z2[c * P + k];
    const R cnk = k == 0 ? (R)0 : Z2[c * P + ny - k];
    H[c * (P / 2) + k] = cmulc(cmk<C>(ck, -cnk), a.dcty[k]);
  }
  __syncthreads();
  C* Zi = (C*)Y;
  for (int idx = tid; idx < cw * half; idx += nt) {
    const int c = idx / half, k = idx - c * half;
    const C xk = H[c * (P / 2) + k];
    const C xr = cconj(H[c * (P / 2) + half - k]);
    const C E = cmk<C>((R)0.5 * (xk.x + xr.x), (R)0.5 * (xk.y + xr.y));
    const C O = cmulc(cmk<C>((R)0.5 * (xk.x - xr.x), (R)0.5 * (xk.y - xr.y)), a.twy[k]);
    Zi[c * (P / 2) + k] = cmk<C>(E.x - O.y, E.y + O.x);
  }
  __syncthreads();
  R* u = (R*)smem_fft<C>(Zi, (C*)X, a.logny - 1, cw, P / 2, a.twy, ny, true);
  for (int idx = tid; idx < cw * ny; idx += nt) {
    const int ky = idx / cw, c = idx - ky * cw;
    const R val = (ky & 1) ? u[c * P + ny - 1 - (ky >> 1)] : u[c * P + (ky >> 1)];
    Sv[(size_t)ky * nx + c0 + c] = val;
  }
}

__global__ void k_logdet_partial(const double* lx, const double* ly, int nx, int ny, double kb, int power,
                                 double* part) {
  __shared__ double red[256];
  const size_t n = (size_t)nx * ny;
  const size_t per = (n + gridDim.x - 1) / gridDim.x;
  const size_t lo = per * blockIdx.x, hi = min(n, lo + per);
  double acc = 0.0;
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const int ky = (int)(i / nx), kx = (int)(i - (size_t)ky * nx);
    acc += log(kb + lx[kx] + ly[ky]);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = power * red[0];
}

__global__ void k_sum_partials(const double* part, int np, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < np; ++i) s += part[i];
    out[0] = s;
  }
}

int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

template <typename R>
PArgs<R> base_args(const PrecondTables& t, const Grid& g, const void* kappa2, double kc) {
  PArgs<R> a{};
  a.nx = t.nx;
  a.ny = t.ny;
  a.lognx = t.lognx;
  a.logny = t.logny;
  a.power = t.power;
  a.form = t.form;
  a.bc = g.bc;
  a.rb = t.rb;
  a.kbar2 = (R)t.kbar2;
  a.roff = t.form == FORM_DIAG ? (R)0 : (R)t.kbar2;
  const double norm = t.kind == GMRF_PREC_CIRCULANT ? 2.0 / ((double)t.nx * t.ny) : 4.0 / ((double)t.nx * t.ny);
  a.dscale = (R)norm;
  a.lamx = (const R*)t.lamx;
  a.lamy = (const R*)t.lamy;
  a.twx = (const typename Cplx<R>::T*)t.twx;
  a.twy = (const typename Cplx<R>::T*)t.twy;
  a.dctx = (const typename Cplx<R>::T*)t.dctx;
  a.dcty = (const typename Cplx<R>::T*)t.dcty;
  a.S = (R*)t.S;
  a.sstride = (size_t)t.ny * (t.nx + 2);
  a.G = (R*)t.G;
  a.Wg = (R*)t.Wg;
  a.kappa2 = (const float*)kappa2;
  a.kappa2_const = t.form == FORM_DIAG ? (R)0 : (R)kc;  // FORM_DIAG without a field: D = 0
  a.n = g.n;
  return a;
}

int col_width(const PrecondTables& t) {
  const int budget = t.fp64 ? 2048 : 4096;
  int cw = budget / t.ny;
  if (t.kind == GMRF_PREC_MIRROR) cw *= 2;
  if (cw < 1) cw = 1;
  if (cw > 16) cw = 16;
  const int ncols = t.kind == GMRF_PREC_CIRCULANT ? t.nx / 2 + 1 : t.nx;
  while (cw > 1 && cw > ncols) cw >>= 1;
  return cw;
}

bool host_has_edge_terms(const PrecondTables& t) {
  return t.kind == GMRF_PREC_CIRCULANT ? t.bc != GMRF_BC_PERIODIC : t.bc != GMRF_BC_NEUMANN;
}
// must match the line count LMAX of k_prow
template <typename R>
size_t row_smem(const PrecondTables& t) {
  return (size_t)4 * (t.rb + (host_has_edge_terms(t) ? 2 : 0)) * (t.nx + 2) * sizeof(R);
}
template <typename R>
size_t col_smem(const PrecondTables& t, int cw) {
  if (t.kind == GMRF_PREC_CIRCULANT) return (size_t)2 * cw * (t.ny + 1) * 2 * sizeof(R);
  return (size_t)3 * cw * (t.ny + 2) * sizeof(R);
}

int ensure_ws(PrecondTables& t, int nvec, cudaStream_t st) {
  const size_t es = t.fp64 ? 8 : 4;
  const size_t sb = (size_t)nvec * t.ny * (t.nx + 2) * es;
  const size_t gb = t.form == FORM_CTC ? (size_t)nvec * t.nx * t.ny * es : 16;
  if (t.S_bytes < sb) {
    if (t.S) cudaFreeAsync(t.S, st);
    t.S = nullptr;
    t.S_bytes = 0;
    if (cudaMallocAsync(&t.S, sb, st) != cudaSuccess) return -1;
    t.S_bytes = sb;
  }
  if (t.G_bytes < gb) {
    if (t.G) cudaFreeAsync(t.G, st);
    t.G = nullptr;
    t.G_bytes = 0;
    if (cudaMallocAsync(&t.G, gb, st) != cudaSuccess) return -1;
    t.G_bytes = gb;
  }
  const bool edges = t.kind == GMRF_PREC_CIRCULANT ? t.bc != GMRF_BC_PERIODIC : t.bc != GMRF_BC_NEUMANN;
  const size_t wb = edges ? (size_t)nvec * t.nx * t.ny * es : 16;
  if (t.Wg_bytes < wb) {
    if (t.Wg) cudaFreeAsync(t.Wg, st);
    t.Wg = nullptr;
    t.Wg_bytes = 0;
    if (cudaMallocAsync(&t.Wg, wb, st) != cudaSuccess) return -1;
    t.Wg_bytes = wb;
  }
  return 0;
}

// R has y-boundary terms (the boundaries of M and Q differ): the middle pass
// needs the w rows of other blocks (M_MIDW + M_MIDG).
bool generic_edges(const PrecondTables& t) {
  return t.kind == GMRF_PREC_CIRCULANT ? t.bc != GMRF_BC_PERIODIC : t.bc != GMRF_BC_NEUMANN;
}

fast::Args fast_args(const PrecondTables& t, const Grid& g, const void* kappa2, double kc) {
  fast::Args a{};
  a.nx = t.nx;
  a.ny = t.ny;
  a.bc = g.bc;
  a.power = t.power;
  a.form = t.form;
  a.kbar2 = (float)t.kbar2;
  a.roff = t.form == FORM_DIAG ? 0.f : (float)t.kbar2;
  a.dscale = (float)(t.kind == GMRF_PREC_CIRCULANT ? 2.0 / ((double)t.nx * t.ny) : 4.0 / ((double)t.nx * t.ny));
  a.lamx = (const float*)t.lamx;
  a.lamy = (const float*)t.lamy;
  a.twx = (const float2*)t.twx;
  a.twy = (const float2*)t.twy;
  a.dctx = (const float2*)t.dctx;
  a.dcty = (const float2*)t.dcty;
  a.pairx = (const float4*)t.pairx;
  a.pairy = (const float4*)t.pairy;
  a.T = (float*)t.S;
  a.tstride = (size_t)t.ny * (t.nx + 2);
  a.G = (float*)t.G;
  a.Wg = (float*)t.Wg;
  a.kappa2 = (const float*)kappa2;
  a.kappa2_const = t.form == FORM_DIAG ? 0.f : (float)kc;  // FORM_DIAG without a field: D = 0
  a.n = g.n;
  return a;
}

int smem_optin() {
  static const int v = [] {  // thread-safe one-time initialisation
    int dev = 0, r = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&r, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      r = 48 * 1024;
    }
    return r;
  }();
  return v;
}

// Raise the dynamic shared memory limit of a kernel once per process.
template <typename K>
cudaError_t allow_smem(K* k, std::atomic<bool>& done) {
  if (done.load(std::memory_order_acquire)) return cudaSuccess;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin() - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.store(true, std::memory_order_release);
  return e;
}

template <typename R, int KIND, int MODE>
cudaError_t row_attr() {
  static std::atomic<bool> done{false};
  return allow_smem(k_prow<R, KIND, MODE>, done);
}
template <typename R, int KIND>
cudaError_t col_attr() {
  static std::atomic<bool> done{false};
  return allow_smem(k_pcol<R, KIND>, done);
}

template <typename R, int KIND, int MODE>
cudaError_t row_launch(const PrecondTables& t, const PArgs<R>& a, int nvec, cudaStream_t s, int kc) {
  const size_t sm = row_smem<R>(t);
  cudaError_t e = row_attr<R, KIND, MODE>();
  if (e != cudaSuccess) return e;
  dim3 grd(t.ny / t.rb, nvec);
  trace_begin(kc, s);
  k_prow<R, KIND, MODE><<<grd, 256, sm, s>>>(a);
  trace_end(kc, s);
  return cudaGetLastError();
}

template <typename R, int KIND>
cudaError_t col_launch(const PrecondTables& t, PArgs<R> a, int nvec, int step_mode, cudaStream_t s, int kc) {
  const int cw = col_width(t);
  a.cw = cw;
  const size_t sm = col_smem<R>(t, cw);
  cudaError_t e = col_attr<R, KIND>();
  if (e != cudaSuccess) return e;
  const int ncols = KIND == GMRF_PREC_CIRCULANT ? t.nx / 2 + 1 : t.nx;
  dim3 grd((ncols + cw - 1) / cw, nvec);
  trace_begin(kc, s);
  k_pcol<R, KIND><<<grd, 256, sm, s>>>(a, step_mode);
  trace_end(kc, s);
  return cudaGetLastError();
}

#define CKE(x)                            \
  do {                                    \
    cudaError_t e_ = (x);                 \
    if (e_ != cudaSuccess) return e_;     \
  } while (0)

template <typename R, int KIND>
cudaError_t run_step(PrecondTables& t, const Grid& g, const void* kappa2, double kc, const LanczosBufs& b,
                     const StepParams& P, cudaStream_t s) {
  if (ensure_ws(t, b.nvec, s)) return cudaErrorMemoryAllocation;
  if (t.fast) {
    fast::Args a = fast_args(t, g, kappa2, kc);
    a.W0 = (float*)b.W[0];
    a.W1 = (float*)b.W[1];
    a.V = (float*)b.V;
    a.P = P;
    a.st = b.st;
    a.alpha = b.alpha;
    a.beta = b.beta;
    a.alpha_f = b.alpha_f;
    a.beta2_f = b.beta2_f;
    a.partials = (Dots<float>*)b.partials;
    a.counters = b.counters;
    a.in = nullptr;
    return KIND == GMRF_PREC_CIRCULANT ? fast_step_circ(a, b.nvec, s) : fast_step_mirror(a, b.nvec, s);
  }
  PArgs<R> a = base_args<R>(t, g, kappa2, kc);
  a.G = (R*)t.G;
  a.S = (R*)t.S;
  a.W0 = (R*)b.W[0];
  a.W1 = (R*)b.W[1];
  a.V = (R*)b.V;
  a.P = P;
  a.st = b.st;
  a.alpha = b.alpha;
  a.beta = b.beta;
  a.alpha_f = b.alpha_f;
  a.beta2_f = b.beta2_f;
  a.partials = (Dots<R>*)b.partials;
  a.counters = b.counters;
  a.in = nullptr;
  CKE((row_launch<R, KIND, M_FWD_FORM>(t, a, b.nvec, s, KC_PRE_ROW_FWD)));
  CKE((col_launch<R, KIND>(t, a, b.nvec, 1, s, KC_PRE_COL)));
  if (generic_edges(t)) {
    CKE((row_launch<R, KIND, M_MIDW>(t, a, b.nvec, s, KC_PRE_ROW_MID)));
    CKE((row_launch<R, KIND, M_MIDG>(t, a, b.nvec, s, KC_PRE_ROW_MID)));
  } else {
    CKE((row_launch<R, KIND, M_MID>(t, a, b.nvec, s, KC_PRE_ROW_MID)));
  }
  CKE((col_launch<R, KIND>(t, a, b.nvec, 1, s, KC_PRE_COL)));
  CKE((row_launch<R, KIND, M_LAST>(t, a, b.nvec, s, KC_PRE_ROW_LAST)));
  return cudaSuccess;
}

// Sbuf: spectrum workspace (nullptr = the tables' own, grown on demand)
template <typename R, int KIND>
cudaError_t run_apply(PrecondTables& t, const Grid& g, const void* in, void* out, int nvec, cudaStream_t s,
                      void* Sbuf = nullptr) {
  if (!Sbuf && ensure_ws(t, nvec, s)) return cudaErrorMemoryAllocation;
  void* S = Sbuf ? Sbuf : t.S;
  if (t.fast) {
    fast::Args a = fast_args(t, g, nullptr, 0.0);
    a.T = (float*)S;
    a.in = (const float*)in;
    a.out = (float*)out;
    return KIND == GMRF_PREC_CIRCULANT ? fast_apply_circ(a, nvec, s) : fast_apply_mirror(a, nvec, s);
  }
  PArgs<R> a = base_args<R>(t, g, nullptr, 0.0);
  a.S = (R*)S;
  a.in = (const R*)in;
  a.out = (R*)out;
  CKE((row_launch<R, KIND, M_FWD_PLAIN>(t, a, nvec, s, KC_PRE_APPLY)));
  CKE((col_launch<R, KIND>(t, a, nvec, 0, s, KC_PRE_APPLY)));
  CKE((row_launch<R, KIND, M_INV_PLAIN>(t, a, nvec, s, KC_PRE_APPLY)));
  return cudaSuccess;
}

template <typename R, int KIND>
cudaError_t run_operator(PrecondTables& t, const Grid& g, const void* kappa2, double kc, const void* v, void* y,
                         int nvec, cudaStream_t s) {
  if (ensure_ws(t, nvec, s)) return cudaErrorMemoryAllocation;
  if (t.fast) {
    fast::Args a = fast_args(t, g, kappa2, kc);
    a.in = (const float*)v;
    a.out = (float*)y;
    return KIND == GMRF_PREC_CIRCULANT ? fast_operator_circ(a, nvec, s) : fast_operator_mirror(a, nvec, s);
  }
  PArgs<R> a = base_args<R>(t, g, kappa2, kc);
  a.S = (R*)t.S;
  a.G = (R*)t.G;
  a.in = (const R*)v;
  a.out = (R*)y;
  CKE((row_launch<R, KIND, M_FWD_PLAIN>(t, a, nvec, s, KC_PRE_APPLY)));
  CKE((col_launch<R, KIND>(t, a, nvec, 0, s, KC_PRE_APPLY)));
  if (generic_edges(t)) {
    CKE((row_launch<R, KIND, M_MIDW>(t, a, nvec, s, KC_PRE_APPLY)));
    CKE((row_launch<R, KIND, M_MIDG>(t, a, nvec, s, KC_PRE_APPLY)));
  } else {
    CKE((row_launch<R, KIND, M_MID>(t, a, nvec, s, KC_PRE_APPLY)));
  }
  CKE((col_launch<R, KIND>(t, a, nvec, 0, s, KC_PRE_APPLY)));
  CKE((row_launch<R, KIND, M_LAST_PLAIN>(t, a, nvec, s, KC_PRE_APPLY)));
  return cudaSuccess;
}

template <typename R, int KIND>
cudaError_t set_attrs() {
  cudaError_t e;
  if ((e = row_attr<R, KIND, M_FWD_PLAIN>()) != cudaSuccess) return e;
  if ((e = row_attr<R, KIND, M_FWD_FORM>()) != cudaSuccess) return e;
  if ((e = row_attr<R, KIND, M_INV_PLAIN>()) != cudaSuccess) return e;
  if ((e = row_attr<R, KIND, M_MID>()) != cudaSuccess) return e;
  if ((e = row_attr<R, KIND, M_MIDW>()) != cudaSuccess) return e;
  if ((e = row_attr<R, KIND, M_MIDG>()) != cudaSuccess) return e;
  if ((e = row_attr<R, KIND, M_LAST>()) != cudaSuccess) return e;
  if ((e = row_attr<R, KIND, M_LAST_PLAIN>()) != cudaSuccess) return e;
  return col_attr<R, KIND>();
}

template <typename R>
int upload_tables(PrecondTables& t, cudaStream_t s, std::vector<double>& lx64, std::vector<double>& ly64) {
  typedef typename Cplx<R>::T C;
  const double pi = 3.14159265358979323846;
  auto lam = [&](int N, std::vector<double>& out) {
    out.resize(N);
    for (int k = 0; k < N; ++k) {
      const double th = t.kind == GMRF_PREC_CIRCULANT ? 2.0 * pi * k / N : pi * k / N;
      out[k] = 2.0 - 2.0 * std::cos(th);
    }
  };
  lam(t.nx, lx64);
  lam(t.ny, ly64);
  auto up = [&](void** dst, const void* src, size_t bytes) -> int {
    if (cudaMallocAsync(dst, bytes, s) != cudaSuccess) return -1;
    if (cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return -1;
    return 0;
  };
  std::vector<R> lxr(lx64.begin(), lx64.end()), lyr(ly64.begin(), ly64.end());
  auto tw = [&](int N, std::vector<C>& out) {
    out.resize(N);
    for (int k = 0; k < N; ++k) {
      out[k].x = (R)std::cos(2.0 * pi * k / N);
      out[k].y = (R)-std::sin(2.0 * pi * k / N);
    }
  };
  auto dct = [&](int N, std::vector<C>& out) {
    out.resize(N + 1);
    for (int k = 0; k <= N; ++k) {
      out[k].x = (R)std::cos(pi * k / (2.0 * N));
      out[k].y = (R)-std::sin(pi * k / (2.0 * N));
    }
  };
  std::vector<C> twx, twy, dx, dy;
  tw(t.nx, twx);
  tw(t.ny, twy);
  dct(t.nx, dx);
  dct(t.ny, dy);
  if (up(&t.lamx, lxr.data(), lxr.size() * sizeof(R)) || up(&t.lamy, lyr.data(), lyr.size() * sizeof(R)) ||
      up(&t.twx, twx.data(), twx.size() * sizeof(C)) || up(&t.twy, twy.data(), twy.size() * sizeof(C)) ||
      up(&t.dctx, dx.data(), dx.size() * sizeof(C)) || up(&t.dcty, dy.data(), dy.size() * sizeof(C)))
    return -1;
  // pair planes of the FP32 mirror passes (the same float values, regrouped)
  auto planes = [&](int N, const std::vector<C>& tw_, const std::vector<C>& d_, const std::vector<R>* lam_,
                    std::vector<R>& pr) {
    const int L = N / 2, HP = L / 2, np = lam_ ? 4 : 3;
    pr.assign((size_t)np * (HP + 1) * 4, (R)0);
    for (int k = 0; k <= HP; ++k) {
      const int kp = L - k;
      // entry q of pair k at float (q / 4) * 4 (HP + 1) + 4 k + q % 4
      auto at = [&](int q) -> R& { return pr[(size_t)(q / 4) * 4 * (HP + 1) + (size_t)4 * k + q % 4]; };
      const C v[6] = {tw_[k], tw_[kp], d_[k], d_[N - k], d_[kp], d_[N - kp]};
      for (int q = 0; q < 6; ++q) {
        at(2 * q) = v[q].x;
        at(2 * q + 1) = v[q].y;
      }
      if (!lam_) continue;
      const std::vector<R>& lm = *lam_;
      if (k == 0) {
        at(12) = lm[0];
        at(13) = lm[L];
      } else {
        at(12) = lm[k];
        at(13) = lm[N - k];
        at(14) = lm[kp];
        at(15) = lm[N - kp];
      }
    }
  };
  std::vector<R> prx, pry;
  if (sizeof(R) == 4 && t.kind == GMRF_PREC_MIRROR && t.nx >= 4 && t.ny >= 4) {
    planes(t.nx, twx, dx, nullptr, prx);
    planes(t.ny, twy, dy, &lyr, pry);
    if (up(&t.pairx, prx.data(), prx.size() * sizeof(R)) || up(&t.pairy, pry.data(), pry.size() * sizeof(R)))
      return -1;
  }
  // host vectors must outlive the async copies
  return cudaStreamSynchronize(s) == cudaSuccess ? 0 : -1;
}

}  // namespace

bool precond_size_ok(int64_t n) {
  if (n < 8 || n > 4096) return false;
  return (n & (n - 1)) == 0;
}

int precond_build(PrecondTables& t, const Grid& g, int kind, int op, double kbar2, bool fp64, cudaStream_t s,
                  double* logdet_M) {
  t.kind = kind;
  t.power = op == GMRF_OP_SHIFTED_LAPLACIAN ? 1 : 2;
  t.form = op == GMRF_OP_SHIFTED_LAPLACIAN ? FORM_SHIFT : (op == GMRF_OP_SPDE_SQUARED ? FORM_CTC : FORM_DIAG);
  t.nx = g.nx;
  t.ny = g.ny;
  t.lognx = ilog2(g.nx);
  t.logny = ilog2(g.ny);
  t.fp64 = fp64;
  t.kbar2 = kbar2;
  t.bc = g.bc;
  t.fast = fast_eligible(kind, fp64, g.nx, g.ny);
  int rb = (fp64 ? 2048 : 4096) / g.nx;
  if (rb < 1) rb = 1;
  if (rb > 16) rb = 16;
  if (rb > g.ny) rb = g.ny;
  t.rb = rb;
  // the generic row and column kernels stage whole lines in shared memory
  // (FP64 4096-point lines fit only without the y-partner rows of edge terms)
  {
    const size_t lim = (size_t)smem_optin() - 2048;
    const size_t rs = fp64 ? row_smem<double>(t) : row_smem<float>(t);
    const int cw = col_width(t);
    const size_t cs = fp64 ? col_smem<double>(t, cw) : col_smem<float>(t, cw);
    if (rs > lim || cs > lim) return GMRF_ERR_UNSUPPORTED;
  }
  std::vector<double> lx64, ly64;
  const int r = fp64 ? upload_tables<double>(t, s, lx64, ly64) : upload_tables<float>(t, s, lx64, ly64);
  if (r) return GMRF_ERR_CUDA;
  // log det of B_bar^p (tau-free), FP64 on the device
  double *dlx = nullptr, *dly = nullptr, *part = nullptr;
  const int np = 256;
  double h = 0.0;
  bool ok = cudaMallocAsync(&dlx, sizeof(double) * t.nx, s) == cudaSuccess &&
            cudaMallocAsync(&dly, sizeof(double) * t.ny, s) == cudaSuccess &&
            cudaMallocAsync(&part, sizeof(double) * (np + 1), s) == cudaSuccess &&
            cudaMemcpyAsync(dlx, lx64.data(), sizeof(double) * t.nx, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(dly, ly64.data(), sizeof(double) * t.ny, cudaMemcpyHostToDevice, s) == cudaSuccess;
  if (ok) {
    k_logdet_partial<<<np, 256, 0, s>>>(dlx, dly, t.nx, t.ny, kbar2, t.power, part);
    k_sum_partials<<<1, 32, 0, s>>>(part, np, part + np);
    ok = cudaGetLastError() == cudaSuccess &&
         cudaMemcpyAsync(&h, part + np, sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
         cudaStreamSynchronize(s) == cudaSuccess;
  }
  if (dlx) cudaFreeAsync(dlx, s);
  if (dly) cudaFreeAsync(dly, s);
  if (part) cudaFreeAsync(part, s);
  if (!ok) {
    cudaGetLastError();
    return GMRF_ERR_CUDA;
  }
  *logdet_M = h;
  return GMRF_OK;
}

void precond_free(PrecondTables& t, cudaStream_t s) {
  void* ps[] = {t.lamx, t.lamy, t.twx, t.twy, t.dctx, t.dcty, t.pairx, t.pairy, t.S, t.G, t.Wg};
  for (void* p : ps)
    if (p) cudaFreeAsync(p, s);
  t = PrecondTables();
}

int precond_blocks_per_vector(const PrecondTables& t) {
  if (!t.nx) return 0;
  int nb = t.ny / t.rb;
  if (t.fast) nb = std::max(nb, t.ny / fast_rows_per_block(t.kind, t.nx));
  return nb;
}

int precond_prepare(PrecondTables& t, int nvec, cudaStream_t s) {
  if (ensure_ws(t, nvec, s)) return GMRF_ERR_OOM;
  cudaError_t e;
  if (t.fp64) e = t.kind == GMRF_PREC_CIRCULANT ? set_attrs<double, GMRF_PREC_CIRCULANT>()
                                               : set_attrs<double, GMRF_PREC_MIRROR>();
  else e = t.kind == GMRF_PREC_CIRCULANT ? set_attrs<float, GMRF_PREC_CIRCULANT>()
                                         : set_attrs<float, GMRF_PREC_MIRROR>();
  return e == cudaSuccess ? GMRF_OK : GMRF_ERR_CUDA;
}

size_t precond_extra_bytes(const PrecondTables& t, size_t es) {
  // spectrum, g = C v, and w when R has y-boundary terms
  return (size_t)t.ny * (t.nx + 2) * es + (size_t)t.nx * t.ny * es +
         (generic_edges(t) ? (size_t)t.nx * t.ny * es : 0);
}

cudaError_t launch_precond_step(PrecondTables& t, const Grid& g, bool fp64, const void* kappa2, double kappa2_const,
                                const LanczosBufs& b, const StepParams& P, cudaStream_t s) {
  if (fp64) {
    if (t.kind == GMRF_PREC_CIRCULANT) return run_step<double, GMRF_PREC_CIRCULANT>(t, g, kappa2, kappa2_const, b, P, s);
    return run_step<double, GMRF_PREC_MIRROR>(t, g, kappa2, kappa2_const, b, P, s);
  }
  if (t.kind == GMRF_PREC_CIRCULANT) return run_step<float, GMRF_PREC_CIRCULANT>(t, g, kappa2, kappa2_const, b, P, s);
  return run_step<float, GMRF_PREC_MIRROR>(t, g, kappa2, kappa2_const, b, P, s);
}

cudaError_t launch_precond_apply(PrecondTables& t, const Grid& g, bool fp64, int which, const void* in, void* out,
                                 int nvec, cudaStream_t s) {
  (void)which;
  if (fp64) {
    if (t.kind == GMRF_PREC_CIRCULANT) return run_apply<double, GMRF_PREC_CIRCULANT>(t, g, in, out, nvec, s);
    return run_apply<double, GMRF_PREC_MIRROR>(t, g, in, out, nvec, s);
  }
  if (t.kind == GMRF_PREC_CIRCULANT) return run_apply<float, GMRF_PREC_CIRCULANT>(t, g, in, out, nvec, s);
  return run_apply<float, GMRF_PREC_MIRROR>(t, g, in, out, nvec, s);
}

size_t precond_apply_scratch_bytes(const PrecondTables& t, int nvec) {
  return (size_t)nvec * t.ny * (t.nx + 2) * (t.fp64 ? 8 : 4);
}

cudaError_t launch_precond_apply_with(PrecondTables& t, const Grid& g, bool fp64, const void* in, void* out, int nvec,
                                      void* S, cudaStream_t s) {
  if (!S) return cudaErrorInvalidValue;
  if (fp64) {
    if (t.kind == GMRF_PREC_CIRCULANT) return run_apply<double, GMRF_PREC_CIRCULANT>(t, g, in, out, nvec, s, S);
    return run_apply<double, GMRF_PREC_MIRROR>(t, g, in, out, nvec, s, S);
  }
  if (t.kind == GMRF_PREC_CIRCULANT) return run_apply<float, GMRF_PREC_CIRCULANT>(t, g, in, out, nvec, s, S);
  return run_apply<float, GMRF_PREC_MIRROR>(t, g, in, out, nvec, s, S);
}

cudaError_t launch_precond_operator(PrecondTables& t, const Grid& g, bool fp64, const void* kappa2,
                                    double kappa2_const, const void* v, void* y, int nvec, cudaStream_t s) {
  if (fp64) {
    if (t.kind == GMRF_PREC_CIRCULANT)
      return run_operator<double, GMRF_PREC_CIRCULANT>(t, g, kappa2, kappa2_const, v, y, nvec, s);
    return run_operator<double, GMRF_PREC_MIRROR>(t, g, kappa2, kappa2_const, v, y, nvec, s);
  }
  if (t.kind == GMRF_PREC_CIRCULANT)
    return run_operator<float, GMRF_PREC_CIRCULANT>(t, g, kappa2, kappa2_const, v, y, nvec, s);
  return run_operator<float, GMRF_PREC_MIRROR>(t, g, kappa2, kappa2_const, v, y, nvec, s);
}

}  // namespace gmrf
