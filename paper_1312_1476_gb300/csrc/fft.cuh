// fft.cuh -- shared-memory transforms for the fast preconditioner apply
// (Section 2: block-circulant matrices are diagonalised by FFTs; Section 5.1).
//
// * smem_fft: batched complex FFT of power-of-two length N on lines held in
//   shared memory (Stockham autosort, radix 2, natural order in and out), all
//   threads of the block cooperating.  Twiddles come from a table
//   tw[t] = exp(-2 pi i t / TN) in global memory, TN a multiple of N.
// * real transforms of length N built on a half-length complex FFT:
//     R2C  X[k] = (Z[k] + conj Z[N/2-k])/2 - i W_N^k (Z[k] - conj Z[N/2-k])/2,
//          z[m] = x[2m] + i x[2m+1], Z = FFT_{N/2}(z), k = 0..N/2;
//     C2R  Z[k] = E[k] + i O[k], E = (X[k] + conj X[N/2-k])/2,
//          O = (X[k] - conj X[N/2-k]) / (2 W_N^k), z = IFFT_{N/2}(Z) (unnormalised),
//          x[2m] = Re z[m], x[2m+1] = Im z[m]   (= (N/2) x);
//     DCT-II (Makhoul): u[m] = x[2m], u[N-1-m] = x[2m+1], U = R2C(u),
//          C[k] = Re(e^{-i pi k/(2N)} U[k]) = sum_n x_n cos(pi k (2n+1)/(2N));
//     inverse: V[k] = e^{i pi k/(2N)} (C[k] - i C[N-k]) (C[N] = 0),
//          u = C2R(V) (= (N/2) u), x[2m] = u[m], x[2m+1] = u[N-1-m].
#pragma once

#include <cuda_runtime.h>

namespace gmrf {

template <typename R>
struct Cplx;
template <>
struct Cplx<float> {
  typedef float2 T;
};
template <>
struct Cplx<double> {
  typedef double2 T;
};

template <typename C>
__device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) {
  C r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) { return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C>
__device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
  return cmk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C>
__device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }

__device__ __forceinline__ int block_tid() { return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z); }
__device__ __forceinline__ int block_nt() { return blockDim.x * blockDim.y * blockDim.z; }

// Batched in-place-by-pointer FFT: lines l = 0..nlines-1 at buf[l*pitch + k].
// Returns the buffer (buf or tmp) holding the result.  inv: conjugate twiddles
// (unnormalised inverse).  Ends with a __syncthreads().
template <typename C>
__device__ C* smem_fft(C* buf, C* tmp, int logN, int nlines, int pitch, const C* __restrict__ tw, int TN, bool inv) {
  const int tid = block_tid(), nt = block_nt();
  const int N = 1 << logN, half = N >> 1;
  C* in = buf;
  C* out = tmp;
  for (int lNs = 0; lNs < logN; ++lNs) {
    const int Ns = 1 << lNs;
    const int tws = TN >> (lNs + 1);  // TN / (2 Ns)
    const int total = nlines << (logN - 1);
    for (int idx = tid; idx < total; idx += nt) {
      const int l = idx >> (logN - 1);
      const int jj = idx & (half - 1);
      const int k = jj & (Ns - 1);
      const C a = in[l * pitch + jj];
      const C b = in[l * pitch + jj + half];
      C w = tw[k * tws];
      if (inv) w.y = -w.y;
      const C bw = cmul(b, w);
      const int o = ((jj - k) << 1) + k;
      out[l * pitch + o] = cadd(a, bw);
      out[l * pitch + o + Ns] = csub(a, bw);
    }
    __syncthreads();
    C* t = in;
    in = out;
    out = t;
  }
  return in;
}

}  // namespace gmrf
