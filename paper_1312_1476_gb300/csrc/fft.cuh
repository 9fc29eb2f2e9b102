// fft.cuh -- shared-memory transforms for the fast preconditioner apply
// (Section 2: block-circulant matrices are diagonalised by FFTs; Section 5.1).
//
// * smem_fft: batched complex FFT of power-of-two length N on lines held in
//   shared memory (Stockham autosort, radix 8 with a radix-4/2 remainder pass,
//   natural order in and out), all
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

// R-point DFT of v[0..R) in registers (R = 2, 4, 8); inv: e^{+i} kernel.
template <typename C>
__device__ __forceinline__ void dft2(C& a, C& b) {
  const C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}
// multiply by -i (forward) or +i (inverse)
template <typename C>
__device__ __forceinline__ C rot90(C a, bool inv) {
  return inv ? cmk<C>(-a.y, a.x) : cmk<C>(a.y, -a.x);
}
template <typename C>
__device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3, bool inv) {
  const C t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), t3 = rot90(csub(v1, v3), inv);
  v0 = cadd(t0, t2);
  v2 = csub(t0, t2);
  v1 = cadd(t1, t3);
  v3 = csub(t1, t3);
}
template <typename C>
__device__ __forceinline__ void dft8(C* v, bool inv) {
  typedef decltype(C::x) R;
  const R h = (R)0.70710678118654752440;
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4(e0, e1, e2, e3, inv);
  dft4(o0, o1, o2, o3, inv);
  // twiddles W8^k, k = 1..3: forward (1 - i)/sqrt2, -i, -(1 + i)/sqrt2
  const C w1 = inv ? cmk<C>(h * (o1.x - o1.y), h * (o1.x + o1.y)) : cmk<C>(h * (o1.x + o1.y), h * (o1.y - o1.x));
  const C w2 = rot90(o2, inv);
  const C w3 = inv ? cmk<C>(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : cmk<C>(h * (o3.y - o3.x), -h * (o3.x + o3.y));
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, w1);
  v[5] = csub(e1, w1);
  v[2] = cadd(e2, w2);
  v[6] = csub(e2, w2);
  v[3] = cadd(e3, w3);
  v[7] = csub(e3, w3);
}

// One Stockham pass of radix RAD on lines of length N = 2^logN; Ns = product
// of the radices of the previous passes.  Twiddles W_{Ns*RAD}^{r k} come from
// tw[t] = exp(-2 pi i t / TN).
template <int RAD, typename C>
__device__ __forceinline__ void stockham_pass(const C* in, C* out, int logN, int lNs, int nlines, int pitch,
                                              const C* __restrict__ tw, int TN, bool inv) {
  const int tid = block_tid(), nt = block_nt();
  constexpr int LR = RAD == 8 ? 3 : (RAD == 4 ? 2 : 1);
  const int lnb = logN - LR;  // log2 of butterflies per line
  const int nbf = 1 << lnb;
  const int Ns = 1 << lNs;
  const int tws = TN >> (lNs + LR);  // TN / (Ns * RAD)
  const int total = nlines << lnb;
  for (int idx = tid; idx < total; idx += nt) {
    const int l = idx >> lnb;
    const int jj = idx & (nbf - 1);
    const int k = jj & (Ns - 1);
    const C* src = in + l * pitch + jj;
    C v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = src[r << lnb];
    if (lNs > 0) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        C w = tw[r * k * tws];
        if (inv) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    if (RAD == 8) dft8(v, inv);
    else if (RAD == 4) dft4(v[0], v[1], v[2], v[3], inv);
    else dft2(v[0], v[1]);
    C* dst = out + l * pitch + ((jj - k) << LR) + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) dst[r << lNs] = v[r];
  }
}

// Batched FFT: lines l = 0..nlines-1 at buf[l*pitch + k], k < 2^logN.
// Radix-8 passes, then one radix-4 or radix-2 pass for the remainder.
// Returns the buffer (buf or tmp) holding the result; ends synchronised.
template <typename C>
__device__ C* smem_fft(C* buf, C* tmp, int logN, int nlines, int pitch, const C* __restrict__ tw, int TN, bool inv) {
  C* in = buf;
  C* out = tmp;
  int lNs = 0;
  while (lNs < logN) {
    const int rem = logN - lNs;
    if (rem >= 3) {
      stockham_pass<8>(in, out, logN, lNs, nlines, pitch, tw, TN, inv);
      lNs += 3;
    } else if (rem == 2) {
      stockham_pass<4>(in, out, logN, lNs, nlines, pitch, tw, TN, inv);
      lNs += 2;
    } else {
      stockham_pass<2>(in, out, logN, lNs, nlines, pitch, tw, TN, inv);
      lNs += 1;
    }
    __syncthreads();
    C* t = in;
    in = out;
    out = t;
  }
  return in;
}

}  // namespace gmrf
