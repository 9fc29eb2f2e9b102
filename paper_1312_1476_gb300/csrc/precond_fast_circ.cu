// precond_fast_circ.cu -- instantiation of the FP32 register-FFT kernels for
// the circulant (torus) preconditioner.
#include "precond_fast.cuh"
#include "precond_fast.h"

namespace gmrf {

cudaError_t fast_step_circ(const fast::Args& a, int nvec, cudaStream_t s) {
  return fast::step_k<GMRF_PREC_CIRCULANT>(a, nvec, s);
}
cudaError_t fast_apply_circ(const fast::Args& a, int nvec, cudaStream_t s) {
  return fast::apply_k<GMRF_PREC_CIRCULANT>(a, nvec, s);
}
cudaError_t fast_operator_circ(const fast::Args& a, int nvec, cudaStream_t s) {
  return fast::operator_k<GMRF_PREC_CIRCULANT>(a, nvec, s);
}

bool fast_eligible(int kind, bool fp64, int nx, int ny) {
  auto p2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  if (fp64 || !p2(nx) || !p2(ny) || nx < 128 || nx > 2048) return false;
  if (kind == GMRF_PREC_CIRCULANT) return ny >= 64 && ny <= 1024;
  return ny >= 128 && ny <= 2048;
}

int fast_rows_per_block(int kind, int nx) {
  const int L = nx / 2, E = L / 32, G = 32 / E;
  const int seg = kind == GMRF_PREC_MIRROR ? 8 : 4;
  return G > seg ? G : seg;
}

}  // namespace gmrf
