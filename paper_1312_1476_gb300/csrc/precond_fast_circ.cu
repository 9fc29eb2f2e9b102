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

// rows per block of the row kernels (the device layout's own rule)
template <int KIND>
static int rows_for(int nx) {
  switch (nx) {
    case 128: return fast::rows_per_block<KIND, 6>();
    case 256: return fast::rows_per_block<KIND, 7>();
    case 512: return fast::rows_per_block<KIND, 8>();
    case 1024: return fast::rows_per_block<KIND, 9>();
    case 2048: return fast::rows_per_block<KIND, 10>();
    default: return 1;
  }
}

int fast_rows_per_block(int kind, int nx) {
  return kind == GMRF_PREC_MIRROR ? rows_for<GMRF_PREC_MIRROR>(nx) : rows_for<GMRF_PREC_CIRCULANT>(nx);
}

}  // namespace gmrf
