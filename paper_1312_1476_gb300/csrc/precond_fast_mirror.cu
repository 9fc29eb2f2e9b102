// precond_fast_mirror.cu -- instantiation of the FP32 register-FFT kernels for
// the mirror-extended (DCT-II) preconditioner.
#include "precond_fast.cuh"
#include "precond_fast.h"

namespace gmrf {

cudaError_t fast_step_mirror(const fast::Args& a, int nvec, cudaStream_t s) {
  return fast::step_k<GMRF_PREC_MIRROR>(a, nvec, s);
}
cudaError_t fast_apply_mirror(const fast::Args& a, int nvec, cudaStream_t s) {
  return fast::apply_k<GMRF_PREC_MIRROR>(a, nvec, s);
}
cudaError_t fast_operator_mirror(const fast::Args& a, int nvec, cudaStream_t s) {
  return fast::operator_k<GMRF_PREC_MIRROR>(a, nvec, s);
}

}  // namespace gmrf
