// Double-float instantiations of the FFT propagator kernels: FP64 operand and
// tables in HBM, every butterfly and block multiply in df64 arithmetic on the
// FP32 units.
#include "prop_impl.cuh"

namespace dq {
cudaError_t launch_prop_df(int L, int side, const double *X, double *Y, int nvec, int ld,
                           const cpx<df64> *E, const double *pre, const double *post,
                           const double *vscale, cudaStream_t st) {
  return launch_prop<df64>(L, side, X, Y, nvec, ld, E, pre, post, vscale, st);
}
}  // namespace dq
