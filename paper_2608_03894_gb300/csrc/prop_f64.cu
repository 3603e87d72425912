// FP64 instantiations of the FFT propagator kernels.
#include "prop_impl.cuh"

namespace dq {
cudaError_t launch_prop_f64(int L, int side, const double *X, double *Y, int nvec, int ld,
                            const cpx<double> *E, const double *pre, const double *post,
                            const double *vscale, cudaStream_t st) {
  return launch_prop<double>(L, side, X, Y, nvec, ld, E, pre, post, vscale, st);
}
}  // namespace dq
