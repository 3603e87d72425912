// FP32 instantiations of the FFT propagator kernels.
#include "prop_impl.cuh"

namespace dq {
cudaError_t launch_prop_f32(int L, int side, const float *X, float *Y, int nvec, int ld,
                            const cpx<float> *E, const float *pre, const float *post,
                            const float *vscale, cudaStream_t st) {
  return launch_prop<float>(L, side, X, Y, nvec, ld, E, pre, post, vscale, st);
}
}  // namespace dq
