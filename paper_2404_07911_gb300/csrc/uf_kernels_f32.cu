// float instantiation of the operator kernels (one translation unit per precision so that the
// two compile in parallel).
#include "uf_kernels.cuh"

namespace uf {

template <>
int launch_vmult<float>(int dim, int n, const DevArrays<float> &d, const void *ts, const void *tp,
                        const Scalars<float> &s, float *y, const float *x, bool adjoint,
                        void *stream, void *const *ev, const LaunchRange *rg) {
  return launch_vmult_impl<float>(dim, n, d, ts, tp, s, y, x, adjoint,
                                  reinterpret_cast<cudaStream_t>(stream), ev, rg);
}

}  // namespace uf
