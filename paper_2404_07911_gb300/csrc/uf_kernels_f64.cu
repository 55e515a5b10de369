// double instantiation of the operator kernels (one translation unit per precision so that the
// two compile in parallel).
#include "uf_kernels.cuh"

namespace uf {

template <>
int launch_vmult<double>(int dim, int n, const DevArrays<double> &d, const void *ts, const void *tp,
                        const Scalars<double> &s, double *y, const double *x, bool adjoint,
                        void *stream, void *const *ev, const LaunchRange *rg) {
  return launch_vmult_impl<double>(dim, n, d, ts, tp, s, y, x, adjoint,
                                  reinterpret_cast<cudaStream_t>(stream), ev, rg);
}

}  // namespace uf
