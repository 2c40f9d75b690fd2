// Sweep kernels instantiated for input storage double, compute double, output double.
#include "sweep_kernels.cuh"

namespace bs {

cudaError_t sweep_f64(const SweepPlan& p, bool adjoint, int N, const void* in, void* out,
                        bs_layout layout, int64_t M, cudaStream_t st, int L, int P) {
  return dispatch_sweep<double, double, double, 2>(p, adjoint, N, reinterpret_cast<const double*>(in),
                                                reinterpret_cast<double*>(out), layout, M, st, L, P);
}

}  // namespace bs
