// Sweep kernels instantiated for input storage float, compute float, output float.
#include "sweep_kernels.cuh"

namespace bs {

cudaError_t sweep_f32(const SweepPlan& p, bool adjoint, int N, const void* in, void* out,
                        bs_layout layout, int64_t M, cudaStream_t st) {
  return dispatch_sweep<float, float, float, 4>(p, adjoint, N, reinterpret_cast<const float*>(in),
                                                reinterpret_cast<float*>(out), layout, M, st);
}

}  // namespace bs
