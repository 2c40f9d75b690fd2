// Sweep kernels instantiated for input storage __nv_bfloat16, compute float, output float.
#include "sweep_kernels.cuh"

namespace bs {

cudaError_t sweep_bf16(const SweepPlan& p, bool adjoint, int N, const void* in, void* out,
                        bs_layout layout, int64_t M, cudaStream_t st) {
  return dispatch_sweep<float, __nv_bfloat16, float, 4>(p, adjoint, N, reinterpret_cast<const __nv_bfloat16*>(in),
                                                reinterpret_cast<float*>(out), layout, M, st);
}

}  // namespace bs
