// Sweep kernels instantiated for input storage float, compute float, output float.
#include "sweep_kernels.cuh"

namespace bs {

template <typename Sin>
int sweep_tma(const SweepPlan&, bool, int, const Sin*, float*, int64_t, cudaStream_t, cudaError_t*);

cudaError_t sweep_f32(const SweepPlan& p, bool adjoint, int N, const void* in, void* out,
                        bs_layout layout, int64_t M, cudaStream_t st, int L, int P) {
  if (layout == BS_INTERLEAVED && !p.periodic && P == 1 && option(BS_OPT_SWEEP_KERNEL) == 2) {
    cudaError_t e = cudaSuccess;
    if (sweep_tma<float>(p, adjoint, N, reinterpret_cast<const float*>(in), reinterpret_cast<float*>(out), M, st, &e))
      return e;
  }
  return dispatch_sweep<float, float, float, 4>(p, adjoint, N, reinterpret_cast<const float*>(in),
                                                reinterpret_cast<float*>(out), layout, M, st, L, P);
}

}  // namespace bs
