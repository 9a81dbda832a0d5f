// The raw-moment counterpart of the fused step (collide.cuh, collide_raw: T = M, N = I;
// with a uniform rate the fluctuating BGK step of Sec. II-A) for D2Q9 and D3Q27 in every
// storage type, with the AA pattern and launch shapes of step.cu (variants 1 and 2).
#include "step_kernels.cuh"

namespace flbm {
namespace {

template <int D, typename S>
cudaError_t raw_typed(int variant, int parity, bool noise, const StepArgs &a, cudaStream_t s) {
  if (parity == 0)
    return noise ? launch_raw_kernel<D, S, 0, true>(variant, a, s) : launch_raw_kernel<D, S, 0, false>(variant, a, s);
  return noise ? launch_raw_kernel<D, S, 1, true>(variant, a, s) : launch_raw_kernel<D, S, 1, false>(variant, a, s);
}

template <int D>
cudaError_t raw_storage(int storage, int variant, int parity, bool noise, const StepArgs &a, cudaStream_t s) {
  if (storage == 0) return raw_typed<D, float>(variant, parity, noise, a, s);
  if (storage == 1) return raw_typed<D, __nv_bfloat16>(variant, parity, noise, a, s);
  return raw_typed<D, __half>(variant, parity, noise, a, s);
}

}  // namespace

cudaError_t launch_step_raw(int D, int storage, int variant, int parity, bool noise, const StepArgs &a,
                            cudaStream_t s) {
  return D == 3 ? raw_storage<3>(storage, variant, parity, noise, a, s)
                : raw_storage<2>(storage, variant, parity, noise, a, s);
}

}  // namespace flbm
