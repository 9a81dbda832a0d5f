// The fused step with BF16 or FP16 deviation storage (FP32 arithmetic): instantiations of
// the kernels of step_kernels.cuh, in a translation unit of their own.
#include "step_kernels.cuh"

namespace flbm {

cudaError_t launch_step_16(int D, int storage, int variant, int parity, bool noise, bool shear, const StepArgs &a,
                           cudaStream_t s) {
  if (D == 3)
    return storage == 1 ? launch_typed<3, __nv_bfloat16, false>(variant, parity, noise, shear, a, s)
                        : launch_typed<3, __half, false>(variant, parity, noise, shear, a, s);
  return storage == 1 ? launch_typed<2, __nv_bfloat16, false>(variant, parity, noise, shear, a, s)
                      : launch_typed<2, __half, false>(variant, parity, noise, shear, a, s);
}

}  // namespace flbm
