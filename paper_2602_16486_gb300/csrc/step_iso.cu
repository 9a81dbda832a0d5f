// The fused step of the isotropic D3Q27 variant (modes 4-6 = trace and deviators of the
// normal stresses; collide.cuh, ISO), every storage type: instantiations of the kernels
// of step_kernels.cuh for step variants 1, 2 and 5.
#include "step_kernels.cuh"

namespace flbm {

cudaError_t launch_step_iso(int storage, int variant, int parity, bool noise, bool shear, const StepArgs &a,
                            cudaStream_t s) {
  if (storage == 0) return launch_typed<3, float, true>(variant, parity, noise, shear, a, s);
  if (storage == 1) return launch_typed<3, __nv_bfloat16, true>(variant, parity, noise, shear, a, s);
  return launch_typed<3, __half, true>(variant, parity, noise, shear, a, s);
}

}  // namespace flbm
