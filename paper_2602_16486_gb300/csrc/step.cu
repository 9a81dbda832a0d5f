// Fused fluctuating central-moment collide-and-stream step (one lattice update).
//
// Per site, in the order of the paper's "Algorithm of computation" (Sec. II-B):
//   load the Q populations arriving at the site, rho and u (Eq. macro),
//   k = T(u) f (Sec. II-B / II-C, factorised, see cm.cuh),
//   k*_v = (1 - L_v) k_v + L_v k^eq_v + I~_v phi_v eta_v (Eq. cm_collision) with
//   k^eq = (rho, 0, ..., 0) and phi_v = sqrt(rho) * sqrt(kBT L_v (2-L_v) b_v / cs^2)
//   (Eq. phi_general), normals from Philox4x32-10 + Box-Muller (philox.cuh),
//   f* = T(u)^{-1} k*, and streaming f_i(x + c_i, t+1) = f*_i(x, t) (Eq. streaming).
//
// Streaming is in place with the AA pattern (one population array): on even steps a
// site reads its own slots i and writes its post-collision values to its own slots
// opposite(i); on odd steps it reads the slot opposite(i) of its neighbour x - c_i and
// writes slot i of its neighbour x + c_i. Each step touches exactly the slots it
// reads, so no two threads race and no second lattice is needed. Logical populations:
// even state f_i(x) = A[i][x]; odd state f_i(x) = A[opposite(i)][x - c_i].
//
// Layout: structure of arrays A[q][z][y][x], x fastest; one thread per site, blocks
// of 128 consecutive x, grid (ceil(nx/128), ny, nz); warps touch 128-byte runs per
// population (FP32), so every load and store is coalesced (odd steps are shifted by
// one element, which costs no extra DRAM traffic).
#include <cuda_runtime.h>

#include "collide.cuh"
#include "internal.h"

namespace flbm {
namespace {

template <int D, typename S, int PARITY, bool NOISE>
__global__ void __launch_bounds__(kStepBlock) step_kernel(const StepArgs a) {
  const int x = blockIdx.x * kStepBlock + threadIdx.x;
  if (x >= a.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const Neighbourhood nb = neighbourhood(x, y, z, a.nx, a.ny, a.nz);
  S *__restrict__ f = static_cast<S *>(a.f);

  float F[3][3][3];
  load_logical<D, S, PARITY>(f, a.plane, nb, F);
  const uint32_t site = (uint32_t)(x + (long long)a.nx * (y + (long long)a.ny * z));
  collide_tile<D, NOISE>(F, a.rho0, a.om, a.phc, site, a.step_lo, a.step_hi, a.key0, a.key1);
  store_streamed<D, S, PARITY>(f, a.plane, nb, F);
}

template <int D, typename S>
cudaError_t launch_typed(int parity, bool noise, const StepArgs &a, cudaStream_t s) {
  const dim3 grid((a.nx + kStepBlock - 1) / kStepBlock, a.ny, a.nz);
  const dim3 block(kStepBlock);
  if (parity == 0) {
    if (noise)
      step_kernel<D, S, 0, true><<<grid, block, 0, s>>>(a);
    else
      step_kernel<D, S, 0, false><<<grid, block, 0, s>>>(a);
  } else {
    if (noise)
      step_kernel<D, S, 1, true><<<grid, block, 0, s>>>(a);
    else
      step_kernel<D, S, 1, false><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step(int D, int storage, int parity, bool noise, const StepArgs &a,
                        cudaStream_t s) {
  if (D == 3) {
    if (storage == 0) return launch_typed<3, float>(parity, noise, a, s);
    if (storage == 1) return launch_typed<3, __nv_bfloat16>(parity, noise, a, s);
    return launch_typed<3, __half>(parity, noise, a, s);
  }
  if (storage == 0) return launch_typed<2, float>(parity, noise, a, s);
  if (storage == 1) return launch_typed<2, __nv_bfloat16>(parity, noise, a, s);
  return launch_typed<2, __half>(parity, noise, a, s);
}

}  // namespace flbm
