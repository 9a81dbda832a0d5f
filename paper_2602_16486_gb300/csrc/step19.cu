// The fused step on D3Q19 (Sec. II-C, "Lattice-agnostic construction and the D3Q19
// example"): the collision of d3q19.cuh between the AA-pattern load and store, one site
// per thread (step variant 1, any nx) or two sites per thread with packed FP32x2
// arithmetic (variants 2 and 5, nx even; 5 allows one more resident block per SM than 2;
// 8 and 7 are 2 and 5 in blocks of four rows for short rows).
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "internal.h"

namespace flbm {
namespace {

template <typename S, int PARITY, bool NOISE, bool SHEAR>
__global__ void __launch_bounds__(kStepBlock) step19_kernel(const StepArgs a) {
  const int x = blockIdx.x * kStepBlock + threadIdx.x;
  if (x >= a.nx) return;
  const int y = blockIdx.y, z = blockIdx.z + a.z_lo;
  const Neighbourhood nb = neighbourhood(x, y, z, a.nx, a.ny, a.nz);
  S *__restrict__ f = static_cast<S *>(a.f);
  float F[19];
  load19<S, PARITY>(f, a.plane, nb, F);
  const uint32_t site = (uint32_t)(x + (long long)a.nx * (y + (long long)a.ny * z)) + a.site_base;
  collide19<NOISE, float, SHEAR>(F, a.rho0, a.om, a.phc, site, a.step_lo, a.step_hi, KeyTable{a.ks0, a.ks1});
  store19<S, PARITY>(f, a.plane, nb, F);
}

// RB rows per block as in step2_kernel (step_kernels.cuh).
template <typename S, int PARITY, bool NOISE, bool SHEAR, int MINB, int RB = 1>
__global__ void __launch_bounds__(kStepBlock, MINB) step19_2_kernel(const StepArgs a) {
  constexpr int BX = kStepBlock / RB;
  const int x0 = 2 * (blockIdx.x * BX + (RB == 1 ? (int)threadIdx.x : (int)threadIdx.x % BX));
  const int y = RB == 1 ? (int)blockIdx.y : (int)blockIdx.y * RB + (int)threadIdx.x / BX;
  if (x0 >= a.nx || y >= a.ny) return;
  const Addr2 ad = addr2(x0, y, blockIdx.z + a.z_lo, a.nx, a.ny, a.nz);
  S *__restrict__ f = static_cast<S *>(a.f);
  float2 F[19];
  load19_pairs<S, PARITY>(f, a.plane, ad, F);
  collide19<NOISE, float2, SHEAR>(F, a.rho0, a.om, a.phc, pair_site0<PARITY>(ad) + a.site_base, a.step_lo,
                                  a.step_hi, KeyTable{a.ks0, a.ks1}, pair_dsite<PARITY>(ad));
  store19_pairs<S, PARITY>(f, a.plane, ad, F);
}

template <typename S, int PARITY, bool NOISE, bool SHEAR>
cudaError_t launch19(int variant, const StepArgs &a, cudaStream_t s) {
  const dim3 block(kStepBlock);
  if (variant == kStepOneSite) {
    step19_kernel<S, PARITY, NOISE, SHEAR><<<dim3((a.nx + kStepBlock - 1) / kStepBlock, a.ny, a.nz_grid), block, 0, s>>>(a);
  } else {
    const dim3 grid((a.nx / 2 + kStepBlock - 1) / kStepBlock, a.ny, a.nz_grid);
    // The general rates hold every central moment through the collision: their two-site
    // kernel gets a 168-register cap (three blocks per SM) instead of spilling.
    constexpr int kMinb = SHEAR ? 4 : 3;
    constexpr int BX = kStepBlock / kRowBlockRows;
    const dim3 grid_r((a.nx / 2 + BX - 1) / BX, (a.ny + kRowBlockRows - 1) / kRowBlockRows, a.nz_grid);
    if (variant == kStepPairOccRows)
      step19_2_kernel<S, PARITY, NOISE, SHEAR, kMinb + 1, kRowBlockRows><<<grid_r, block, 0, s>>>(a);
    else if (variant == kStepPairRows)
      step19_2_kernel<S, PARITY, NOISE, SHEAR, kMinb, kRowBlockRows><<<grid_r, block, 0, s>>>(a);
    else if (variant == kStepPairOcc || variant == kStepPairRolledOcc)
      step19_2_kernel<S, PARITY, NOISE, SHEAR, kMinb + 1><<<grid, block, 0, s>>>(a);
    else
      step19_2_kernel<S, PARITY, NOISE, SHEAR, kMinb><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename S>
cudaError_t launch19_typed(int variant, int parity, bool noise, bool shear, const StepArgs &a, cudaStream_t s) {
  if (parity == 0) {
    if (noise)
      return shear ? launch19<S, 0, true, true>(variant, a, s) : launch19<S, 0, true, false>(variant, a, s);
    return shear ? launch19<S, 0, false, true>(variant, a, s) : launch19<S, 0, false, false>(variant, a, s);
  }
  if (noise) return shear ? launch19<S, 1, true, true>(variant, a, s) : launch19<S, 1, true, false>(variant, a, s);
  return shear ? launch19<S, 1, false, true>(variant, a, s) : launch19<S, 1, false, false>(variant, a, s);
}

}  // namespace

cudaError_t launch_step_d3q19(int storage, int variant, int parity, bool noise, bool shear, const StepArgs &a,
                              cudaStream_t s) {
  if (storage == 0) return launch19_typed<float>(variant, parity, noise, shear, a, s);
  if (storage == 1) return launch19_typed<__nv_bfloat16>(variant, parity, noise, shear, a, s);
  return launch19_typed<__half>(variant, parity, noise, shear, a, s);
}

}  // namespace flbm
