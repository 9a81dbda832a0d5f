// Kernel templates of the fused step (documented in step.cu), shared by the translation
// units that instantiate them: step.cu (FP32 storage and the dispatch), step_16.cu
// (BF16 and FP16 storage) and step_iso.cu (the isotropic D3Q27 variant).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "collide.cuh"
#include "internal.h"

namespace flbm {
namespace {

template <int D, typename S, int PARITY, bool NOISE, bool SHEAR, bool ISO, bool RAW = false>
__global__ void __launch_bounds__(kStepBlock) step_kernel(const StepArgs a) {
  const int x = blockIdx.x * kStepBlock + threadIdx.x;
  if (x >= a.nx) return;
  const int y = blockIdx.y, z = blockIdx.z + a.z_lo;
  const Neighbourhood nb = neighbourhood(x, y, z, a.nx, a.ny, a.nz);
  S *__restrict__ f = static_cast<S *>(a.f);

  float F[3][3][3];
  load_logical<D, S, PARITY>(f, a.plane, nb, F);
  const uint32_t site = (uint32_t)(x + (long long)a.nx * (y + (long long)a.ny * z)) + a.site_base;
  collide_tile<D, NOISE, float, false, SHEAR, ISO, RAW>(F, a.rho0, a.om_t, a.phc_t, site, a.step_lo, a.step_hi,
                                                        a.ks0, a.ks1);
  store_streamed<D, S, PARITY>(f, a.plane, nb, F);
}

// RB rows per block: 1 (128 pair slots of one row; y block-uniform) or kRowBlockRows
// (each warp one row of 32 pair slots, for rows shorter than 256 sites).
template <int D, typename S, int PARITY, bool NOISE, bool ROLLED, bool SHEAR, int MINB, bool ISO, bool RAW = false,
          int RB = 1>
__global__ void __launch_bounds__(kStepBlock, MINB) step2_kernel(const StepArgs a) {
  constexpr int BX = kStepBlock / RB;
  const int x0 = 2 * (blockIdx.x * BX + (RB == 1 ? (int)threadIdx.x : (int)threadIdx.x % BX));
  const int y = RB == 1 ? (int)blockIdx.y : (int)blockIdx.y * RB + (int)threadIdx.x / BX;
  if (x0 >= a.nx || y >= a.ny) return;
  const Addr2 ad = addr2(x0, y, blockIdx.z + a.z_lo, a.nx, a.ny, a.nz);
  S *__restrict__ f = static_cast<S *>(a.f);

  float2 F[3][3][3];
  load_pairs<D, S, PARITY>(f, a.plane, ad, F);
  collide_tile<D, NOISE, float2, ROLLED, SHEAR, ISO, RAW>(F, a.rho0, a.om_t, a.phc_t,
                                                          pair_site0<PARITY>(ad) + a.site_base, a.step_lo,
                                                          a.step_hi, a.ks0, a.ks1, pair_dsite<PARITY>(ad));
  store_pairs<D, S, PARITY>(f, a.plane, ad, F);
}

template <typename S>
constexpr int storage_code() {
  return sizeof(S) == 4 ? 0 : (std::is_same<S, __nv_bfloat16>::value ? 1 : 2);
}

// One launch of variant 1, 2, 3, 5 or 6 (the pipelined variant 4 lives in
// step_pipe.cu). ISO kernels exist for variants 1, 2 and 5 only; the host maps 3 and 6
// to 2 and 5 for them.
template <int D, typename S, int PARITY, bool NOISE, bool SHEAR, bool ISO>
cudaError_t launch_kernel(int variant, const StepArgs &a, cudaStream_t s) {
  const dim3 block(kStepBlock);
  if (variant != kStepOneSite) {
    // Register caps: 128 (four blocks of 128 threads per SM) or, for variants 5 and 6,
    // 102 for D3Q27 (five blocks: more warps to hide latency, at the risk of spills) and
    // 64 for the lighter D2Q9 update (eight blocks; ten, at 51 registers, left the even
    // step waiting on its loads: 0.214 against 0.183 ms at 4096^2).
    constexpr int kOcc = D == 3 ? 5 : 8;
    const dim3 grid((a.nx / 2 + kStepBlock - 1) / kStepBlock, a.ny, a.nz_grid);
    const bool occ = variant == kStepPairOcc || variant == kStepPairRolledOcc;
    const bool rolled = !ISO && (variant == kStepPairRolled || variant == kStepPairRolledOcc);
    if (variant == kStepPairOccRows || variant == kStepPairRows) {
      constexpr int BX = kStepBlock / kRowBlockRows;
      const dim3 grid_r((a.nx / 2 + BX - 1) / BX, (a.ny + kRowBlockRows - 1) / kRowBlockRows, a.nz_grid);
      if (variant == kStepPairOccRows)
        step2_kernel<D, S, PARITY, NOISE, false, SHEAR, kOcc, ISO, false, kRowBlockRows><<<grid_r, block, 0, s>>>(a);
      else
        step2_kernel<D, S, PARITY, NOISE, false, SHEAR, 4, ISO, false, kRowBlockRows><<<grid_r, block, 0, s>>>(a);
    } else if (occ) {
      if (rolled)
        step2_kernel<D, S, PARITY, NOISE, !ISO, SHEAR, kOcc, ISO><<<grid, block, 0, s>>>(a);
      else
        step2_kernel<D, S, PARITY, NOISE, false, SHEAR, kOcc, ISO><<<grid, block, 0, s>>>(a);
    } else {
      if (rolled)
        step2_kernel<D, S, PARITY, NOISE, !ISO, SHEAR, 4, ISO><<<grid, block, 0, s>>>(a);
      else
        step2_kernel<D, S, PARITY, NOISE, false, SHEAR, 4, ISO><<<grid, block, 0, s>>>(a);
    }
  } else {
    const dim3 grid((a.nx + kStepBlock - 1) / kStepBlock, a.ny, a.nz_grid);
    step_kernel<D, S, PARITY, NOISE, SHEAR, ISO><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <int D, typename S, bool ISO>
cudaError_t launch_typed(int variant, int parity, bool noise, bool shear, const StepArgs &a, cudaStream_t s) {
  if (!ISO && variant == kStepPipelined)
    return launch_step_pipelined(D, storage_code<S>(), parity, noise, shear, a, s);
  if (parity == 0) {
    if (noise)
      return shear ? launch_kernel<D, S, 0, true, true, ISO>(variant, a, s)
                   : launch_kernel<D, S, 0, true, false, ISO>(variant, a, s);
    return shear ? launch_kernel<D, S, 0, false, true, ISO>(variant, a, s)
                 : launch_kernel<D, S, 0, false, false, ISO>(variant, a, s);
  }
  if (noise)
    return shear ? launch_kernel<D, S, 1, true, true, ISO>(variant, a, s)
                 : launch_kernel<D, S, 1, true, false, ISO>(variant, a, s);
  return shear ? launch_kernel<D, S, 1, false, true, ISO>(variant, a, s)
               : launch_kernel<D, S, 1, false, false, ISO>(variant, a, s);
}

// The raw-moment counterpart (collide_raw): one site per thread or two (nx even).
template <int D, typename S, int PARITY, bool NOISE>
cudaError_t launch_raw_kernel(int variant, const StepArgs &a, cudaStream_t s) {
  const dim3 block(kStepBlock);
  if (variant == kStepOneSite)
    step_kernel<D, S, PARITY, NOISE, false, false, true>
        <<<dim3((a.nx + kStepBlock - 1) / kStepBlock, a.ny, a.nz_grid), block, 0, s>>>(a);
  else
    step2_kernel<D, S, PARITY, NOISE, false, false, 4, false, true>
        <<<dim3((a.nx / 2 + kStepBlock - 1) / kStepBlock, a.ny, a.nz_grid), block, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace
}  // namespace flbm
