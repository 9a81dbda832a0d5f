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
// Layout: structure of arrays A[q][z][y][x], x fastest. Kernels (launch variants, all
// computing the same update; see StepVariant in internal.h):
//   step_kernel  - one site per thread, blocks of 128 consecutive x, grid
//                  (ceil(nx/128), ny, nz); any nx;
//   step2_kernel - two sites per thread (x0 = 2 t, x0 + 1; nx even): every floating-
//                  point step runs as packed FP32x2, population pairs move as one 8-byte
//                  (FP32) or 4-byte (16-bit) access, per-population address offsets are
//                  block-uniform; capped at 128 registers (4 blocks of 4 warps per SM)
//                  or 102 (5 blocks); the noise loop is unrolled or rolled (smaller code).
// Warps touch contiguous runs of every population, so all accesses are coalesced (odd
// steps are shifted by one element, which costs no extra DRAM traffic).
#include <cuda_runtime.h>

#include <type_traits>

#include "collide.cuh"
#include "internal.h"

namespace flbm {
namespace {

template <int D, typename S, int PARITY, bool NOISE, bool SHEAR>
__global__ void __launch_bounds__(kStepBlock) step_kernel(const StepArgs a) {
  const int x = blockIdx.x * kStepBlock + threadIdx.x;
  if (x >= a.nx) return;
  const int y = blockIdx.y, z = blockIdx.z;
  const Neighbourhood nb = neighbourhood(x, y, z, a.nx, a.ny, a.nz);
  S *__restrict__ f = static_cast<S *>(a.f);

  float F[3][3][3];
  load_logical<D, S, PARITY>(f, a.plane, nb, F);
  const uint32_t site = (uint32_t)(x + (long long)a.nx * (y + (long long)a.ny * z));
  collide_tile<D, NOISE, float, false, SHEAR>(F, a.rho0, a.om, a.phc, site, a.step_lo, a.step_hi, a.ks0,
                                              a.ks1);
  store_streamed<D, S, PARITY>(f, a.plane, nb, F);
}

template <int D, typename S, int PARITY, bool NOISE, bool ROLLED, bool SHEAR, int MINB>
__global__ void __launch_bounds__(kStepBlock, MINB) step2_kernel(const StepArgs a) {
  const int x0 = 2 * (blockIdx.x * kStepBlock + threadIdx.x);
  if (x0 >= a.nx) return;
  const Addr2 ad = addr2(x0, blockIdx.y, blockIdx.z, a.nx, a.ny, a.nz);
  S *__restrict__ f = static_cast<S *>(a.f);

  float2 F[3][3][3];
  load_logical2<D, S, PARITY>(f, a.plane, ad, F);
  collide_tile<D, NOISE, float2, ROLLED, SHEAR>(F, a.rho0, a.om, a.phc, (uint32_t)ad.s0, a.step_lo,
                                                a.step_hi, a.ks0, a.ks1);
  store_streamed2<D, S, PARITY>(f, a.plane, ad, F);
}

template <typename S>
constexpr int storage_code() {
  return sizeof(S) == 4 ? 0 : (std::is_same<S, __nv_bfloat16>::value ? 1 : 2);
}

template <int D, typename S, int PARITY, bool NOISE, bool SHEAR>
cudaError_t launch_kernel(int variant, const StepArgs &a, cudaStream_t s) {
  const dim3 block(kStepBlock);
  if (variant != kStepOneSite) {
    // Register caps: 128 (four blocks of 128 threads per SM) or, for D3Q27, 102 (five
    // blocks: more warps to hide latency, at the risk of spills). D2Q9 needs fewer than
    // 102 registers either way, so its variants 5 and 6 are 2 and 3.
    constexpr int kOcc = D == 3 ? 5 : 4;
    const dim3 grid((a.nx / 2 + kStepBlock - 1) / kStepBlock, a.ny, a.nz);
    if (variant == kStepPairRolled)
      step2_kernel<D, S, PARITY, NOISE, true, SHEAR, 4><<<grid, block, 0, s>>>(a);
    else if (variant == kStepPairOcc)
      step2_kernel<D, S, PARITY, NOISE, false, SHEAR, kOcc><<<grid, block, 0, s>>>(a);
    else if (variant == kStepPairRolledOcc)
      step2_kernel<D, S, PARITY, NOISE, true, SHEAR, kOcc><<<grid, block, 0, s>>>(a);
    else
      step2_kernel<D, S, PARITY, NOISE, false, SHEAR, 4><<<grid, block, 0, s>>>(a);
  } else {
    const dim3 grid((a.nx + kStepBlock - 1) / kStepBlock, a.ny, a.nz);
    step_kernel<D, S, PARITY, NOISE, SHEAR><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <int D, typename S>
cudaError_t launch_typed(int variant, int parity, bool noise, bool shear, const StepArgs &a,
                         cudaStream_t s) {
  if (variant == kStepPipelined)
    return launch_step_pipelined(D, storage_code<S>(), parity, noise, shear, a, s);
  if (parity == 0) {
    if (noise)
      return shear ? launch_kernel<D, S, 0, true, true>(variant, a, s)
                   : launch_kernel<D, S, 0, true, false>(variant, a, s);
    return shear ? launch_kernel<D, S, 0, false, true>(variant, a, s)
                 : launch_kernel<D, S, 0, false, false>(variant, a, s);
  }
  if (noise)
    return shear ? launch_kernel<D, S, 1, true, true>(variant, a, s)
                 : launch_kernel<D, S, 1, true, false>(variant, a, s);
  return shear ? launch_kernel<D, S, 1, false, true>(variant, a, s)
               : launch_kernel<D, S, 1, false, false>(variant, a, s);
}

}  // namespace

cudaError_t launch_step(int D, int storage, int variant, int parity, bool noise, bool shear,
                        const StepArgs &a, cudaStream_t s) {
  if (D == 3) {
    if (storage == 0) return launch_typed<3, float>(variant, parity, noise, shear, a, s);
    if (storage == 1) return launch_typed<3, __nv_bfloat16>(variant, parity, noise, shear, a, s);
    return launch_typed<3, __half>(variant, parity, noise, shear, a, s);
  }
  if (storage == 0) return launch_typed<2, float>(variant, parity, noise, shear, a, s);
  if (storage == 1) return launch_typed<2, __nv_bfloat16>(variant, parity, noise, shear, a, s);
  return launch_typed<2, __half>(variant, parity, noise, shear, a, s);
}

}  // namespace flbm
