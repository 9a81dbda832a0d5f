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
// Layout: structure of arrays A[q][z][y][x], x fastest. Kernels (step_kernels.cuh; launch
// variants, all computing the same update; see StepVariant in internal.h):
//   step_kernel  - one site per thread, blocks of 128 consecutive x, grid
//                  (ceil(nx/128), ny, nz); any nx;
//   step2_kernel - two sites per thread (x0 = 2 t, x0 + 1; nx even): every floating-
//                  point step runs as packed FP32x2, population pairs move as one 8-byte
//                  (FP32) or 4-byte (16-bit) access, per-population address offsets are
//                  block-uniform; capped at 128 registers (4 blocks of 4 warps per SM)
//                  or, for more warps, 102 (5 blocks; 3-D lattices) or 64 (8 blocks;
//                  D2Q9); the noise loop is unrolled or rolled (smaller code); blocks
//                  cover one row of 128 pair slots, or four rows of 32 (one per warp) for
//                  rows shorter than 256 sites.
// Warps touch contiguous runs of every population, so all accesses are coalesced (odd
// steps are shifted by one element, which costs no extra DRAM traffic).
#include "step_kernels.cuh"

namespace flbm {

cudaError_t launch_step(int lattice, int storage, int variant, int parity, bool noise, bool shear,
                        const StepArgs &a, cudaStream_t s) {
  if (lattice == 2) return launch_step_iso(storage, variant, parity, noise, shear, a, s);
  if (lattice == 3) return launch_step_d3q19(storage, variant, parity, noise, shear, a, s);
  const int D = lattice == 0 ? 2 : 3;
  if (storage != 0) return launch_step_16(D, storage, variant, parity, noise, shear, a, s);
  return D == 3 ? launch_typed<3, float, false>(variant, parity, noise, shear, a, s)
                : launch_typed<2, float, false>(variant, parity, noise, shear, a, s);
}

}  // namespace flbm
