// The stochastic central-moment collision of one site, on the register tile.
//
//   k*_v = (1 - L_v) k_v + L_v k^eq_v + I~_v phi_v eta_v        (Eq. cm_collision)
//   k^eq = (rho, 0, ..., 0)                                     (Sec. II-B, Sec. II-C)
//   phi_v = sqrt(rho kBT L_v (2 - L_v) b_v / cs^2)              (Eq. phi_general)
// with I~_v = 1 exactly for the non-conserved modes v > D and the conserved modes
// relaxed at rate 1 (k*_0 = rho, k*_1..D = 0), as the paper fixes in Sec. II-B and II-C.
// The caller passes om_v = 1 - L_v and phc_v = sqrt(kBT L_v (2 - L_v) b_v / cs^2)
// (host-computed), so phi_v = sqrt(rho) phc_v uses the local density.
// Noise: mode v uses normal n = v - D - 1 of block n / 4 of the site's Philox stream.
// On return the tile holds the post-collision deviations d*_i = f*_i - w_i rho0.
#pragma once

#include "cm.cuh"
#include "philox.cuh"

namespace flbm {

template <int D, bool NOISE>
__device__ __forceinline__ void collide_tile(float (&F)[3][3][3], float rho0, const float *om,
                                             const float *phc, uint32_t site, uint32_t step_lo,
                                             uint32_t step_hi, uint32_t key0, uint32_t key1) {
  float drho, rho, ux, uy, uz;
  site_central_moments<D>(F, rho0, drho, rho, ux, uy, uz);
  const float srho = sqrtf(rho);
  if (D == 3) {
#pragma unroll
    for (int v = 4; v < 27; ++v) {
      const int t = d3q27_mode_tensor(v);
      float &k = F[t / 9][(t / 3) % 3][t % 3];
      k = om[v] * k;
    }
    if (NOISE) {
#pragma unroll
      for (int blk = 0; blk < 6; ++blk) {
        const Normals4 n = normals4(site, step_lo, step_hi, (uint32_t)blk, key0, key1);
        const float zz[4] = {n.z0, n.z1, n.z2, n.z3};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int v = 4 + 4 * blk + j;
          if (v < 27) {
            const int t = d3q27_mode_tensor(v);
            float &k = F[t / 9][(t / 3) % 3][t % 3];
            k = fmaf(srho * phc[v], zz[j], k);
          }
        }
      }
    }
    F[0][0][1] = 0.0f;  // k*_1 (x momentum, central)
    F[0][1][0] = 0.0f;  // k*_2
    F[1][0][0] = 0.0f;  // k*_3
  } else {
    // D2Q9: modes 3 and 4 are the sum and difference of the (2,0) and (0,2) moments.
    const float kxx = F[1][0][2], kyy = F[1][2][0];
    float k3 = om[3] * (kxx + kyy);
    float k4 = om[4] * (kxx - kyy);
    float k5 = om[5] * F[1][1][1];
    float k6 = om[6] * F[1][1][2];
    float k7 = om[7] * F[1][2][1];
    float k8 = om[8] * F[1][2][2];
    if (NOISE) {
      const Normals4 n0 = normals4(site, step_lo, step_hi, 0u, key0, key1);
      const Normals4 n1 = normals4(site, step_lo, step_hi, 1u, key0, key1);
      k3 = fmaf(srho * phc[3], n0.z0, k3);
      k4 = fmaf(srho * phc[4], n0.z1, k4);
      k5 = fmaf(srho * phc[5], n0.z2, k5);
      k6 = fmaf(srho * phc[6], n0.z3, k6);
      k7 = fmaf(srho * phc[7], n1.z0, k7);
      k8 = fmaf(srho * phc[8], n1.z1, k8);
    }
    F[1][0][2] = 0.5f * (k3 + k4);
    F[1][2][0] = 0.5f * (k3 - k4);
    F[1][1][1] = k5;
    F[1][1][2] = k6;
    F[1][2][1] = k7;
    F[1][2][2] = k8;
    F[1][0][1] = 0.0f;  // k*_1
    F[1][1][0] = 0.0f;  // k*_2
  }
  // r* = N^{-1} k* (entry (0,0,0) = k*_0 = rho), then d* = M^{-1} r* - w rho0.
  tile_shift_inv<D>(F, ux, uy, uz);
  mom<D>(F, 0, 0, 0) = drho;
  tile_raw_inv<D>(F);
}

}  // namespace flbm
