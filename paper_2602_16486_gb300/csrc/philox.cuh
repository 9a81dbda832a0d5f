// Counter-based normals for the stochastic collision (Eq. cm_collision: eta_v are
// independent standard normals; the paper does not name a generator).
//
// Philox4x32-10 as published by Salmon, Moraes, Dror & Shaw ("Parallel random numbers:
// as easy as 1, 2, 3", SC'11): ten rounds of the 4x32 Philox S-box, multipliers
// 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85. Each output
// word gives a 23-bit uniform u = (w/2^9 + 1/2) 2^-23 in (0, 1), exact in FP32, and
// each word pair gives two normals by the Box-Muller transform (Box & Muller, 1958):
//   r = sqrt(-2 ln u_a),  z_a = r cos(2 pi u_b),  z_b = r sin(2 pi u_b).
// Keying: key = seed, counter = (site, step lo, step hi, tag << 16 | block).
#pragma once

#include <cstdint>

namespace flbm {

struct Normals4 {
  float z0, z1, z2, z3;
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * ctr.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, ctr.x);
    const uint32_t lo1 = 0xCD9E8D57u * ctr.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, ctr.z);
    ctr = make_uint4(hi1 ^ ctr.y ^ k0, lo1, hi0 ^ ctr.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return ctr;
}

// (w >> 9) + 1/2, scaled by 2^-23: the integer converts exactly and the FMA result
// (m + 0.5) 2^-23 has 24 significant bits, so it is exact in FP32.
__device__ __forceinline__ float uniform01(uint32_t w) {
  return fmaf(static_cast<float>(w >> 9), 0x1p-23f, 0x1p-24f);
}

__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float &za, float &zb) {
  const float ua = uniform01(wa);
  const float ub = uniform01(wb);
  const float r = sqrtf(-2.0f * logf(ua));
  float s, c;
  sincospif(2.0f * ub, &s, &c);
  za = r * c;
  zb = r * s;
}

__device__ __forceinline__ Normals4 normals4(uint32_t site, uint32_t step_lo, uint32_t step_hi,
                                             uint32_t tag_blk, uint32_t k0, uint32_t k1) {
  const uint4 w = philox4x32_10(make_uint4(site, step_lo, step_hi, tag_blk), k0, k1);
  Normals4 n;
  box_muller(w.x, w.y, n.z0, n.z1);
  box_muller(w.z, w.w, n.z2, n.z3);
  return n;
}

}  // namespace flbm
