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

#include "vec.cuh"

namespace flbm {

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

// Round keys of Philox4x32-10: key + r (W0, W1). KeyTable reads them precomputed (kernel
// arguments, constant bank); KeyBase forms them from the key (per-lattice keys in memory).
struct KeyTable {
  const uint32_t *t0, *t1;
  __device__ __forceinline__ uint32_t k0(int r) const { return t0[r]; }
  __device__ __forceinline__ uint32_t k1(int r) const { return t1[r]; }
};
struct KeyBase {
  uint32_t b0, b1;
  __device__ __forceinline__ uint32_t k0(int r) const { return b0 + (uint32_t)r * 0x9E3779B9u; }
  __device__ __forceinline__ uint32_t k1(int r) const { return b1 + (uint32_t)r * 0xBB67AE85u; }
};

// Philox4x32-10; the 64-bit products give each round's high and low words in one multiply.
template <typename K>
__device__ __forceinline__ uint4 philox4x32_10_ks(uint4 ctr, const K &keys) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * ctr.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * ctr.z;
    ctr = make_uint4((uint32_t)(p1 >> 32) ^ ctr.y ^ keys.k0(round), (uint32_t)p1,
                     (uint32_t)(p0 >> 32) ^ ctr.w ^ keys.k1(round), (uint32_t)p0);
  }
  return ctr;
}

// Box-Muller, angle: cos and sin of 2 pi u_b depend only on u_b mod 1, and the word read
// as a signed integer s_b is that residue times 2^32: u_b = (floor(s_b / 2^9) + 1/2) 2^-23
// mod 1. The angle is taken as 2 pi (s_b 2^-32 + 2^-24), with s_b converted to FP32 (rounded to
// 24 bits), which lies within pi 2^-23 (3.7e-7 rad) of 2 pi u_b: one conversion and one FMA,
// in (-pi, pi]. cos / sin come from the hardware approximations (__sincosf; absolute error
// about 4e-7 on [-pi, pi]), which cost two instructions instead of a polynomial.
//
// The radius: u_a = (2 m_a + 1) 2^-24 with y = 2 m_a + 1 an odd integer below 2^24, so
// -2 ln u_a = -2 (ln y - 24 ln 2). y converts to FP32 exactly; the argument reduction
// of Cody & Waite (Software Manual for the Elementary Functions, 1980) writes y = 2^k x
// with x in [sqrt(1/2), sqrt(2)), and ln x = 2 atanh(s) = 2 (s + s^3/3 + ... + s^9/9),
// s = (x - 1)/(x + 1), |s| < 0.172 (truncation below 1e-9 relative). x - 1 is exact,
// so the result keeps its relative accuracy as u_a -> 1, where r -> 0 (a hardware
// logarithm has an absolute error there that exceeds the value). Checked against the FP64
// definition over all 2^23 codes: relative error of -2 ln u_a below 3e-7.
constexpr float kAngleScale = 0x1p-32f * 6.28318530717958647692f;  // 2 pi 2^-32
constexpr float kAngleOffset = 0x1p-23f * 3.14159265358979323846f;  // pi 2^-23 = 2 pi 2^-24

// Four normals of Philox block `blk` for each lane's site (lane l: site0 + l * dsite),
// each multiplied by sqrt(rho) of its lane: the radius is taken as sqrt(-2 rho ln u_a)
// (hardware square root, PTX sqrt.approx.ftz) in one product and one root per lane.
template <typename T, typename K>
__device__ __forceinline__ void normals4_scaled(uint32_t site0, uint32_t step_lo, uint32_t step_hi,
                                                uint32_t blk, const K &keys, T rho, T (&z)[4],
                                                uint32_t dsite = 1) {
  constexpr int L = Lanes<T>::n;
  float ang[L][2];
  uint32_t wav[L][2];
#pragma unroll
  for (int l = 0; l < L; ++l) {
    const uint4 w = philox4x32_10_ks(make_uint4(site0 + uint32_t(l) * dsite, step_lo, step_hi, blk), keys);
    wav[l][0] = w.x;
    wav[l][1] = w.z;
    ang[l][0] = fmaf((float)(int)w.y, kAngleScale, kAngleOffset);
    ang[l][1] = fmaf((float)(int)w.w, kAngleScale, kAngleOffset);
  }
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    T x, kf;
#pragma unroll
    for (int l = 0; l < L; ++l) {
      // ix = bits(y) - bits(sqrt(1/2)) - 24 * 2^23: its top bits give k - 24 directly (an
      // arithmetic shift; the range [-0x0BB504F3, 0x004AFB0C] cannot overflow) and its low 23
      // bits the mantissa of x.
      const uint32_t y = (wav[l][p] >> 8) | 1u;
      const uint32_t ix = __float_as_uint((float)y) - (0x3F3504F3u + (24u << 23));
      set_lane(x, l, __uint_as_float((ix & 0x007FFFFFu) + 0x3F3504F3u));
      set_lane(kf, l, (float)((int)ix >> 23));
    }
    const T t = vsub(x, splat<T>(1.0f));
    const T d = vadd(x, splat<T>(1.0f));
    T rd;
#pragma unroll
    for (int l = 0; l < L; ++l) {
      float r_;
      asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r_) : "f"(lane(d, l)));
      set_lane(rd, l, r_);
    }
    const T sx = vmul(t, rd);
    const T s2 = vmul(sx, sx);
    T P = vfma(s2, splat<T>(-4.0f / 9.0f), splat<T>(-4.0f / 7.0f));  // -2 * 2 * (1/(2j+1))
    P = vfma(P, s2, splat<T>(-4.0f / 5.0f));
    P = vfma(P, s2, splat<T>(-4.0f / 3.0f));
    P = vfma(P, s2, splat<T>(-4.0f));
    const T a = vfma(kf, splat<T>(-1.38629436f), vmul(sx, P));  // -2 ln u_a (kf = k - 24)
    const T rad = sqrt_fast_lanes(vmul(a, rho));  // sqrt(rho) sqrt(-2 ln u_a)
    T c, sn;
#pragma unroll
    for (int l = 0; l < L; ++l) {
      float sl, cl;
      __sincosf(ang[l][p], &sl, &cl);
      set_lane(sn, l, sl);
      set_lane(c, l, cl);
    }
    z[2 * p] = vmul(rad, c);
    z[2 * p + 1] = vmul(rad, sn);
  }
}

}  // namespace flbm
