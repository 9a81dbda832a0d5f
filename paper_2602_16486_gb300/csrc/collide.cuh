// The stochastic central-moment collision of one site (T = float) or of two sites at
// once (T = float2), on the register tile.
//
//   k*_v = (1 - L_v) k_v + L_v k^eq_v + I~_v phi_v eta_v        (Eq. cm_collision)
//   k^eq = (rho, 0, ..., 0)                                     (Sec. II-B, Sec. II-C)
//   phi_v = sqrt(rho kBT L_v (2 - L_v) b_v / cs^2)              (Eq. phi_general)
// with I~_v = 1 exactly for the non-conserved modes v > D and the conserved modes
// relaxed at rate 1 (k*_0 = rho, k*_1..D = 0), as the paper fixes in Sec. II-B and II-C.
// The caller passes om_v = 1 - L_v and phc_v = sqrt(kBT L_v (2 - L_v) b_v / cs^2)
// (host-computed), so phi_v = sqrt(rho) phc_v uses the local density; both come multiplied
// by the mode's tile scale (lattice.cuh, tile_scale), because the inverse transforms take
// the post-collision moments in the halved convention of cm.cuh.
// Noise: mode v uses normal n = v - D - 1 of block n / 4 of the site's Philox stream.
// On return the tile holds the post-collision deviations d*_i = f*_i - w_i rho0.
#pragma once

#include "cm.cuh"
#include "philox.cuh"

namespace flbm {

// ---- relaxation rates and noise amplitudes, as the collision reads them --------------
// ArrayRates: om_v = 1 - L_v and phc_v = sqrt(kBT L_v (2 - L_v) b_v / cs^2) per mode, times
// the mode's tile scale, from a kernel-argument array (constant bank; host-computed).
struct ArrayRates {
  const float *om_, *phc_;
  __device__ __forceinline__ float om(int v) const { return om_[v]; }
  __device__ __forceinline__ float phc(int v) const { return phc_[v]; }
};

// sqrt(b_v / cs^2) = sqrt(3 b_v) of the modes, b_v the product of the 1-D norms
// (1, 1/3, 2/9) over the tensor orders (D2Q9 modes 3 and 4: 2 * 2/9). Compile-time.
__host__ __device__ constexpr double csqrt(double x) {
  double r = x > 1.0 ? x : 1.0;
  for (int i = 0; i < 64; ++i) r = 0.5 * (r + x / r);
  return r;
}
__host__ __device__ constexpr double bnorm1(int order) { return order == 0 ? 1.0 : order == 1 ? 1.0 / 3.0 : 2.0 / 9.0; }
template <int D>
__host__ __device__ constexpr float noise_unit(int v) {
  return D == 3 ? (float)csqrt(3.0 * bnorm1(d3q27_mode_tensor(v) % 3) * bnorm1((d3q27_mode_tensor(v) / 3) % 3) *
                               bnorm1(d3q27_mode_tensor(v) / 9))
         : (v == 3 || v == 4) ? (float)csqrt(3.0 * 2.0 * bnorm1(2))
                              : (float)csqrt(3.0 * bnorm1(d2q9_mode_tensor(v) % 3) * bnorm1(d2q9_mode_tensor(v) / 3));
}

// ShearRates: the paper's structure (L_v = 1 except the shear modes, which share one
// rate): om = 0 and phc_v = sqrt(kBT) sqrt(3 b_v) off the shear modes, om_sh and phc_sh
// on them. phc_sh is the amplitude of a shear mode with b = 1/9 (D3Q27 v = 7..9, D2Q9
// v = 5); D2Q9 mode 4 has b = 4/9 and so twice that amplitude (an exact scaling). Three
// numbers per lattice; the tile scales are compile-time factors.
template <int D>
struct ShearRates {
  float sqrt_kbt, om_sh, phc_sh;
  __device__ __forceinline__ static bool is_shear(int v) { return D == 3 ? (v >= 7 && v <= 9) : (v == 4 || v == 5); }
  __device__ __forceinline__ float om(int v) const { return is_shear(v) ? om_sh * tile_scale<D>(v) : 0.0f; }
  __device__ __forceinline__ float phc(int v) const {
    return is_shear(v) ? ((D == 2 && v == 4) ? 2.0f * tile_scale<D>(v) : tile_scale<D>(v)) * phc_sh
                       : sqrt_kbt * (noise_unit<D>(v) * tile_scale<D>(v));
  }
};

// D3Q27: adds phi_v eta_v (eta already scaled by sqrt(rho)) to the four modes that
// Philox block BLK feeds, v = 4 + 4 BLK + j (j < 4, v < 27).
template <int BLK, typename T, typename R>
__device__ __forceinline__ void add_noise_block(T (&F)[3][3][3], const R &rates, const T (&z)[4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int v = 4 + 4 * BLK + j;
    if (v < 27) {
      const int t = d3q27_mode_tensor(v);
      T &k = F[t / 9][(t / 3) % 3][t % 3];
      k = vfma(splat<T>(rates.phc(v)), z[j], k);
    }
  }
}

// ROLLED: generate the D3Q27 noise in a loop over the six Philox blocks instead of six
// unrolled copies, which shrinks the kernel's instruction footprint about fourfold (the
// unrolled body overflows the instruction cache); the arithmetic is identical.
// SHEAR: the caller guarantees the paper's relaxation structure, L_v = 1 for every
// non-conserved mode except the shear modes (D3Q27 v = 7, 8, 9; D2Q9 v = 4, 5; Sec. II-C
// and II-B). Then k*_v = phi_v eta_v needs no pre-collision value, and only the shear
// central moments are formed, directly as k_ab = r_ab - rho u_a u_b (Sec. II-C prints
// k7-k9 in this form) instead of through the full velocity shift.
//
// ISO (D3Q27 only): the isotropic variant, whose modes 4-6 are the trace and two deviators
// of the normal stresses, M4' = M4 + M5 + M6, M5' = M4 - M5, M6' = M4 + M5 - 2 M6 (the
// reading that gives one viscosity for every shear direction). The three tensor slots of
// modes 4-6 hold (M4', M5', M6') while the modes are relaxed and the noise is added, and
// are rotated back before the inverse transform. With SHEAR and ISO every non-conserved
// mode but 4-9 relaxes at rate 1; modes 4-9 are formed directly from the raw second
// moments: k_aa = P_aa - rho u_a^2, k_ab = P_ab - rho u_a u_b.
// The raw-moment counterpart of the scheme (T = M, N = I; Sec. II-C notes that this
// reduces the collision to raw moments, and with a uniform rate to the fluctuating BGK
// operator of Sec. II-A): the moments of the tile stay raw, the equilibrium raw moments
// of mode (a, b, c) are rho m_a(u_x) m_b(u_y) m_c(u_z) with m = (1, u, u^2) (the raw moments
// of the product equilibrium in the 1-D basis {1, c, c^2 - cs^2}), the non-conserved modes
// relax as k*_v = k^eq_v + (1 - L_v)(k_v - k^eq_v) + phi_v eta_v with the same amplitudes and
// normals, and only the raw inverse follows (halved convention, as below).
template <int D, bool NOISE, typename T, typename R, typename K>
__device__ __forceinline__ void collide_raw(T (&F)[3][3][3], float rho0, const R &rates, uint32_t site0,
                                            uint32_t step_lo, uint32_t step_hi, const K &keys, uint32_t dsite) {
  T drho, rho, ux, uy, uz;
  site_macros<D>(F, rho0, drho, rho, ux, uy, uz);  // raw moments of the deviations
  const T one = splat<T>(1.0f);
  const T mx[3] = {one, ux, vmul(ux, ux)}, my[3] = {one, uy, vmul(uy, uy)}, mz[3] = {one, uz, vmul(uz, uz)};
  if (D == 3) {
#pragma unroll
    for (int v = 4; v < 27; ++v) {
      const int t = d3q27_mode_tensor(v);
      T &k = F[t / 9][(t / 3) % 3][t % 3];
      const T keq = vmul(vmul(rho, mx[t % 3]), vmul(my[(t / 3) % 3], mz[t / 9]));
      k = vfma(splat<T>(rates.om(v)), vsub(k, keq), vmul(splat<T>(tile_scale<3>(v)), keq));
    }
    if (NOISE) {
#pragma unroll
      for (int blk = 0; blk < 6; ++blk) {
        T z[4];
        normals4_scaled<T>(site0, step_lo, step_hi, (uint32_t)blk, keys, rho, z, dsite);
        switch (blk) {
          case 0: add_noise_block<0>(F, rates, z); break;
          case 1: add_noise_block<1>(F, rates, z); break;
          case 2: add_noise_block<2>(F, rates, z); break;
          case 3: add_noise_block<3>(F, rates, z); break;
          case 4: add_noise_block<4>(F, rates, z); break;
          default: add_noise_block<5>(F, rates, z); break;
        }
      }
    }
    const T h = splat<T>(0.5f);  // momentum slots in the halved convention
    F[0][0][1] = vmul(h, F[0][0][1]);
    F[0][1][0] = vmul(h, F[0][1][0]);
    F[1][0][0] = vmul(h, F[1][0][0]);
  } else {
    const T rxx = F[1][0][2], ryy = F[1][2][0];
    const T exx = vmul(rho, mx[2]), eyy = vmul(rho, my[2]);
    T k[9], keq[9];
    k[3] = vadd(rxx, ryy);
    keq[3] = vadd(exx, eyy);
    k[4] = vsub(rxx, ryy);
    keq[4] = vsub(exx, eyy);
    k[5] = F[1][1][1];
    keq[5] = vmul(vmul(rho, ux), uy);
    k[6] = F[1][1][2];
    keq[6] = vmul(exx, uy);
    k[7] = F[1][2][1];
    keq[7] = vmul(eyy, ux);
    k[8] = F[1][2][2];
    keq[8] = vmul(exx, my[2]);
#pragma unroll
    for (int v = 3; v < 9; ++v)
      k[v] = vfma(splat<T>(rates.om(v)), vsub(k[v], keq[v]), vmul(splat<T>(tile_scale<2>(v)), keq[v]));
    if (NOISE) {
      T z0[4], z1[4];
      normals4_scaled<T>(site0, step_lo, step_hi, 0u, keys, rho, z0, dsite);
      normals4_scaled<T>(site0, step_lo, step_hi, 1u, keys, rho, z1, dsite);
#pragma unroll
      for (int v = 3; v < 9; ++v) k[v] = vfma(splat<T>(rates.phc(v)), v < 7 ? z0[v - 3] : z1[v - 7], k[v]);
    }
    const T h = splat<T>(0.5f);
    F[1][0][2] = vmul(h, vadd(k[3], k[4]));
    F[1][2][0] = vmul(h, vsub(k[3], k[4]));
    F[1][1][1] = k[5];
    F[1][1][2] = k[6];
    F[1][2][1] = k[7];
    F[1][2][2] = k[8];
    F[1][0][1] = vmul(h, F[1][0][1]);
    F[1][1][0] = vmul(h, F[1][1][0]);
  }
  tile_raw_inv_h<D>(F);  // entry (0,0,0) still holds rho - rho0
}

template <int D, bool NOISE, typename T, bool ROLLED = false, bool SHEAR = false, bool ISO = false, typename R,
          typename K>
__device__ __forceinline__ void collide_rates(T (&F)[3][3][3], float rho0, const R &rates, uint32_t site0,
                                              uint32_t step_lo, uint32_t step_hi, const K &keys,
                                              uint32_t dsite = 1) {
  static_assert(!ISO || D == 3, "the isotropic variant is a D3Q27 basis");
  T drho, rho, ux, uy, uz;
  T Pm[3];  // D3Q27, paper structure: raw P_xy, P_xz, P_yz
  if (SHEAR && D == 3 && !ISO) {
    T jv[3];
    shear_raw_moments(F, drho, jv, Pm);
    rho = vadd(splat<T>(rho0), drho);
    const T inv_rho = rcp_fast_lanes(rho);
    ux = vmul(jv[0], inv_rho);
    uy = vmul(jv[1], inv_rho);
    uz = vmul(jv[2], inv_rho);
    mom<D>(F, 0, 0, 0) = rho;  // k*_0 = rho for the way back
  } else if (SHEAR) {
    site_macros<D>(F, rho0, drho, rho, ux, uy, uz);
    mom<D>(F, 0, 0, 0) = rho;  // k*_0 = rho for the way back
    if (D == 3) {
      Pm[0] = F[0][1][1];
      Pm[1] = F[1][0][1];
      Pm[2] = F[1][1][0];
    }
  } else {
    site_central_moments<D>(F, rho0, drho, rho, ux, uy, uz);
  }
  if (D == 3) {
    if (SHEAR) {
      // raw (1,1,0), (1,0,1), (0,1,1) -> central; every other non-conserved mode restarts
      // from k^eq = 0 (ISO: also the normal stresses, rotated).
      const T nrho = vmul(splat<T>(-1.0f), rho);
      const T kxy = vfma(vmul(nrho, ux), uy, Pm[0]);
      const T kxz = vfma(vmul(nrho, ux), uz, Pm[1]);
      const T kyz = vfma(vmul(nrho, uy), uz, Pm[2]);
      T kxx, kyy, kzz;
      if (ISO) {
        kxx = vfma(vmul(nrho, ux), ux, F[0][0][2]);
        kyy = vfma(vmul(nrho, uy), uy, F[0][2][0]);
        kzz = vfma(vmul(nrho, uz), uz, F[2][0][0]);
        iso_rotate(kxx, kyy, kzz);
      }
#pragma unroll
      for (int v = 4; v < 27; ++v) {
        const int t = d3q27_mode_tensor(v);
        F[t / 9][(t / 3) % 3][t % 3] = splat<T>(0.0f);
      }
      F[0][1][1] = vmul(splat<T>(rates.om(7)), kxy);
      F[1][0][1] = vmul(splat<T>(rates.om(8)), kxz);
      F[1][1][0] = vmul(splat<T>(rates.om(9)), kyz);
      if (ISO) {
        F[0][0][2] = vmul(splat<T>(rates.om(4)), kxx);
        F[0][2][0] = vmul(splat<T>(rates.om(5)), kyy);
        F[2][0][0] = vmul(splat<T>(rates.om(6)), kzz);
      }
    } else {
      if (ISO) iso_rotate(F[0][0][2], F[0][2][0], F[2][0][0]);
#pragma unroll
      for (int v = 4; v < 27; ++v) {
        const int t = d3q27_mode_tensor(v);
        T &k = F[t / 9][(t / 3) % 3][t % 3];
        k = vmul(splat<T>(rates.om(v)), k);
      }
    }
    if (NOISE && ROLLED) {
#pragma unroll 1
      for (int blk = 0; blk < 6; ++blk) {
        T z[4];
        normals4_scaled<T>(site0, step_lo, step_hi, (uint32_t)blk, keys, rho, z, dsite);
        switch (blk) {  // block-uniform branch: modes 4 + 4 blk .. 7 + 4 blk
          case 0: add_noise_block<0>(F, rates, z); break;
          case 1: add_noise_block<1>(F, rates, z); break;
          case 2: add_noise_block<2>(F, rates, z); break;
          case 3: add_noise_block<3>(F, rates, z); break;
          case 4: add_noise_block<4>(F, rates, z); break;
          default: add_noise_block<5>(F, rates, z); break;
        }
      }
    } else if (NOISE) {
#pragma unroll
      for (int blk = 0; blk < 6; ++blk) {
        T z[4];
        normals4_scaled<T>(site0, step_lo, step_hi, (uint32_t)blk, keys, rho, z, dsite);
        switch (blk) {
          case 0: add_noise_block<0>(F, rates, z); break;
          case 1: add_noise_block<1>(F, rates, z); break;
          case 2: add_noise_block<2>(F, rates, z); break;
          case 3: add_noise_block<3>(F, rates, z); break;
          case 4: add_noise_block<4>(F, rates, z); break;
          default: add_noise_block<5>(F, rates, z); break;
        }
      }
    }
    if (ISO) iso_unrotate_h(F[0][0][2], F[0][2][0], F[2][0][0]);
    F[0][0][1] = splat<T>(0.0f);  // k*_1 (x momentum, central)
    F[0][1][0] = splat<T>(0.0f);  // k*_2
    F[1][0][0] = splat<T>(0.0f);  // k*_3
  } else {
    // D2Q9: modes 3 and 4 are the sum and difference of the (2,0) and (0,2) moments.
    T k3, k4, k5, k6, k7, k8;
    if (SHEAR) {
      // k4 = r_xx - r_yy - rho (ux^2 - uy^2), k5 = r_xy - rho ux uy (Sec. II-B); the
      // other non-conserved modes restart from k^eq = 0.
      const T nrho = vmul(splat<T>(-1.0f), rho);
      const T d2 = vsub(vmul(ux, ux), vmul(uy, uy));
      k4 = vmul(splat<T>(rates.om(4)), vfma(nrho, d2, vsub(F[1][0][2], F[1][2][0])));
      k5 = vmul(splat<T>(rates.om(5)), vfma(vmul(nrho, ux), uy, F[1][1][1]));
      k3 = k6 = k7 = k8 = splat<T>(0.0f);
    } else {
      const T kxx = F[1][0][2], kyy = F[1][2][0];
      k3 = vmul(splat<T>(rates.om(3)), vadd(kxx, kyy));
      k4 = vmul(splat<T>(rates.om(4)), vsub(kxx, kyy));
      k5 = vmul(splat<T>(rates.om(5)), F[1][1][1]);
      k6 = vmul(splat<T>(rates.om(6)), F[1][1][2]);
      k7 = vmul(splat<T>(rates.om(7)), F[1][2][1]);
      k8 = vmul(splat<T>(rates.om(8)), F[1][2][2]);
    }
    if (NOISE) {
      T z0[4], z1[4];
      normals4_scaled<T>(site0, step_lo, step_hi, 0u, keys, rho, z0, dsite);
      normals4_scaled<T>(site0, step_lo, step_hi, 1u, keys, rho, z1, dsite);
      k3 = vfma(splat<T>(rates.phc(3)), z0[0], k3);
      k4 = vfma(splat<T>(rates.phc(4)), z0[1], k4);
      k5 = vfma(splat<T>(rates.phc(5)), z0[2], k5);
      k6 = vfma(splat<T>(rates.phc(6)), z0[3], k6);
      k7 = vfma(splat<T>(rates.phc(7)), z1[0], k7);
      k8 = vfma(splat<T>(rates.phc(8)), z1[1], k8);
    }
    const T h = splat<T>(0.5f);
    F[1][0][2] = vmul(h, vadd(k3, k4));
    F[1][2][0] = vmul(h, vsub(k3, k4));
    F[1][1][1] = k5;
    F[1][1][2] = k6;
    F[1][2][1] = k7;
    F[1][2][2] = k8;
    F[1][0][1] = splat<T>(0.0f);  // k*_1
    F[1][1][0] = splat<T>(0.0f);  // k*_2
  }
  // r* = N^{-1} k* (entry (0,0,0) = k*_0 = rho), then d* = M^{-1} r* - w rho0, on the tile
  // in the halved convention (every other entry already carries its tile scale).
  tile_shift_inv_h<D>(F, ux, uy, uz);
  mom<D>(F, 0, 0, 0) = drho;
  tile_raw_inv_h<D>(F);
}

// The collision with per-mode arrays om_v, phc_v (kernel arguments).
// dsite: site index of a pair's lane y minus that of lane x (1, or 1 - nx across a row's end).
// RAW: the raw-moment counterpart (collide_raw).
template <int D, bool NOISE, typename T, bool ROLLED = false, bool SHEAR = false, bool ISO = false,
          bool RAW = false>
__device__ __forceinline__ void collide_tile(T (&F)[3][3][3], float rho0, const float *om,
                                             const float *phc, uint32_t site0, uint32_t step_lo,
                                             uint32_t step_hi, const uint32_t *ks0,
                                             const uint32_t *ks1, uint32_t dsite = 1) {
  if constexpr (RAW)
    collide_raw<D, NOISE, T>(F, rho0, ArrayRates{om, phc}, site0, step_lo, step_hi, KeyTable{ks0, ks1}, dsite);
  else
    collide_rates<D, NOISE, T, ROLLED, SHEAR, ISO>(F, rho0, ArrayRates{om, phc}, site0, step_lo, step_hi,
                                                   KeyTable{ks0, ks1}, dsite);
}

}  // namespace flbm
