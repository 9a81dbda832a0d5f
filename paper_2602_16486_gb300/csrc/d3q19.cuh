// D3Q19 (Sec. II-C, "Lattice-agnostic construction and the D3Q19 example"): the per-site
// algebra of the fused step and its AA-pattern population access.
//
// Velocities are the first 19 of the D3Q27 order (Lat<3>: rest, axes, face diagonals), so
// population i of D3Q19 is plane i of a 19-plane array, addressed exactly as D3Q27 with
// the eight corners left out. The moment transforms are the generated straight-line code
// of d3q19_gen.cuh (raw moments, central shift N(u), its inverse by forward substitution,
// populations from raw moments); the collision is Eq. cm_collision with k^eq = (rho, 0,
// ...), phi_v = sqrt(rho) phc_v and the noisy modes v = 4..18 fed by Philox blocks
// (v - 4) / 4, slot (v - 4) mod 4, as for the other lattices.
#pragma once

#include "cm.cuh"
#include "collide.cuh"
#include "d3q19_gen.cuh"
#include "philox.cuh"

namespace flbm {

__host__ __device__ constexpr bool d3q19_has(int dx, int dy, int dz) { return dx * dx + dy * dy + dz * dz < 3; }

// ---- population access, AA pattern (as load_logical / store_streamed) --------------------
template <typename S, int PARITY>
__device__ __forceinline__ void load19(const S *__restrict__ f, long long plane, const Neighbourhood &nb,
                                       float (&F)[19]) {
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (!d3q19_has(dx, dy, dz)) continue;
        const int i = Lat<3>::index(dx, dy, dz);
        const S *p = PARITY == 0 ? f + i * plane + nb.row[1][1] + nb.xs[1]
                                 : f + opposite<3>(i) * plane + nb.row[1 - dz][1 - dy] + nb.xs[1 - dx];
        F[i] = Storage<S>::load(p);
      }
}

template <typename S, int PARITY>
__device__ __forceinline__ void store19(S *__restrict__ f, long long plane, const Neighbourhood &nb,
                                        const float (&F)[19]) {
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (!d3q19_has(dx, dy, dz)) continue;
        const int i = Lat<3>::index(dx, dy, dz);
        S *p = PARITY == 0 ? f + opposite<3>(i) * plane + nb.row[1][1] + nb.xs[1]
                           : f + i * plane + nb.row[1 + dz][1 + dy] + nb.xs[1 + dx];
        Storage<S>::store(p, F[i]);
      }
}

template <typename S, int PARITY>
__device__ __forceinline__ void load19_2(const S *__restrict__ f, long long plane, const Addr2 &ad,
                                         float2 (&F)[19]) {
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (!d3q19_has(dx, dy, dz)) continue;
        const int i = Lat<3>::index(dx, dy, dz);
        float2 v;
        if (PARITY == 0) {
          v = Storage2<S>::load(f + i * plane + ad.s0);
        } else {
          const S *b = f + opposite<3>(i) * plane + ad.dy[1 - dy] + ad.dz[1 - dz];
          if (dx == 0) {
            v = Storage2<S>::load(b + ad.s0);
          } else if (dx == 1) {
            v.x = Storage<S>::load(b + ad.sm1);
            v.y = Storage<S>::load(b + ad.s0);
          } else {
            v.x = Storage<S>::load(b + ad.s0 + 1);
            v.y = Storage<S>::load(b + ad.sp2);
          }
        }
        F[i] = v;
      }
}

template <typename S, int PARITY>
__device__ __forceinline__ void store19_2(S *__restrict__ f, long long plane, const Addr2 &ad,
                                          const float2 (&F)[19]) {
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (!d3q19_has(dx, dy, dz)) continue;
        const int i = Lat<3>::index(dx, dy, dz);
        const float2 v = F[i];
        if (PARITY == 0) {
          Storage2<S>::store(f + opposite<3>(i) * plane + ad.s0, v);
        } else {
          S *b = f + i * plane + ad.dy[1 + dy] + ad.dz[1 + dz];
          if (dx == 0) {
            Storage2<S>::store(b + ad.s0, v);
          } else if (dx == 1) {
            Storage<S>::store(b + ad.s0 + 1, v.x);
            Storage<S>::store(b + ad.sp2, v.y);
          } else {
            Storage<S>::store(b + ad.sm1, v.x);
            Storage<S>::store(b + ad.s0, v.y);
          }
        }
      }
}

// The pairing of load_pairs / store_pairs (cm.cuh): on odd steps lanes hold x0 + 1 and x0 + 2,
// so the populations with c_x = +-1 (10 of 19) move as aligned pairs.
template <typename S, int PARITY>
__device__ __forceinline__ void load19_pairs(const S *__restrict__ f, long long plane, const Addr2 &ad,
                                             float2 (&F)[19]) {
  if (PARITY == 0) {
    load19_2<S, 0>(f, plane, ad, F);
    return;
  }
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (!d3q19_has(dx, dy, dz)) continue;
        const int i = Lat<3>::index(dx, dy, dz);
        const S *b = f + opposite<3>(i) * plane + ad.dy[1 - dy] + ad.dz[1 - dz];
        float2 v;
        if (dx == 0) {
          v.x = Storage<S>::load(b + ad.s0 + 1);
          v.y = Storage<S>::load(b + ad.sp2);
        } else {
          v = Storage2<S>::load(b + (dx == 1 ? ad.s0 : ad.sp2));
        }
        F[i] = v;
      }
}
template <typename S, int PARITY>
__device__ __forceinline__ void store19_pairs(S *__restrict__ f, long long plane, const Addr2 &ad,
                                              const float2 (&F)[19]) {
  if (PARITY == 0) {
    store19_2<S, 0>(f, plane, ad, F);
    return;
  }
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        if (!d3q19_has(dx, dy, dz)) continue;
        const int i = Lat<3>::index(dx, dy, dz);
        S *b = f + i * plane + ad.dy[1 + dy] + ad.dz[1 + dz];
        const float2 v = F[i];
        if (dx == 0) {
          Storage<S>::store(b + ad.s0 + 1, v.x);
          Storage<S>::store(b + ad.sp2, v.y);
        } else {
          Storage2<S>::store(b + (dx == 1 ? ad.sp2 : ad.s0), v);
        }
      }
}

// rho, u and the raw moments of the deviations (r_0 = rho - rho0).
template <typename T>
__device__ __forceinline__ void d3q19_macros(const T (&F)[19], float rho0, T (&r)[19], T &rho, T &ux, T &uy,
                                             T &uz) {
  d3q19_raw(F, r);
  rho = vadd(splat<T>(rho0), r[0]);
  const T inv_rho = rcp_fast_lanes(rho);
  ux = vmul(r[1], inv_rho);
  uy = vmul(r[2], inv_rho);
  uz = vmul(r[3], inv_rho);
}

// The collision of one site (float) or two (float2); on return F holds the post-collision
// deviations. SHEAR: the paper's rates (1 except the shear modes 7-9), so only k_7..9 are
// formed. om_v = 1 - Lambda_v, phc_v = sqrt(kBT Lambda_v (2 - Lambda_v) b_v / cs^2).
template <bool NOISE, typename T, bool SHEAR, typename K>
__device__ __forceinline__ void collide19(T (&F)[19], float rho0, const float *om, const float *phc, uint32_t site0,
                                          uint32_t step_lo, uint32_t step_hi, const K &keys, uint32_t dsite = 1) {
  T r[19], rho, ux, uy, uz;
  d3q19_macros(F, rho0, r, rho, ux, uy, uz);
  const T jx = r[1], jy = r[2], jz = r[3], drho = r[0];
  if (SHEAR) {
    T k7, k8, k9;
    d3q19_shear_central(r, rho, ux, uy, uz, k7, k8, k9);
#pragma unroll
    for (int v = 4; v < 19; ++v) r[v] = splat<T>(0.0f);
    r[7] = vmul(splat<T>(om[7]), k7);
    r[8] = vmul(splat<T>(om[8]), k8);
    r[9] = vmul(splat<T>(om[9]), k9);
  } else {
    d3q19_central_lr(r, rho, ux, uy, uz);
#pragma unroll
    for (int v = 4; v < 19; ++v) r[v] = vmul(splat<T>(om[v]), r[v]);
  }
  if (NOISE) {
  #pragma unroll
    for (int blk = 0; blk < 4; ++blk) {
      T z[4];
      normals4_scaled<T>(site0, step_lo, step_hi, (uint32_t)blk, keys, rho, z, dsite);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int v = 4 + 4 * blk + j;
        if (v < 19) r[v] = vfma(splat<T>(phc[v]), z[j], r[v]);
      }
    }
  }
  // The general rates keep more values live; they use the register-lean inverse.
  if (SHEAR)
    d3q19_raw_from_central(r, rho, ux, uy, uz);
  else
    d3q19_raw_from_central_lr(r, rho, ux, uy, uz);
  r[0] = drho;  // populations as deviations from w rho0
  r[1] = jx;    // r*_a = j_a (momentum conserved)
  r[2] = jy;
  r[3] = jz;
  d3q19_pop(r, F);
}

}  // namespace flbm
