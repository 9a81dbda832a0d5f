// Per-site central-moment algebra of the fused step, in registers.
//
// The paper writes k = T(u) f with T = N M (Sec. II-B): M maps populations to raw
// moments and N(u) shifts raw to central moments; the collision is Eq. cm_collision
// and the way back is r* = N^{-1} k*, f* = M^{-1} r* (Sec. II-B, Eqs. post_coll_rms and
// post_coll_pops). Because both bases are tensor products of the 1-D polynomials
// {1, c, c^2 - cs^2} (see lattice.cuh), M, N and their inverses factor into one 3-point
// transform per axis, applied to a 3x3x3 register tile F[z][y][x]:
//   raw    : (v(-1), v(0), v(+1)) -> (sum v, sum c v, sum (c^2 - cs^2) v)
//   shift  : (m0, m1, m2) -> (m0, m1 - u m0, m2 - 2u m1 + u^2 m0)
// and their inverses. This is an implementation choice: it computes the same T(u)
// the paper defines, in 3x(Q/3) small transforms instead of a dense Q x Q product.
//
// Deviation storage: the tile holds d_i = f_i - w_i rho0. The raw moments of w_i rho0
// vanish except the zeroth (= rho0), so only entry [0][0][0] differs between f and d;
// it is set to rho during the velocity shifts and back to rho - rho0 afterwards.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lattice.cuh"

namespace flbm {

// ---- storage conversion ---------------------------------------------------------
template <typename S>
struct Storage;
template <>
struct Storage<float> {
  __device__ __forceinline__ static float load(const float *p) { return *p; }
  __device__ __forceinline__ static void store(float *p, float v) { *p = v; }
};
template <>
struct Storage<__nv_bfloat16> {
  __device__ __forceinline__ static float load(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
  __device__ __forceinline__ static void store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};
template <>
struct Storage<__half> {
  __device__ __forceinline__ static float load(const __half *p) { return __half2float(*p); }
  __device__ __forceinline__ static void store(__half *p, float v) { *p = __float2half_rn(v); }
};

// ---- 1-D building blocks ---------------------------------------------------------
// In: p0 = v(c=-1), p1 = v(c=0), p2 = v(c=+1). Out: p0 = sum v, p1 = sum c v,
// p2 = sum (c^2 - cs^2) v.
__device__ __forceinline__ void raw_fwd(float &p0, float &p1, float &p2) {
  const float e = p2 + p0;
  const float s = p1 + e;
  const float d = p2 - p0;
  p2 = fmaf(-kCs2, s, e);
  p1 = d;
  p0 = s;
}

// Inverse of raw_fwd.
__device__ __forceinline__ void raw_inv(float &p0, float &p1, float &p2) {
  const float s = p0, d = p1;
  const float e = fmaf(kCs2, s, p2);
  p1 = s - e;
  p2 = 0.5f * (e + d);
  p0 = 0.5f * (e - d);
}

// Raw -> central moments along one axis with velocity component u.
__device__ __forceinline__ void shift_fwd(float &m0, float &m1, float &m2, float u) {
  const float k1 = fmaf(-u, m0, m1);
  m2 = fmaf(-u, m1 + k1, m2);
  m1 = k1;
}

// Central -> raw moments along one axis (inverse of shift_fwd).
__device__ __forceinline__ void shift_inv(float &k0, float &k1, float &k2, float u) {
  const float r1 = fmaf(u, k0, k1);
  k2 = fmaf(u, k1 + r1, k2);
  k1 = r1;
}

// ---- tile transforms ---------------------------------------------------------------
// Tile layout: F[z][y][x]; for D = 2 only the plane z = 1 is used.
template <int D>
__device__ __forceinline__ void tile_raw_fwd(float (&F)[3][3][3]) {
  constexpr int z0 = (D == 3) ? 0 : 1, z1 = (D == 3) ? 3 : 2;
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int y = 0; y < 3; ++y) raw_fwd(F[z][y][0], F[z][y][1], F[z][y][2]);
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int a = 0; a < 3; ++a) raw_fwd(F[z][0][a], F[z][1][a], F[z][2][a]);
  if (D == 3) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) raw_fwd(F[0][b][a], F[1][b][a], F[2][b][a]);
  }
}

template <int D>
__device__ __forceinline__ void tile_raw_inv(float (&F)[3][3][3]) {
  constexpr int z0 = (D == 3) ? 0 : 1, z1 = (D == 3) ? 3 : 2;
  if (D == 3) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) raw_inv(F[0][b][a], F[1][b][a], F[2][b][a]);
  }
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int a = 0; a < 3; ++a) raw_inv(F[z][0][a], F[z][1][a], F[z][2][a]);
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int y = 0; y < 3; ++y) raw_inv(F[z][y][0], F[z][y][1], F[z][y][2]);
}

template <int D>
__device__ __forceinline__ void tile_shift_fwd(float (&F)[3][3][3], float ux, float uy, float uz) {
  constexpr int z0 = (D == 3) ? 0 : 1, z1 = (D == 3) ? 3 : 2;
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int b = 0; b < 3; ++b) shift_fwd(F[z][b][0], F[z][b][1], F[z][b][2], ux);
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int a = 0; a < 3; ++a) shift_fwd(F[z][0][a], F[z][1][a], F[z][2][a], uy);
  if (D == 3) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) shift_fwd(F[0][b][a], F[1][b][a], F[2][b][a], uz);
  }
}

template <int D>
__device__ __forceinline__ void tile_shift_inv(float (&F)[3][3][3], float ux, float uy, float uz) {
  constexpr int z0 = (D == 3) ? 0 : 1, z1 = (D == 3) ? 3 : 2;
  if (D == 3) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) shift_inv(F[0][b][a], F[1][b][a], F[2][b][a], uz);
  }
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int a = 0; a < 3; ++a) shift_inv(F[z][0][a], F[z][1][a], F[z][2][a], uy);
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int b = 0; b < 3; ++b) shift_inv(F[z][b][0], F[z][b][1], F[z][b][2], ux);
}

// Moment (a, b, c) of the tile after the forward transforms (c = 0 for D = 2).
template <int D>
__device__ __forceinline__ float &mom(float (&F)[3][3][3], int a, int b, int c) {
  return D == 3 ? F[c][b][a] : F[1][b][a];
}

// Central moments of one site in the paper's mode order (Sec. II-B / II-C), from the
// tile after tile_shift_fwd with entry (0,0,0) = rho.
template <int D>
__device__ __forceinline__ void paper_modes(float (&F)[3][3][3], float *k) {
  if (D == 3) {
#pragma unroll
    for (int v = 0; v < 27; ++v) {
      const int t = d3q27_mode_tensor(v);
      k[v] = F[t / 9][(t / 3) % 3][t % 3];
    }
  } else {
#pragma unroll
    for (int v = 0; v < 9; ++v) {
      const int t = d2q9_mode_tensor(v);
      if (t >= 0) k[v] = F[1][t / 3][t % 3];
    }
    k[3] = F[1][0][2] + F[1][2][0];
    k[4] = F[1][0][2] - F[1][2][0];
  }
}

// ---- periodic neighbourhood and AA-pattern addressing -----------------------------------
struct Neighbourhood {
  int xs[3];          // x - 1, x, x + 1 (periodic)
  long long row[3][3];  // row[dz+1][dy+1]: index of the first site of row (y+dy, z+dz)
};

__device__ __forceinline__ Neighbourhood neighbourhood(int x, int y, int z, int nx, int ny, int nz) {
  Neighbourhood nb;
  nb.xs[0] = x == 0 ? nx - 1 : x - 1;
  nb.xs[1] = x;
  nb.xs[2] = x == nx - 1 ? 0 : x + 1;
  const int ys[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
  const int zs[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int k = 0; k < 3; ++k) nb.row[j][k] = ((long long)zs[j] * ny + ys[k]) * nx;
  return nb;
}

// Logical populations (deviations) arriving at the site, as stored after an even
// (PARITY 0: f_i(x) = A[i][x]) or odd (PARITY 1: f_i(x) = A[opposite(i)][x - c_i])
// number of AA-pattern steps. F[dz+1][dy+1][dx+1] holds the population of velocity
// (dx, dy, dz).
template <int D, typename S, int PARITY>
__device__ __forceinline__ void load_logical(const S *__restrict__ f, long long plane,
                                             const Neighbourhood &nb, float (&F)[3][3][3]) {
  constexpr int z0 = (D == 3) ? -1 : 0, z1 = (D == 3) ? 1 : 0;
#pragma unroll
  for (int dz = z0; dz <= z1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = Lat<D>::index(dx, dy, dz);
        const S *p;
        if (PARITY == 0)
          p = f + i * plane + nb.row[1][1] + nb.xs[1];
        else
          p = f + opposite<D>(i) * plane + nb.row[1 - dz][1 - dy] + nb.xs[1 - dx];
        F[dz + 1][dy + 1][dx + 1] = Storage<S>::load(p);
      }
}

// Post-collision populations written where the AA pattern keeps them: PARITY 0 writes
// f*_i(x) to A[opposite(i)][x]; PARITY 1 writes it to A[i][x + c_i].
template <int D, typename S, int PARITY>
__device__ __forceinline__ void store_streamed(S *__restrict__ f, long long plane,
                                               const Neighbourhood &nb, const float (&F)[3][3][3]) {
  constexpr int z0 = (D == 3) ? -1 : 0, z1 = (D == 3) ? 1 : 0;
#pragma unroll
  for (int dz = z0; dz <= z1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = Lat<D>::index(dx, dy, dz);
        S *p;
        if (PARITY == 0)
          p = f + opposite<D>(i) * plane + nb.row[1][1] + nb.xs[1];
        else
          p = f + i * plane + nb.row[1 + dz][1 + dy] + nb.xs[1 + dx];
        Storage<S>::store(p, F[dz + 1][dy + 1][dx + 1]);
      }
}

// Forward part shared by the step and the statistics: raw moments of the deviation
// tile, rho and u (Eq. macro), then central moments with entry (0,0,0) = rho.
template <int D>
__device__ __forceinline__ void site_central_moments(float (&F)[3][3][3], float rho0, float &drho,
                                                     float &rho, float &ux, float &uy, float &uz) {
  tile_raw_fwd<D>(F);
  drho = mom<D>(F, 0, 0, 0);
  rho = rho0 + drho;
  const float inv_rho = 1.0f / rho;
  ux = mom<D>(F, 1, 0, 0) * inv_rho;
  uy = mom<D>(F, 0, 1, 0) * inv_rho;
  uz = (D == 3) ? mom<D>(F, 0, 0, 1) * inv_rho : 0.0f;
  mom<D>(F, 0, 0, 0) = rho;
  tile_shift_fwd<D>(F, ux, uy, uz);
}

}  // namespace flbm
