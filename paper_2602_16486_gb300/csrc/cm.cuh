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
#include "vec.cuh"

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
  __device__ __forceinline__ static float load(const __nv_bfloat16 *p) {
    return __uint_as_float((uint32_t)(*reinterpret_cast<const unsigned short *>(p)) << 16);
  }
  __device__ __forceinline__ static void store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
};
template <>
struct Storage<__half> {
  __device__ __forceinline__ static float load(const __half *p) { return __half2float(*p); }
  __device__ __forceinline__ static void store(__half *p, float v) { *p = __float2half_rn(v); }
};

// ---- 1-D building blocks (T = float: one site; T = float2: two sites) -----------------
// In: p0 = v(c=-1), p1 = v(c=0), p2 = v(c=+1). Out: p0 = sum v, p1 = sum c v,
// p2 = sum (c^2 - cs^2) v.
template <typename T>
__device__ __forceinline__ void raw_fwd(T &p0, T &p1, T &p2) {
  const T e = vadd(p2, p0);
  const T s = vadd(p1, e);
  const T d = vsub(p2, p0);
  p2 = vfma(splat<T>(-kCs2), s, e);
  p1 = d;
  p0 = s;
}

// Inverse of raw_fwd.
template <typename T>
__device__ __forceinline__ void raw_inv(T &p0, T &p1, T &p2) {
  const T s = p0, d = p1;
  const T e = vfma(splat<T>(kCs2), s, p2);
  p1 = vsub(s, e);
  p2 = vmul(splat<T>(0.5f), vadd(e, d));
  p0 = vmul(splat<T>(0.5f), vsub(e, d));
}

// Raw -> central moments along one axis; nu = -u (velocity component, negated).
template <typename T>
__device__ __forceinline__ void shift_fwd(T &m0, T &m1, T &m2, T nu) {
  const T k1 = vfma(nu, m0, m1);
  m2 = vfma(nu, vadd(m1, k1), m2);
  m1 = k1;
}

// Central -> raw moments along one axis (inverse of shift_fwd), velocity component u.
template <typename T>
__device__ __forceinline__ void shift_inv(T &k0, T &k1, T &k2, T u) {
  const T r1 = vfma(u, k0, k1);
  k2 = vfma(u, vadd(k1, r1), k2);
  k1 = r1;
}

// The inverses in the halved convention: along the transformed axis the slots of order 1
// and 2 hold half their moment (order 0 is whole). raw_inv_h takes (s, p1/2, p2/2) and
// gives the three values, (v(+1), v(-1)) = (cs^2 s + p2 +- p1) / 2 and v(0) = s - cs^2 s - p2,
// in 4 operations instead of 6; shift_inv_h keeps the convention (hu = u / 2).
template <typename T>
__device__ __forceinline__ void raw_inv_h(T &p0, T &p1, T &p2) {
  const T s = p0;
  const T e = vfma(splat<T>(0.5f * kCs2), s, p2);  // (cs^2 s + p2) / 2
  p0 = vsub(e, p1);
  p2 = vadd(e, p1);
  p1 = vfma(splat<T>(-2.0f), e, s);
}

template <typename T>
__device__ __forceinline__ void shift_inv_h(T &k0, T &k1, T &k2, T u, T hu) {
  const T r1 = vfma(hu, k0, k1);   // (k1 + u k0) / 2
  k2 = vfma(u, vadd(k1, r1), k2);  // (k2 + 2 u k1 + u^2 k0) / 2
  k1 = r1;
}

// ---- tile transforms ---------------------------------------------------------------
// Tile layout: F[z][y][x]; for D = 2 only the plane z = 1 is used.
template <int D, typename T>
__device__ __forceinline__ void tile_raw_fwd(T (&F)[3][3][3]) {
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

template <int D, typename T>
__device__ __forceinline__ void tile_raw_inv(T (&F)[3][3][3]) {
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

// Central shift of all moments with the negated velocity (nux, nuy, nuz).
template <int D, typename T>
__device__ __forceinline__ void tile_shift_fwd(T (&F)[3][3][3], T nux, T nuy, T nuz) {
  constexpr int z0 = (D == 3) ? 0 : 1, z1 = (D == 3) ? 3 : 2;
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int b = 0; b < 3; ++b) shift_fwd(F[z][b][0], F[z][b][1], F[z][b][2], nux);
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int a = 0; a < 3; ++a) shift_fwd(F[z][0][a], F[z][1][a], F[z][2][a], nuy);
  if (D == 3) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) shift_fwd(F[0][b][a], F[1][b][a], F[2][b][a], nuz);
  }
}

template <int D, typename T>
__device__ __forceinline__ void tile_shift_inv(T (&F)[3][3][3], T ux, T uy, T uz) {
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

// Inverses of the whole tile in the halved convention (tile_scale in lattice.cuh): central
// moments scaled by 2^-(nonzero orders) -> raw moments (same scaling) -> populations.
template <int D, typename T>
__device__ __forceinline__ void tile_shift_inv_h(T (&F)[3][3][3], T ux, T uy, T uz) {
  constexpr int z0 = (D == 3) ? 0 : 1, z1 = (D == 3) ? 3 : 2;
  const T h = splat<T>(0.5f);
  if (D == 3) {
    const T huz = vmul(h, uz);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) shift_inv_h(F[0][b][a], F[1][b][a], F[2][b][a], uz, huz);
  }
  const T huy = vmul(h, uy), hux = vmul(h, ux);
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int a = 0; a < 3; ++a) shift_inv_h(F[z][0][a], F[z][1][a], F[z][2][a], uy, huy);
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int b = 0; b < 3; ++b) shift_inv_h(F[z][b][0], F[z][b][1], F[z][b][2], ux, hux);
}

template <int D, typename T>
__device__ __forceinline__ void tile_raw_inv_h(T (&F)[3][3][3]) {
  constexpr int z0 = (D == 3) ? 0 : 1, z1 = (D == 3) ? 3 : 2;
  if (D == 3) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) raw_inv_h(F[0][b][a], F[1][b][a], F[2][b][a]);
  }
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int a = 0; a < 3; ++a) raw_inv_h(F[z][0][a], F[z][1][a], F[z][2][a]);
#pragma unroll
  for (int z = z0; z < z1; ++z)
#pragma unroll
    for (int y = 0; y < 3; ++y) raw_inv_h(F[z][y][0], F[z][y][1], F[z][y][2]);
}

// Moment (a, b, c) of the tile after the forward transforms (c = 0 for D = 2).
template <int D, typename T>
__device__ __forceinline__ T &mom(T (&F)[3][3][3], int a, int b, int c) {
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

// ---- two sites per thread: x0 and x0 + 1 (x0 even, nx even) ------------------------------
// Pair loads/stores of two consecutive x; the array is 2-element aligned because nx is
// even and the buffer is 256-byte aligned.
template <typename S>
struct Storage2;
template <>
struct Storage2<float> {
  __device__ __forceinline__ static float2 load(const float *p) { return *reinterpret_cast<const float2 *>(p); }
  __device__ __forceinline__ static void store(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
};
template <>
struct Storage2<__nv_bfloat16> {
  __device__ __forceinline__ static float2 load(const __nv_bfloat16 *p) {
    // bf16 is the top half of an FP32 word: two bit operations per pair.
    const uint32_t x = *reinterpret_cast<const uint32_t *>(p);
    return make_float2(__uint_as_float(x << 16), __uint_as_float(x & 0xFFFF0000u));
  }
  __device__ __forceinline__ static void store(__nv_bfloat16 *p, float2 v) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(v.x, v.y);
  }
};
template <>
struct Storage2<__half> {
  __device__ __forceinline__ static float2 load(const __half *p) {
    return __half22float2(*reinterpret_cast<const __half2 *>(p));
  }
  __device__ __forceinline__ static void store(__half *p, float2 v) {
    *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v.x, v.y);
  }
};

// Site indices of a thread's pair and the periodic row / plane offsets of its block.
// y and z are fixed per block, so dy and dz are the same for every thread of it; only
// s0, sm1 and sp2 (the x seam) vary between threads.
struct Addr2 {
  long long s0;          // site x0
  long long sm1, sp2;    // sites x0 - 1 and x0 + 2 of the same row (periodic)
  long long dy[3];       // offset of row y - 1, y, y + 1 (periodic)
  long long dz[3];       // offset of plane z - 1, z, z + 1 (periodic)
};

__device__ __forceinline__ Addr2 addr2(int x0, int y, int z, int nx, int ny, int nz) {
  Addr2 a;
  a.s0 = ((long long)z * ny + y) * nx + x0;
  a.sm1 = a.s0 + (x0 == 0 ? nx - 1 : -1);
  a.sp2 = a.s0 + (x0 + 2 == nx ? 2 - nx : 2);
  const long long row = nx, pl = (long long)nx * ny;
  a.dy[0] = (y == 0) ? (long long)(ny - 1) * row : -row;
  a.dy[1] = 0;
  a.dy[2] = (y == ny - 1) ? -(long long)(ny - 1) * row : row;
  a.dz[0] = (z == 0) ? (long long)(nz - 1) * pl : -pl;
  a.dz[1] = 0;
  a.dz[2] = (z == nz - 1) ? -(long long)(nz - 1) * pl : pl;
  return a;
}

// As load_logical, for the pair: lane x holds site x0, lane y site x0 + 1.
template <int D, typename S, int PARITY>
__device__ __forceinline__ void load_logical2(const S *__restrict__ f, long long plane, const Addr2 &ad,
                                              float2 (&F)[3][3][3]) {
  constexpr int z0 = (D == 3) ? -1 : 0, z1 = (D == 3) ? 1 : 0;
#pragma unroll
  for (int dz = z0; dz <= z1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = Lat<D>::index(dx, dy, dz);
        float2 v;
        if (PARITY == 0) {
          v = Storage2<S>::load(f + i * plane + ad.s0);
        } else {
          // f_i(x) = A[opposite(i)][x - c_i]
          const S *b = f + opposite<D>(i) * plane + ad.dy[1 - dy] + ad.dz[1 - dz];
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
        F[dz + 1][dy + 1][dx + 1] = v;
      }
}

// As store_streamed, for the pair.
template <int D, typename S, int PARITY>
__device__ __forceinline__ void store_streamed2(S *__restrict__ f, long long plane, const Addr2 &ad,
                                                const float2 (&F)[3][3][3]) {
  constexpr int z0 = (D == 3) ? -1 : 0, z1 = (D == 3) ? 1 : 0;
#pragma unroll
  for (int dz = z0; dz <= z1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = Lat<D>::index(dx, dy, dz);
        const float2 v = F[dz + 1][dy + 1][dx + 1];
        if (PARITY == 0) {
          Storage2<S>::store(f + opposite<D>(i) * plane + ad.s0, v);
        } else {
          // f*_i(x) goes to A[i][x + c_i]
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

// Pairs of the step kernels: on even steps (PARITY 0) lane x holds site x0 and lane y site
// x0 + 1; on odd steps lane x holds x0 + 1 and lane y x0 + 2, which is the row's first site
// when x0 + 2 = nx (ad.sp2). An odd step reads slot opposite(i) at x - c_i and writes slot i
// at x + c_i, so with this pairing the populations with c_x = +-1 (18 of 27 on D3Q27) move as
// aligned pairs, (x0, x0 + 1) or (x0 + 2, x0 + 3), and only those with c_x = 0 take two scalar
// accesses. Every site of a row is still covered once.
template <int D, typename S, int PARITY>
__device__ __forceinline__ void load_pairs(const S *__restrict__ f, long long plane, const Addr2 &ad,
                                           float2 (&F)[3][3][3]) {
  if (PARITY == 0) {
    load_logical2<D, S, 0>(f, plane, ad, F);
    return;
  }
  constexpr int z0 = (D == 3) ? -1 : 0, z1 = (D == 3) ? 1 : 0;
#pragma unroll
  for (int dz = z0; dz <= z1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = Lat<D>::index(dx, dy, dz);
        const S *b = f + opposite<D>(i) * plane + ad.dy[1 - dy] + ad.dz[1 - dz];  // row of x - c_i
        float2 v;
        if (dx == 0) {
          v.x = Storage<S>::load(b + ad.s0 + 1);
          v.y = Storage<S>::load(b + ad.sp2);
        } else {
          v = Storage2<S>::load(b + (dx == 1 ? ad.s0 : ad.sp2));
        }
        F[dz + 1][dy + 1][dx + 1] = v;
      }
}

template <int D, typename S, int PARITY>
__device__ __forceinline__ void store_pairs(S *__restrict__ f, long long plane, const Addr2 &ad,
                                            const float2 (&F)[3][3][3]) {
  if (PARITY == 0) {
    store_streamed2<D, S, 0>(f, plane, ad, F);
    return;
  }
  constexpr int z0 = (D == 3) ? -1 : 0, z1 = (D == 3) ? 1 : 0;
#pragma unroll
  for (int dz = z0; dz <= z1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = Lat<D>::index(dx, dy, dz);
        S *b = f + i * plane + ad.dy[1 + dy] + ad.dz[1 + dz];  // row of x + c_i
        const float2 v = F[dz + 1][dy + 1][dx + 1];
        if (dx == 0) {
          Storage<S>::store(b + ad.s0 + 1, v.x);
          Storage<S>::store(b + ad.sp2, v.y);
        } else {
          Storage2<S>::store(b + (dx == 1 ? ad.sp2 : ad.s0), v);
        }
      }
}

// Site index of a pair's lane x and the step from it to lane y (the pairing of load_pairs).
template <int PARITY>
__device__ __forceinline__ uint32_t pair_site0(const Addr2 &ad) {
  return (uint32_t)(PARITY == 0 ? ad.s0 : ad.s0 + 1);
}
template <int PARITY>
__device__ __forceinline__ uint32_t pair_dsite(const Addr2 &ad) {
  return PARITY == 0 ? 1u : (uint32_t)(ad.sp2 - ad.s0 - 1);
}

// Raw moments of the deviation tile and rho, u (Eq. macro); entry (0,0,0) stays rho - rho0.
template <int D, typename T>
__device__ __forceinline__ void site_macros(T (&F)[3][3][3], float rho0, T &drho, T &rho, T &ux, T &uy,
                                            T &uz) {
  tile_raw_fwd<D>(F);
  drho = mom<D>(F, 0, 0, 0);
  rho = vadd(splat<T>(rho0), drho);
  const T inv_rho = rcp_fast_lanes(rho);
  ux = vmul(mom<D>(F, 1, 0, 0), inv_rho);
  uy = vmul(mom<D>(F, 0, 1, 0), inv_rho);
  uz = (D == 3) ? vmul(mom<D>(F, 0, 0, 1), inv_rho) : splat<T>(0.0f);
}

// D3Q27 with the paper's rate structure needs only rho, j and the three mixed raw second
// moments (shear modes, Sec. II-C). Per-axis sums and first moments of the deviation tile
// (three passes that skip every second-order output): drho = sum d, j, and
// P = (P_xy, P_xz, P_yz) = sum (cx cy, cx cz, cy cz) d. The tile is left partly reduced.
template <typename T>
__device__ __forceinline__ void shear_raw_moments(T (&F)[3][3][3], T &drho, T (&j)[3], T (&P)[3]) {
  T r0[3][3], r1[3][3];  // [z][y]: sum over x, first moment in x
#pragma unroll
  for (int z = 0; z < 3; ++z)
#pragma unroll
    for (int y = 0; y < 3; ++y) {
      r0[z][y] = vadd(F[z][y][1], vadd(F[z][y][0], F[z][y][2]));
      r1[z][y] = vsub(F[z][y][2], F[z][y][0]);
    }
  T q00[3], q01[3], q10[3], q11[3];  // [z]: (x order, y order) = 00, 01 (c_y), 10 (c_x), 11 (c_x c_y)
#pragma unroll
  for (int z = 0; z < 3; ++z) {
    q00[z] = vadd(r0[z][1], vadd(r0[z][0], r0[z][2]));
    q01[z] = vsub(r0[z][2], r0[z][0]);
    q10[z] = vadd(r1[z][1], vadd(r1[z][0], r1[z][2]));
    q11[z] = vsub(r1[z][2], r1[z][0]);
  }
  drho = vadd(q00[1], vadd(q00[0], q00[2]));
  j[2] = vsub(q00[2], q00[0]);
  j[0] = vadd(q10[1], vadd(q10[0], q10[2]));
  P[1] = vsub(q10[2], q10[0]);  // c_x c_z
  j[1] = vadd(q01[1], vadd(q01[0], q01[2]));
  P[2] = vsub(q01[2], q01[0]);  // c_y c_z
  P[0] = vadd(q11[1], vadd(q11[0], q11[2]));  // c_x c_y
}

// Forward part shared by the step and the statistics: raw moments of the deviation
// tile, rho and u (Eq. macro), then central moments with entry (0,0,0) = rho.
template <int D, typename T>
__device__ __forceinline__ void site_central_moments(T (&F)[3][3][3], float rho0, T &drho, T &rho,
                                                     T &ux, T &uy, T &uz) {
  site_macros<D>(F, rho0, drho, rho, ux, uy, uz);
  mom<D>(F, 0, 0, 0) = rho;
  const T m1 = splat<T>(-1.0f);
  tile_shift_fwd<D>(F, vmul(m1, ux), vmul(m1, uy), vmul(m1, uz));
}

// ---- the isotropic D3Q27 variant ----------------------------------------------------------
// Modes 4-6 of the variant are the trace and two deviators of the normal-stress modes of
// Sec. II-C: M4' = M4 + M5 + M6, M5' = M4 - M5, M6' = M4 + M5 - 2 M6 (mutually orthogonal,
// norms 2/3, 4/9, 4/3). These map the three values in place.
template <typename T>
__device__ __forceinline__ void iso_rotate(T &a, T &b, T &c) {  // (k4, k5, k6) -> (M4', M5', M6')
  const T s = vadd(a, b);
  const T d1 = vsub(a, b);
  const T d2 = vfma(splat<T>(-2.0f), c, s);
  a = vadd(s, c);
  b = d1;
  c = d2;
}
// iso_unrotate, each output halved (the halved convention of the inverse transforms).
template <typename T>
__device__ __forceinline__ void iso_unrotate_h(T &a, T &b, T &c) {
  const T s4 = vmul(splat<T>(1.0f / 12.0f), vfma(splat<T>(2.0f), a, c));  // (k4 + k5) / 4
  const T k6 = vmul(splat<T>(1.0f / 6.0f), vsub(a, c));                   // k6 / 2
  const T k4 = vfma(splat<T>(0.25f), b, s4);   // ((k4 + k5) + (k4 - k5)) / 4
  const T k5 = vfma(splat<T>(-0.25f), b, s4);
  a = k4;
  b = k5;
  c = k6;
}
template <typename T>
__device__ __forceinline__ void iso_unrotate(T &a, T &b, T &c) {  // (M4', M5', M6') -> (k4, k5, k6)
  const T third = splat<T>(1.0f / 3.0f), half = splat<T>(0.5f);
  const T s = vmul(third, vfma(splat<T>(2.0f), a, c));  // k4 + k5 = (2 M4' + M6') / 3
  const T k6 = vmul(third, vsub(a, c));                 // (M4' - M6') / 3
  const T k4 = vmul(half, vadd(s, b));
  const T k5 = vmul(half, vsub(s, b));
  a = k4;
  b = k5;
  c = k6;
}

}  // namespace flbm
