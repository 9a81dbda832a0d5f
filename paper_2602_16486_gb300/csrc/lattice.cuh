// Device-side lattice tables for the fused step: D2Q9 (Sec. II-B), D3Q27 (Sec. II-C) and
// D3Q19 (Sec. II-C example) in the paper's velocity order, written as constexpr index functions so that every
// table lookup in an unrolled loop folds to a constant.
//
// Moment bookkeeping. Both orthogonal bases are (up to a rotation of two D2Q9 modes)
// tensor products of the 1-D polynomials P0 = 1, P1 = c, P2 = c^2 - cs^2:
//   D3Q27: M_v = P_a(c_x) P_b(c_y) P_c(c_z) with (a,b,c) = mode_tensor(v) below,
//   D2Q9 : M_3 = P2(x) + P2(y), M_4 = P2(x) - P2(y), every other M_v = P_a(x) P_b(y).
// The fused kernels therefore work on a 3x3x3 tensor of moments K[c][b][a] (a = x
// order, b = y order, c = z order) and translate to the paper's mode index v only in
// the collision.
#pragma once

#include <cstdint>

namespace flbm {

constexpr float kCs2 = 1.0f / 3.0f;

template <int D>
struct Lat;

// D2Q9, Sec. II-B: c_x = [0, 1, 0, -1, 0, 1, -1, -1, 1], c_y = [0, 0, 1, 0, -1, 1, 1, -1, -1].
template <>
struct Lat<2> {
  static constexpr int D = 2;
  static constexpr int Q = 9;
  __host__ __device__ static constexpr int index(int cx, int cy, int /*cz*/) {
    return (cx == 0 && cy == 0)   ? 0
           : (cy == 0)            ? (cx > 0 ? 1 : 3)
           : (cx == 0)            ? (cy > 0 ? 2 : 4)
           : (cx > 0 && cy > 0)   ? 5
           : (cx < 0 && cy > 0)   ? 6
           : (cx < 0 && cy < 0)   ? 7
                                  : 8;
  }
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
  }
  __host__ __device__ static constexpr int cz(int) { return 0; }
};

// D3Q27, Sec. II-C: rest; axis +-x, +-y, +-z (1..6); xy, xz, yz face diagonals
// (7..10, 11..14, 15..18, first component fastest, + before -); corners (19..26).
template <>
struct Lat<3> {
  static constexpr int D = 3;
  static constexpr int Q = 27;
  __host__ __device__ static constexpr int index(int cx, int cy, int cz) {
    return (cx == 0 && cy == 0 && cz == 0) ? 0
           : (cy == 0 && cz == 0)          ? (cx > 0 ? 1 : 2)
           : (cx == 0 && cz == 0)          ? (cy > 0 ? 3 : 4)
           : (cx == 0 && cy == 0)          ? (cz > 0 ? 5 : 6)
           : (cz == 0)                     ? 7 + (cx < 0) + 2 * (cy < 0)
           : (cy == 0)                     ? 11 + (cx < 0) + 2 * (cz < 0)
           : (cx == 0)                     ? 15 + (cy < 0) + 2 * (cz < 0)
                                           : 19 + (cx < 0) + 2 * (cy < 0) + 4 * (cz < 0);
  }
  __host__ __device__ static constexpr int cx(int i) {
    return i == 0 ? 0
           : i <= 6 ? (i == 1 ? 1 : i == 2 ? -1 : 0)
           : i <= 10 ? (((i - 7) & 1) ? -1 : 1)
           : i <= 14 ? (((i - 11) & 1) ? -1 : 1)
           : i <= 18 ? 0
                     : (((i - 19) & 1) ? -1 : 1);
  }
  __host__ __device__ static constexpr int cy(int i) {
    return i == 0 ? 0
           : i <= 6 ? (i == 3 ? 1 : i == 4 ? -1 : 0)
           : i <= 10 ? (((i - 7) & 2) ? -1 : 1)
           : i <= 14 ? 0
           : i <= 18 ? (((i - 15) & 1) ? -1 : 1)
                     : (((i - 19) & 2) ? -1 : 1);
  }
  __host__ __device__ static constexpr int cz(int i) {
    return i == 0 ? 0
           : i <= 6 ? (i == 5 ? 1 : i == 6 ? -1 : 0)
           : i <= 10 ? 0
           : i <= 14 ? (((i - 11) & 2) ? -1 : 1)
           : i <= 18 ? (((i - 15) & 2) ? -1 : 1)
                     : (((i - 19) & 4) ? -1 : 1);
  }
};

// D3Q19 (Sec. II-C, "Lattice-agnostic construction and the D3Q19 example"): the rest
// velocity, the six axes and the twelve face diagonals, i.e. the first 19 velocities of
// the D3Q27 order. Kernels that address populations by velocity take the lattice code 19.
template <>
struct Lat<19> {
  static constexpr int D = 3;
  static constexpr int Q = 19;
  __host__ __device__ static constexpr int index(int cx, int cy, int cz) { return Lat<3>::index(cx, cy, cz); }
  __host__ __device__ static constexpr int cx(int i) { return Lat<3>::cx(i); }
  __host__ __device__ static constexpr int cy(int i) { return Lat<3>::cy(i); }
  __host__ __device__ static constexpr int cz(int i) { return Lat<3>::cz(i); }
};

template <int D>
__host__ __device__ constexpr int opposite(int i) {
  return Lat<D>::index(-Lat<D>::cx(i), -Lat<D>::cy(i), -Lat<D>::cz(i));
}

// 1-D weights of c in {0, +-1}: 2/3 and 1/6. The lattice weight is their product.
__host__ __device__ constexpr double weight1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }

template <int D>
__host__ __device__ constexpr double weight(int i) {
  return D == 19 ? (i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0))  // D3Q19: not a product
                 : weight1d(Lat<D>::cx(i)) * weight1d(Lat<D>::cy(i)) * (D == 3 ? weight1d(Lat<D>::cz(i)) : 1.0);
}

// Tensor orders (a, b, c) of D3Q27 mode v (Sec. II-C basis, with M_15 = c_y^2 c_z - cs^2 c_z),
// packed as a + 3 b + 9 c.
__host__ __device__ constexpr int d3q27_mode_tensor(int v) {
  //                 v:  0  1  2  3   4   5   6  7   8   9  10  11  12  13  14  15  16  17  18  19  20  21  22  23  24  25  26
  return v == 0    ? 0
         : v == 1  ? 1
         : v == 2  ? 3
         : v == 3  ? 9
         : v == 4  ? 2
         : v == 5  ? 6
         : v == 6  ? 18
         : v == 7  ? 1 + 3
         : v == 8  ? 1 + 9
         : v == 9  ? 3 + 9
         : v == 10 ? 2 + 3
         : v == 11 ? 2 + 9
         : v == 12 ? 1 + 6
         : v == 13 ? 1 + 18
         : v == 14 ? 3 + 18
         : v == 15 ? 6 + 9
         : v == 16 ? 1 + 3 + 9
         : v == 17 ? 2 + 6
         : v == 18 ? 2 + 18
         : v == 19 ? 6 + 18
         : v == 20 ? 1 + 3 + 18
         : v == 21 ? 1 + 6 + 9
         : v == 22 ? 2 + 3 + 9
         : v == 23 ? 2 + 3 + 18
         : v == 24 ? 2 + 6 + 9
         : v == 25 ? 1 + 6 + 18
                   : 2 + 6 + 18;
}

// Tensor orders of the D2Q9 modes that are single tensor products (v = 0,1,2,5,6,7,8),
// packed as a + 3 b; modes 3 and 4 are the sum and difference of (2,0) and (0,2).
__host__ __device__ constexpr int d2q9_mode_tensor(int v) {
  return v == 0 ? 0 : v == 1 ? 1 : v == 2 ? 3 : v == 5 ? 4 : v == 6 ? 5 : v == 7 ? 7 : v == 8 ? 8 : -1;
}

// Scale of mode v in the tile the inverse transforms take (cm.cuh, tile_shift_inv_h and
// tile_raw_inv_h): 2^-n, n the number of axes along which the mode has a nonzero order.
// The collision writes k*_v times this scale, so that the 1/2 of every 3-point inverse
// is folded into its constants. D2Q9 modes 3 and 4 combine (2,0) and (0,2): 1/2.
__host__ __device__ constexpr int nonzero_orders(int t) {
  return (t % 3 != 0 ? 1 : 0) + ((t / 3) % 3 != 0 ? 1 : 0) + (t / 9 != 0 ? 1 : 0);
}
template <int D>
__host__ __device__ constexpr float tile_scale(int v) {
  return D == 3 ? 1.0f / float(1 << nonzero_orders(d3q27_mode_tensor(v)))
                : (v == 0 ? 1.0f : (v <= 4 ? 0.5f : 0.25f));
}

}  // namespace flbm
