// Gram-matrix accumulation of the statistics (Sec. III diagnostics and the mode
// covariances of Sec. II-B) for the statistics kernel (stats.cu).
//
// Every recorded sum is an entry of G = sum_x c(x) c(x)^T over the per-site column
//   c = [1, rho - rho0, j_x, j_y, j_z, u_x, u_y, u_z, k_{D+1} .. k_{Q-1}, 0 ...]
// (NC = 32 entries for D3Q27 and D3Q19, 16 for D2Q9). G is a dense contraction over the
// sites, so it runs on the tensor cores: warp-level mma.sync m16n8k16 with BF16 inputs and
// FP32 accumulation, the K dimension running over sites. Each input is split into
// x_hi = bf16(x) and x_lo = bf16(x - x_hi) (both rounded to nearest; x - x_hi is exact in
// FP32), and every product is formed as hi*hi + hi*lo + lo*hi + lo*lo: what is left out is
// the rounding of x_lo, about 2^-16 of x with either sign, so the products carry no bias
// and about 2^-15 relative error each. BF16 keeps FP32's exponent range, so no column needs
// scaling. A block of kStatsBlock threads works on tiles of 2 kStatsBlock sites, each
// thread on two: its pair packs into one bf16x2 word per column (the pair of K indices an
// MMA fragment register holds). Each warp owns 32 rows of the shared-memory tile (one row
// per thread, i.e. per site pair): its lanes stage the split columns there, and the warp
// accumulates the upper block-triangle of G over those 64 sites in FP32 fragments. Warps
// therefore only synchronise among their own lanes (__syncwarp), never with the block.
// The fragments go to the block's FP64 sums in shared memory every kFlushTiles tiles;
// at the end the block adds its sums to the output record with one FP64 atomic per
// entry. Output record: the upper triangle of G in FP64, row-major, then the number of
// non-finite sites.
#pragma once

#include <cuda_runtime.h>

#include "cm.cuh"
#include "internal.h"

namespace flbm {

template <int D>  // D: 2 (D2Q9), 3 (D3Q27) or 19 (D3Q19)
struct StatsPlan {
  static constexpr int NC = D == 2 ? 16 : 32;  // columns, padded to whole MMA tiles
  static constexpr int LD = 32;                // shared-memory row: 32 words (see chunk_pos)
  static constexpr int MT = NC / 16;           // 16-row tiles of G
  static constexpr int NT = NC / 8;            // 8-column tiles of G
  // Upper block-triangle: tiles (mt, nt) with nt >= 2 mt.
  static constexpr int NTILE = D == 2 ? 2 : 6;
  static constexpr int NREC = NC * (NC + 1) / 2;
};

namespace gram {

constexpr int kTileSites = 2 * kStatsBlock;  // two sites per thread
constexpr int kRows = kStatsBlock;           // staged rows: the site pair of every thread
constexpr int kFlushTiles = 16;  // FP32 sums over at most 16 x 64 sites per fragment entry
                                  // (a tile gives every warp 64 sites)

template <int D>
__host__ __device__ constexpr int tile_mt(int i) {
  return D != 2 ? (i < 4 ? 0 : 1) : 0;
}
template <int D>
__host__ __device__ constexpr int tile_nt(int i) {
  return D != 2 ? (i < 4 ? i : i - 2) : i;
}

// A shared-memory row holds the 32 words of one site pair in eight 16-byte chunks: chunk g
// carries the columns g, g + 8, g + 16, g + 24, which are the words a lane with
// g = lane / 4 needs for its A fragments (rows g and g + 8 of both 16-row tiles), so a
// fragment row comes in with one 16-byte load (8-byte for D2Q9, whose 16 columns use
// the first two words of a chunk). Chunk g of row r sits at position
// g ^ 2 (r mod 4) ^ (bit 2 of r): the eight lanes of each quarter-warp phase then hit
// eight different chunks both when staging (eight consecutive rows, one chunk) and when
// loading fragments (rows s0 + t or s0 + t + 4, chunks g).
__device__ __forceinline__ int chunk_pos(int g, int r) { return g ^ ((r & 3) << 1) ^ ((r >> 2) & 1); }

// bf16x2 of (a, b): a in the low half (the lower K index), b in the high half; rounded to
// nearest.
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}

// D (16x8, FP32) += A (16x16, BF16, row-major) * B (16x8, BF16, column-major). Not
// volatile: the compiler may interleave independent accumulations.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// The block's shared memory: BF16 high and low parts of the tile's columns (bf16x2 words,
// one per site pair and column), then the FP64 sums of every warp's fragments.
template <int D>
struct Smem {
  uint32_t *hi, *lo;
  double *acc64;  // [NTILE * 4][32]
};

template <int D>
__host__ __device__ constexpr size_t smem_bytes() {
  return 2 * sizeof(uint32_t) * kRows * StatsPlan<D>::LD + sizeof(double) * StatsPlan<D>::NTILE * 4 * 32;
}

template <int D>
__device__ __forceinline__ Smem<D> smem_layout(unsigned char *raw) {
  Smem<D> s;
  s.hi = reinterpret_cast<uint32_t *>(raw);
  s.lo = s.hi + kRows * StatsPlan<D>::LD;
  s.acc64 = reinterpret_cast<double *>(s.lo + kRows * StatsPlan<D>::LD);
  return s;
}

template <int D>
__device__ __forceinline__ void zero_acc64(const Smem<D> &s) {
  for (int e = threadIdx.x; e < StatsPlan<D>::NTILE * 4 * 32; e += blockDim.x) s.acc64[e] = 0.0;
}

// Columns of a pair (lane x: first site, lane y: second) from its central moments: F as
// left by site_central_moments (entry (0,0,0) = rho; Q = 27 or 9), drho = rho - rho0.
// v0 / v1: the site exists. A site whose column holds a NaN or an infinity makes the sum
// of its entries non-finite (the entries are far below overflow); such a site
// contributes a zero column (select, not multiply: it may hold NaN) and is counted.
template <int D, bool ISO, int NC>
__device__ __forceinline__ void moment_columns(const float2 (&F)[3][3][3], float2 drho, float2 rho, float2 ux,
                                               float2 uy, float2 uz, bool v0, bool v1, float2 (&col)[NC],
                                               unsigned &nonfinite) {
  constexpr int Q = Lat<D>::Q;
  float2 k[Q];
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
    k[3] = vadd(F[1][0][2], F[1][2][0]);
    k[4] = vsub(F[1][0][2], F[1][2][0]);
  }
  if (ISO) iso_rotate(k[4], k[5], k[6]);  // the isotropic variant's modes 4-6
  col[0] = make_float2(v0 ? 1.0f : 0.0f, v1 ? 1.0f : 0.0f);
  col[1] = drho;
  col[2] = vmul(rho, ux);
  col[3] = vmul(rho, uy);
  col[4] = vmul(rho, uz);
  col[5] = ux;
  col[6] = uy;
  col[7] = uz;
#pragma unroll
  for (int v = D + 1; v < Q; ++v) col[8 + v - D - 1] = k[v];
#pragma unroll
  for (int c = 8 + Q - D - 1; c < NC; ++c) col[c] = make_float2(0.0f, 0.0f);
  float2 sum = col[1];
#pragma unroll
  for (int c = 2; c < 8 + Q - D - 1; ++c) sum = vadd(sum, col[c]);
  const bool valid[2] = {v0, v1};
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    if (valid[l] && !isfinite(lane(sum, l))) {
      ++nonfinite;
#pragma unroll
      for (int c = 0; c < NC; ++c) set_lane(col[c], l, 0.0f);
    }
  }
}

// The row of this thread: 32 w + lane (w: its warp).
__device__ __forceinline__ int own_row() { return threadIdx.x; }

// Split columns of this thread's site pair (lane x: lower K index) into its row.
template <int D, int NC>
__device__ __forceinline__ void stage_columns(const Smem<D> &s, const float2 (&col)[NC]) {
  constexpr int LD = StatsPlan<D>::LD, P = NC / 8;  // words used per chunk
  const int r = own_row();
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    uint32_t h[4], e[4];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const float2 x = col[g + 8 * p];
      h[p] = pack_bf16x2(x.x, x.y);
      const float hx = __uint_as_float(h[p] << 16), hy = __uint_as_float(h[p] & 0xFFFF0000u);
      e[p] = pack_bf16x2(x.x - hx, x.y - hy);  // exact differences, rounded to BF16
    }
    const int w = r * LD + 4 * chunk_pos(g, r);
    if (P == 4) {
      *reinterpret_cast<uint4 *>(s.hi + w) = make_uint4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<uint4 *>(s.lo + w) = make_uint4(e[0], e[1], e[2], e[3]);
    } else {
      *reinterpret_cast<uint2 *>(s.hi + w) = make_uint2(h[0], h[1]);
      *reinterpret_cast<uint2 *>(s.lo + w) = make_uint2(e[0], e[1]);
    }
  }
}

// One warp's FP32 fragments of the upper block-triangle of G.
template <int D>
struct Warp {
  using P = StatsPlan<D>;
  float d[P::NTILE][4];
  int off_a, off_b;  // word offsets of the lane's chunk in rows s0 + t and s0 + t + 4

  __device__ __forceinline__ void init() {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int i = 0; i < P::NTILE; ++i)
#pragma unroll
      for (int r = 0; r < 4; ++r) d[i][r] = 0.0f;
    off_a = 4 * chunk_pos(g, t);
    off_b = 4 * chunk_pos(g, t + 4);
  }

  // This warp's 32 rows (64 sites) of the staged tile, 8 rows = 16 sites per MMA step (the
  // K dimension); the caller has made its lanes' staging visible (__syncwarp). Rows s0 + t
  // and s0 + t + 4 (s0 a multiple of 8) keep their chunk positions at every step, so the
  // steps only move the row base. A fragments: a0, a1 = columns m0 + g, m0 + g + 8 of the
  // site pair of row t (K indices 2t, 2t + 1); a2, a3 = the same columns of row t + 4
  // (K indices 2t + 8, 2t + 9), m0 = 0, 16.
  __device__ __forceinline__ void tile(const Smem<D> &s) {
    const int warp = threadIdx.x >> 5, t = threadIdx.x & 3;
    constexpr int LD = P::LD;
#pragma unroll 2
    for (int ks = 0; ks < 4; ++ks) {
      const int ra = (warp * 32 + ks * 8 + t) * LD + off_a, rb = (warp * 32 + ks * 8 + t + 4) * LD + off_b;
      uint32_t ah[P::MT][4], al[P::MT][4], bh[P::NT][2], bl[P::NT][2];
      if (P::MT == 2) {
        const uint4 ha = *reinterpret_cast<const uint4 *>(s.hi + ra), hb = *reinterpret_cast<const uint4 *>(s.hi + rb);
        const uint4 la = *reinterpret_cast<const uint4 *>(s.lo + ra), lb = *reinterpret_cast<const uint4 *>(s.lo + rb);
        ah[0][0] = ha.x; ah[0][1] = ha.y; ah[0][2] = hb.x; ah[0][3] = hb.y;
        ah[P::MT - 1][0] = ha.z; ah[P::MT - 1][1] = ha.w; ah[P::MT - 1][2] = hb.z; ah[P::MT - 1][3] = hb.w;
        al[0][0] = la.x; al[0][1] = la.y; al[0][2] = lb.x; al[0][3] = lb.y;
        al[P::MT - 1][0] = la.z; al[P::MT - 1][1] = la.w; al[P::MT - 1][2] = lb.z; al[P::MT - 1][3] = lb.w;
      } else {
        const uint2 ha = *reinterpret_cast<const uint2 *>(s.hi + ra), hb = *reinterpret_cast<const uint2 *>(s.hi + rb);
        const uint2 la = *reinterpret_cast<const uint2 *>(s.lo + ra), lb = *reinterpret_cast<const uint2 *>(s.lo + rb);
        ah[0][0] = ha.x; ah[0][1] = ha.y; ah[0][2] = hb.x; ah[0][3] = hb.y;
        al[0][0] = la.x; al[0][1] = la.y; al[0][2] = lb.x; al[0][3] = lb.y;
      }
      // G is symmetric (A = K^T, B = K): the B fragment of column tile nt is the pair
      // (a0, a2) or (a1, a3) of row tile nt / 2, already loaded.
#pragma unroll
      for (int nt = 0; nt < P::NT; ++nt) {
        const int mt = nt / 2, h = nt % 2;
        bh[nt][0] = ah[mt][h];
        bh[nt][1] = ah[mt][h + 2];
        bl[nt][0] = al[mt][h];
        bl[nt][1] = al[mt][h + 2];
      }
      // hi*hi, hi*lo, lo*hi, then lo*lo over all tiles: consecutive MMAs go to different
      // accumulators, so none waits for the one before it.
#pragma unroll
      for (int i = 0; i < P::NTILE; ++i) mma_bf16(d[i], ah[tile_mt<D>(i)], bh[tile_nt<D>(i)]);
#pragma unroll
      for (int i = 0; i < P::NTILE; ++i) mma_bf16(d[i], ah[tile_mt<D>(i)], bl[tile_nt<D>(i)]);
#pragma unroll
      for (int i = 0; i < P::NTILE; ++i) mma_bf16(d[i], al[tile_mt<D>(i)], bh[tile_nt<D>(i)]);
#pragma unroll
      for (int i = 0; i < P::NTILE; ++i) mma_bf16(d[i], al[tile_mt<D>(i)], bl[tile_nt<D>(i)]);
    }
  }

  // Adds the fragments to the block's FP64 sums and clears them.
  __device__ __forceinline__ void flush(const Smem<D> &s) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < P::NTILE; ++i)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        atomicAdd(&s.acc64[(i * 4 + r) * 32 + lane], (double)d[i][r]);
        d[i][r] = 0.0f;
      }
  }
};

// After the block's last flush and a barrier: sums the warps' fragments and adds the
// upper triangle of G (and the block's non-finite count) to the output record.
template <int D>
__device__ __forceinline__ void finish(const Smem<D> &s, unsigned nonfinite_block, double *__restrict__ acc) {
  using P = StatsPlan<D>;
  constexpr int NC = P::NC;
  for (int e = threadIdx.x; e < P::NTILE * 4 * 32; e += blockDim.x) {
    const int i = e / 128, r = (e / 32) % 4, ln = e % 32;
    const int row = tile_mt<D>(i) * 16 + (ln >> 2) + (r >= 2 ? 8 : 0);
    const int colx = tile_nt<D>(i) * 8 + 2 * (ln & 3) + (r & 1);
    if (row > colx) continue;
    atomicAdd(&acc[row * NC - row * (row - 1) / 2 + (colx - row)], s.acc64[e]);
  }
  if (threadIdx.x == 0 && nonfinite_block) atomicAdd(&acc[P::NREC], (double)nonfinite_block);
}

}  // namespace gram
}  // namespace flbm
