// Statistics reduction over one lattice state: the diagnostics of Sec. III (spatial
// means <u_a>, <u_a u_b> for the equipartition tests, Eq. for <u_a^2> = kBT/rho0) and
// the central-moment means and covariances whose equilibrium form is C^eq (Sec. II-B,
// "Structural properties"), plus mass and momentum for the conservation checks.
//
// Output record (doubles, read by the host in api.cu):
//   [0] number of finite sites         [1] sum (rho - rho0)   [2..4] sum j
//   [5..7] sum u                        [8..13] sum u_a u_b (xx, yy, zz, xy, xz, yz)
//   [14 .. 14+Q) sum k_v                then sum k_v k_w for v <= w (row-major upper)
//   [nacc] number of non-finite sites
//
// Every one of these sums is an entry of the Gram matrix G = sum_x c(x) c(x)^T of the
// per-site column vector
//   c = [1, rho - rho0, j_x, j_y, j_z, u_x, u_y, u_z, k_0 .. k_{Q-1}, 0 ...]
// (row 0 of G gives the linear sums). Persistent blocks of 128 threads walk tiles of 256
// sites; each thread computes two sites with the packed FP32x2 algebra of the step
// (cm.cuh) and writes their columns as (site a, site b) pairs to shared memory. The
// needed 4 x 4 blocks of G are then accumulated in registers, each packed FMA adding one
// entry for both sites of a pair; per-tile sums collect in shared memory in FP32, go to
// FP64 (also in shared memory) every 8 tiles and to the output with one FP64 atomic per
// entry and block. Sites with a non-finite value
// contribute a zero column and are counted.
#include <cuda_runtime.h>

#include "cm.cuh"
#include "internal.h"

namespace flbm {

int stats_nacc(int Q) { return 14 + Q + Q * (Q + 1) / 2; }

namespace {

constexpr int kTilePairs = kStatsBlock;  // 128 threads x 2 sites = 256 sites per tile
constexpr int kFlushTiles = 8;

template <int D>
struct GramPlan {
  static constexpr int Q = Lat<D>::Q;
  static constexpr int NCOL = 8 + Q;
  static constexpr int G = (NCOL + 3) / 4;  // column groups of 4
  static constexpr int NC = 4 * G;
  // Shared-memory row stride (float2): padded by 2 so that rows read at the same time by
  // the different site-pair ranges of a warp start on different banks.
  static constexpr int LDT = NC + 2;
  // Needed blocks (gi, gj), gi <= gj: (0, *) linear sums, (1, 1) u u, (k, k) covariances.
  static constexpr int NBLK = G + 1 + (G - 2) * (G - 1) / 2;
  static constexpr int PARTS = kStatsBlock / NBLK;  // site-pair ranges per block
};

template <int D>
__device__ __forceinline__ void block_of(int b, int &gi, int &gj) {
  constexpr int G = GramPlan<D>::G;
  if (b < G) {
    gi = 0;
    gj = b;
    return;
  }
  if (b == G) {
    gi = gj = 1;
    return;
  }
  int r = b - G - 1;
  gi = 2;
  while (r >= G - gi) {
    r -= G - gi;
    ++gi;
  }
  gj = gi + r;
}

// Record index of Gram entry (c1, c2), c1 <= c2, or -1 if the record does not keep it.
template <int D>
__device__ __forceinline__ int record_index(int c1, int c2) {
  constexpr int Q = Lat<D>::Q;
  if (c2 >= 8 + Q) return -1;
  if (c1 == 0) return c2 < 8 ? c2 : 14 + (c2 - 8);
  if (c1 >= 5 && c1 <= 7 && c2 >= 5 && c2 <= 7) {
    const int a = c1 - 5, b = c2 - 5;
    return a == b ? 8 + a : (a == 0 ? (b == 1 ? 11 : 12) : 13);
  }
  if (c1 >= 8) {
    const int v = c1 - 8, w = c2 - 8;
    return 14 + Q + v * Q - v * (v - 1) / 2 + (w - v);
  }
  return -1;
}

// Columns of the two sites of a pair (lane x: site s, lane y: site s + 1). PAIRROW: nx is
// even, so s (even) and s + 1 share a row and load as pairs (cm.cuh, load_logical2).
template <int D, typename S, int PARITY, bool PAIRROW>
__device__ __forceinline__ void pair_columns(const S *__restrict__ f, long long plane, int nx, int ny, int nz,
                                             float rho0, long long s, long long N, float2 *col,
                                             unsigned &nonfinite) {
  constexpr int Q = Lat<D>::Q;
  float2 F[3][3][3];
  bool valid[2] = {s < N, s + 1 < N};
  if (PAIRROW) {
    if (valid[0]) {
      const int x0 = (int)(s % nx), y = (int)((s / nx) % ny), z = (int)(s / ((long long)nx * ny));
      load_logical2<D, S, PARITY>(f, plane, addr2(x0, y, z, nx, ny, nz), F);
    } else {
#pragma unroll
      for (int a = 0; a < 27; ++a) (&F[0][0][0])[a] = make_float2(0.0f, 0.0f);
    }
  } else {
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const long long sl = s + l;
      float Fl[3][3][3];
      if (valid[l]) {
        const int x = (int)(sl % nx), y = (int)((sl / nx) % ny), z = (int)(sl / ((long long)nx * ny));
        load_logical<D, S, PARITY>(f, plane, neighbourhood(x, y, z, nx, ny, nz), Fl);
      } else {
#pragma unroll
        for (int a = 0; a < 27; ++a) (&Fl[0][0][0])[a] = 0.0f;
      }
#pragma unroll
      for (int a = 0; a < 27; ++a) set_lane((&F[0][0][0])[a], l, (&Fl[0][0][0])[a]);
    }
  }
  float2 drho, rho, ux, uy, uz;
  site_central_moments<D>(F, rho0, drho, rho, ux, uy, uz);
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
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    bool ok = valid[l] && isfinite(lane(rho, l)) && isfinite(lane(ux, l)) && isfinite(lane(uy, l)) &&
              isfinite(lane(uz, l));
#pragma unroll
    for (int v = 0; v < Q; ++v) ok = ok && isfinite(lane(k[v], l));
    if (valid[l] && !ok) ++nonfinite;
    // Zero the whole column of a skipped site (select, not multiply: it may hold NaN).
    set_lane(col[0], l, ok ? 1.0f : 0.0f);
    set_lane(col[1], l, ok ? lane(drho, l) : 0.0f);
    set_lane(col[2], l, ok ? lane(rho, l) * lane(ux, l) : 0.0f);
    set_lane(col[3], l, ok ? lane(rho, l) * lane(uy, l) : 0.0f);
    set_lane(col[4], l, ok ? lane(rho, l) * lane(uz, l) : 0.0f);
    set_lane(col[5], l, ok ? lane(ux, l) : 0.0f);
    set_lane(col[6], l, ok ? lane(uy, l) : 0.0f);
    set_lane(col[7], l, ok ? lane(uz, l) : 0.0f);
#pragma unroll
    for (int v = 0; v < Q; ++v) set_lane(col[8 + v], l, ok ? lane(k[v], l) : 0.0f);
  }
}

template <int D, typename S, int PARITY, bool PAIRROW>
__global__ void __launch_bounds__(kStatsBlock, 4) stats_kernel(const S *__restrict__ f, long long plane,
                                                               int nx, int ny, int nz, float rho0,
                                                               double *__restrict__ acc) {
  using P = GramPlan<D>;
  constexpr int NC = P::NC;
  constexpr int LDT = P::LDT;
  constexpr int NACC = 14 + P::Q + P::Q * (P::Q + 1) / 2;
  constexpr int NWORK = P::NBLK * P::PARTS;
  __shared__ __align__(16) float2 tile[kTilePairs * LDT];
  __shared__ float part32[16][NWORK];   // FP32 partial sums of the current tile group
  __shared__ double part64[16][NWORK];  // FP64 running sums
  __shared__ unsigned int nonfinite_block;

  const int work = threadIdx.x;
  const bool active = work < NWORK;
  if (threadIdx.x == 0) nonfinite_block = 0u;
  if (active) {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      part32[e][work] = 0.0f;
      part64[e][work] = 0.0;
    }
  }
  // This thread's Gram block and site-pair range in phase 2.
  int gi = 0, gj = 0;
  const int part = active ? work % P::PARTS : 0;
  if (active) block_of<D>(work / P::PARTS, gi, gj);
  const int p0 = part * kTilePairs / P::PARTS, p1 = (part + 1) * kTilePairs / P::PARTS;

  unsigned nonfinite = 0u;
  const long long N = plane;
  const long long tile_sites = 2LL * kTilePairs;
  int tiles_done = 0;
  for (long long base = (long long)blockIdx.x * tile_sites; base < N; base += (long long)gridDim.x * tile_sites) {
    // Phase 1: columns of this thread's two sites.
    {
      float2 col[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) col[c] = make_float2(0.0f, 0.0f);
      pair_columns<D, S, PARITY, PAIRROW>(f, plane, nx, ny, nz, rho0, base + 2 * threadIdx.x, N, col,
                                          nonfinite);
      float4 *dst = reinterpret_cast<float4 *>(tile + threadIdx.x * LDT);
#pragma unroll
      for (int c = 0; c < NC; c += 2) dst[c / 2] = make_float4(col[c].x, col[c].y, col[c + 1].x, col[c + 1].y);
    }
    __syncthreads();
    // Phase 2: the thread's 4 x 4 Gram block over its range of site pairs.
    if (active) {
      float2 g[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) g[i][j] = make_float2(0.0f, 0.0f);
#pragma unroll 4
      for (int p = p0; p < p1; ++p) {
        const float4 *row = reinterpret_cast<const float4 *>(tile + p * LDT);
        const float4 a01 = row[2 * gi], a23 = row[2 * gi + 1];
        const float4 b01 = row[2 * gj], b23 = row[2 * gj + 1];
        const float2 a[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w), make_float2(a23.x, a23.y),
                             make_float2(a23.z, a23.w)};
        const float2 b[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w), make_float2(b23.x, b23.y),
                             make_float2(b23.z, b23.w)};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) g[i][j] = __ffma2_rn(a[i], b[j], g[i][j]);
      }
      const bool flush = (tiles_done + 1 == kFlushTiles);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float t = part32[4 * i + j][work] + (g[i][j].x + g[i][j].y);
          if (flush) {
            part64[4 * i + j][work] += (double)t;
            part32[4 * i + j][work] = 0.0f;
          } else {
            part32[4 * i + j][work] = t;
          }
        }
    }
    if (++tiles_done == kFlushTiles) tiles_done = 0;
    __syncthreads();
  }
  if (active) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c1 = 4 * gi + i, c2 = 4 * gj + j;
        if (gi == gj && j < i) continue;  // lower half of a diagonal block
        const int e = record_index<D>(c1, c2);
        if (e >= 0) atomicAdd(&acc[e], part64[4 * i + j][work] + (double)part32[4 * i + j][work]);
      }
  }
  if (nonfinite) atomicAdd(&nonfinite_block, nonfinite);
  __syncthreads();
  if (threadIdx.x == 0 && nonfinite_block) atomicAdd(&acc[NACC], (double)nonfinite_block);
}

template <int D, typename S>
cudaError_t launch_typed(int parity, const void *f, long long plane, int nx, int ny, int nz,
                         float rho0, double *acc, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long tiles = (plane + 2LL * kTilePairs - 1) / (2LL * kTilePairs);
  const long long cap = (long long)(sms > 0 ? sms : 1) * 4;
  const int grid = (int)(tiles < cap ? tiles : cap);
  const S *p = static_cast<const S *>(f);
  const bool pairrow = nx % 2 == 0;
  if (parity == 0) {
    if (pairrow)
      stats_kernel<D, S, 0, true><<<grid, kStatsBlock, 0, s>>>(p, plane, nx, ny, nz, rho0, acc);
    else
      stats_kernel<D, S, 0, false><<<grid, kStatsBlock, 0, s>>>(p, plane, nx, ny, nz, rho0, acc);
  } else {
    if (pairrow)
      stats_kernel<D, S, 1, true><<<grid, kStatsBlock, 0, s>>>(p, plane, nx, ny, nz, rho0, acc);
    else
      stats_kernel<D, S, 1, false><<<grid, kStatsBlock, 0, s>>>(p, plane, nx, ny, nz, rho0, acc);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stats(int D, int storage, int parity, const void *f, long long plane, int nx,
                         int ny, int nz, float rho0, double *acc, cudaStream_t s) {
  if (D == 3) {
    if (storage == 0) return launch_typed<3, float>(parity, f, plane, nx, ny, nz, rho0, acc, s);
    if (storage == 1)
      return launch_typed<3, __nv_bfloat16>(parity, f, plane, nx, ny, nz, rho0, acc, s);
    return launch_typed<3, __half>(parity, f, plane, nx, ny, nz, rho0, acc, s);
  }
  if (storage == 0) return launch_typed<2, float>(parity, f, plane, nx, ny, nz, rho0, acc, s);
  if (storage == 1)
    return launch_typed<2, __nv_bfloat16>(parity, f, plane, nx, ny, nz, rho0, acc, s);
  return launch_typed<2, __half>(parity, f, plane, nx, ny, nz, rho0, acc, s);
}

}  // namespace flbm
