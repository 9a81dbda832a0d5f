// Statistics reduction over one lattice state: the diagnostics of Sec. III (spatial
// means <u_a>, <u_a u_b> for the equipartition tests, Eq. for <u_a^2> = kBT/rho0) and
// the central-moment means and covariances whose equilibrium form is C^eq (Sec. II-B,
// "Structural properties"), plus mass and momentum for the conservation checks.
//
// Every one of these sums is an entry of the Gram matrix G = sum_x c(x) c(x)^T of the
// per-site column vector (NC = 32 entries for D3Q27, 16 for D2Q9)
//   c = [1, rho - rho0, j_x, j_y, j_z, u_x, u_y, u_z, k_{D+1} .. k_{Q-1}, 0 ...]
// (row 0 of G gives the linear sums; k_0 = rho and the central moments k_1..k_D, which
// vanish identically, are rebuilt or set to zero by the host). The output record is the
// upper triangle of G in FP64, row-major, followed by the number of non-finite sites;
// api.cu maps it to flbm_stats_t.
//
// G is a dense contraction over the sites, so it runs on the tensor cores (warp-level
// mma.sync m16n8k8 with TF32 inputs and FP32 accumulation). Each input x is split into
// x_hi = tf32(x) and x_lo = tf32(x - x_hi) and every product is formed as
// hi*hi + hi*lo + lo*hi, which keeps about 2^-21 relative accuracy per product (the
// three-pass TF32 scheme). Persistent blocks of 128 threads walk tiles of 256 sites:
// each thread computes two sites with the packed FP32x2 algebra of the step (cm.cuh)
// and writes their split columns to shared memory (swizzled rows, conflict-free); each
// warp then accumulates the upper block-triangle of G over 64 sites of the tile in FP32
// fragments, adds them to the block's FP64 sums (shared memory) every 8 tiles and, at
// the end, the block adds its sums to the output with one FP64 atomic per entry. Sites with a non-finite value contribute a zero column and are
// counted.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "cm.cuh"
#include "d3q19.cuh"
#include "internal.h"

namespace flbm {

template <int D>
struct StatsPlan {
  static constexpr int Q = Lat<D>::Q;
  static constexpr int NC = D == 2 ? 16 : 32;  // columns, padded to whole MMA tiles
  static constexpr int LD = 32;                // shared-memory row: 32 words, swizzled (see swz)
  static constexpr int MT = NC / 16;           // 16-row tiles of G
  static constexpr int NT = NC / 8;            // 8-column tiles of G
  // Upper block-triangle: tiles (mt, nt) with nt >= 2 mt.
  static constexpr int NTILE = D == 2 ? 2 : 6;
  static constexpr int NREC = NC * (NC + 1) / 2;
};

int stats_nacc(int Q) { return Q == 9 ? StatsPlan<2>::NREC : StatsPlan<3>::NREC; }

namespace {

constexpr int kTileSites = 2 * kStatsBlock;  // 128 threads x 2 sites
constexpr int kFlushTiles = 8;

template <int D>
__host__ __device__ constexpr int tile_mt(int i) {
  return D != 2 ? (i < 4 ? 0 : 1) : 0;
}
template <int D>
__host__ __device__ constexpr int tile_nt(int i) {
  return D != 2 ? (i < 4 ? i : i - 2) : i;
}

// Shared-memory rows hold 32 words; column c of row r sits at word c ^ swz(r). With
// swz(r) = 8 (r mod 4) + 4 (bit 2 of r), the 16-byte stores of eight consecutive rows
// and the fragment loads of an MMA step (rows s0 + t or s0 + t + 4, columns m0 + g) hit
// 32 different banks.
__device__ __forceinline__ int swz(int r) { return ((r & 3) << 3) | (((r >> 2) & 1) << 2); }

// The D3Q19 columns of two sites s, s + 1 (lattice code 19): [1, rho - rho0, j, u,
// k_4 .. k_18, 0 ...] from the generated transforms of d3q19_gen.cuh.
template <typename S, int PARITY, bool PAIRROW>
__device__ __forceinline__ void pair_columns19(const S *__restrict__ f, long long plane, int nx, int ny, int nz,
                                               float rho0, long long s, long long N, float2 *col,
                                               unsigned &nonfinite) {
  float2 F[19];
  const bool valid[2] = {s < N, s + 1 < N};
  if (PAIRROW) {
    if (valid[0]) {
      const uint32_t r = (uint32_t)s / (uint32_t)nx, q = r / (uint32_t)ny;
      const int x0 = (int)((uint32_t)s - r * (uint32_t)nx), y = (int)(r - q * (uint32_t)ny), z = (int)q;
      load19_2<S, PARITY>(f, plane, addr2(x0, y, z, nx, ny, nz), F);
    } else {
#pragma unroll
      for (int a = 0; a < 19; ++a) F[a] = make_float2(0.0f, 0.0f);
    }
  } else {
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const long long sl = s + l;
      float Fl[19];
      if (valid[l]) {
        const uint32_t r = (uint32_t)sl / (uint32_t)nx, q = r / (uint32_t)ny;
        const int x = (int)((uint32_t)sl - r * (uint32_t)nx), y = (int)(r - q * (uint32_t)ny), z = (int)q;
        load19<S, PARITY>(f, plane, neighbourhood(x, y, z, nx, ny, nz), Fl);
      } else {
#pragma unroll
        for (int a = 0; a < 19; ++a) Fl[a] = 0.0f;
      }
#pragma unroll
      for (int a = 0; a < 19; ++a) set_lane(F[a], l, Fl[a]);
    }
  }
  float2 r[19], rho, ux, uy, uz;
  d3q19_macros(F, rho0, r, rho, ux, uy, uz);
  const float2 drho = r[0];
  d3q19_central(r, rho, ux, uy, uz);
  col[0] = make_float2(valid[0] ? 1.0f : 0.0f, valid[1] ? 1.0f : 0.0f);
  col[1] = drho;
  col[2] = vmul(rho, ux);
  col[3] = vmul(rho, uy);
  col[4] = vmul(rho, uz);
  col[5] = ux;
  col[6] = uy;
  col[7] = uz;
#pragma unroll
  for (int v = 4; v < 19; ++v) col[8 + v - 4] = r[v];
  float2 sum = col[1];
#pragma unroll
  for (int c = 2; c < 8 + 15; ++c) sum = vadd(sum, col[c]);
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    if (valid[l] && !isfinite(lane(sum, l))) {
      ++nonfinite;
#pragma unroll
      for (int c = 0; c < 8 + 15; ++c) set_lane(col[c], l, 0.0f);
    }
  }
}

// Round to TF32 (nearest, ties away): x_hi = tf32(x), x_lo = tf32(x - x_hi). Both are
// rounded to nearest, so the split carries no bias (truncating x_lo would shrink every
// product by about 2^-20 on average).
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// D (16x8, FP32) += A (16x8, TF32, row-major) * B (8x8, TF32, column-major).
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Columns of the two sites of a pair (lane x: site s, lane y: site s + 1). PAIRROW: nx is
// even, so s (even) and s + 1 share a row and load as pairs (cm.cuh, load_logical2).
template <int D, typename S, int PARITY, bool PAIRROW, bool ISO>
__device__ __forceinline__ void pair_columns(const S *__restrict__ f, long long plane, int nx, int ny, int nz,
                                             float rho0, long long s, long long N, float2 *col,
                                             unsigned &nonfinite) {
  constexpr int Q = Lat<D>::Q;
  float2 F[3][3][3];
  bool valid[2] = {s < N, s + 1 < N};
  if (PAIRROW) {
    if (valid[0]) {
      const uint32_t r = (uint32_t)s / (uint32_t)nx, q = r / (uint32_t)ny;
      const int x0 = (int)((uint32_t)s - r * (uint32_t)nx), y = (int)(r - q * (uint32_t)ny), z = (int)q;
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
        const uint32_t r = (uint32_t)sl / (uint32_t)nx, q = r / (uint32_t)ny;
        const int x = (int)((uint32_t)sl - r * (uint32_t)nx), y = (int)(r - q * (uint32_t)ny), z = (int)q;
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
  if (ISO) iso_rotate(k[4], k[5], k[6]);  // the isotropic variant's modes 4-6
  col[0] = make_float2(valid[0] ? 1.0f : 0.0f, valid[1] ? 1.0f : 0.0f);
  col[1] = drho;
  col[2] = vmul(rho, ux);
  col[3] = vmul(rho, uy);
  col[4] = vmul(rho, uz);
  col[5] = ux;
  col[6] = uy;
  col[7] = uz;
#pragma unroll
  for (int v = D + 1; v < Q; ++v) col[8 + v - D - 1] = k[v];
  // A site whose column holds a NaN or an infinity makes the sum of its entries non-
  // finite (the entries are far below overflow); such a site contributes a zero column
  // (select, not multiply: it may hold NaN) and is counted.
  float2 sum = col[1];
#pragma unroll
  for (int c = 2; c < 8 + Q - D - 1; ++c) sum = vadd(sum, col[c]);
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    if (valid[l] && !isfinite(lane(sum, l))) {
      ++nonfinite;
#pragma unroll
      for (int c = 0; c < 8 + Q - D - 1; ++c) set_lane(col[c], l, 0.0f);
    }
  }
}

template <int D, typename S, int PARITY, bool PAIRROW, bool ISO>
__global__ void __launch_bounds__(kStatsBlock, 3) stats_kernel(const S *__restrict__ f, long long plane,
                                                               int nx, int ny, int nz, float rho0,
                                                               double *__restrict__ acc) {
  using P = StatsPlan<D>;
  constexpr int NC = P::NC, LD = P::LD, NTILE = P::NTILE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint32_t *hi = reinterpret_cast<uint32_t *>(smem_raw);  // [row][LD] TF32 high parts
  uint32_t *lo = hi + kTileSites * LD;                      // [row][LD] TF32 low parts
  double *acc64 = reinterpret_cast<double *>(lo + kTileSites * LD);  // [NTILE*4][32], all warps
  __shared__ unsigned int nonfinite_block;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  if (threadIdx.x == 0) nonfinite_block = 0u;
  for (int e = threadIdx.x; e < NTILE * 4 * 32; e += blockDim.x) acc64[e] = 0.0;

  float d[NTILE][4];
#pragma unroll
  for (int i = 0; i < NTILE; ++i)
#pragma unroll
    for (int r = 0; r < 4; ++r) d[i][r] = 0.0f;

  // Word offsets of this lane's A-fragment entries within its two rows (see phase 2).
  int off[P::MT][4];
#pragma unroll
  for (int mt = 0; mt < P::MT; ++mt) {
    const int c = mt * 16 + g;
    off[mt][0] = c ^ swz(t);
    off[mt][1] = (c + 8) ^ swz(t);
    off[mt][2] = c ^ swz(t + 4);
    off[mt][3] = (c + 8) ^ swz(t + 4);
  }

  unsigned nonfinite = 0u;
  const long long N = plane;
  int tiles_done = 0;
  for (long long base = (long long)blockIdx.x * kTileSites; base < N; base += (long long)gridDim.x * kTileSites) {
    // Phase 1: split columns of this thread's two sites.
    {
      float2 col[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) col[c] = make_float2(0.0f, 0.0f);
      if constexpr (D == 19)
        pair_columns19<S, PARITY, PAIRROW>(f, plane, nx, ny, nz, rho0, base + 2 * threadIdx.x, N, col,
                                           nonfinite);
      else
        pair_columns<D, S, PARITY, PAIRROW, ISO>(f, plane, nx, ny, nz, rho0, base + 2 * threadIdx.x, N, col,
                                          nonfinite);
      // The two sites go to rows tid and tid + 128 (the sums do not depend on the order).
      const int r0 = threadIdx.x, r1 = threadIdx.x + kStatsBlock;
      uint32_t *h0 = hi + r0 * LD, *l0 = lo + r0 * LD, *h1 = hi + r1 * LD, *l1 = lo + r1 * LD;
      const int z0 = swz(r0), z1 = swz(r1);
#pragma unroll
      for (int c = 0; c < NC; c += 4) {
        uint4 ha, hb, la, lb;
        uint32_t *hav = &ha.x, *hbv = &hb.x, *lav = &la.x, *lbv = &lb.x;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t xa = to_tf32(col[c + q].x), xb = to_tf32(col[c + q].y);
          hav[q] = xa;
          hbv[q] = xb;
          lav[q] = to_tf32(col[c + q].x - __uint_as_float(xa));
          lbv[q] = to_tf32(col[c + q].y - __uint_as_float(xb));
        }
        *reinterpret_cast<uint4 *>(h0 + (c ^ z0)) = ha;
        *reinterpret_cast<uint4 *>(h1 + (c ^ z1)) = hb;
        *reinterpret_cast<uint4 *>(l0 + (c ^ z0)) = la;
        *reinterpret_cast<uint4 *>(l1 + (c ^ z1)) = lb;
      }
    }
    __syncthreads();
    // Phase 2: this warp's 64 sites, 8 per MMA step (the K dimension). Rows s0 + t and
    // s0 + t + 4 (s0 a multiple of 8) have swizzles 8 t and 8 t + 4 at every step, so a
    // lane's word offsets within the two rows are fixed (off[]), and the steps only move
    // the row base.
#pragma unroll 2
    for (int ks = 0; ks < 8; ++ks) {
      const int ra = (warp * 64 + ks * 8 + t) * LD, rb = ra + 4 * LD;
      uint32_t ah[P::MT][4], al[P::MT][4], bh[P::NT][2], bl[P::NT][2];
#pragma unroll
      for (int mt = 0; mt < P::MT; ++mt) {
        ah[mt][0] = hi[ra + off[mt][0]];
        ah[mt][1] = hi[ra + off[mt][1]];
        ah[mt][2] = hi[rb + off[mt][2]];
        ah[mt][3] = hi[rb + off[mt][3]];
        al[mt][0] = lo[ra + off[mt][0]];
        al[mt][1] = lo[ra + off[mt][1]];
        al[mt][2] = lo[rb + off[mt][2]];
        al[mt][3] = lo[rb + off[mt][3]];
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
#pragma unroll
      for (int i = 0; i < NTILE; ++i) {
        const int mt = tile_mt<D>(i), nt = tile_nt<D>(i);
        mma_tf32(d[i], ah[mt], bh[nt]);
        mma_tf32(d[i], ah[mt], bl[nt]);
        mma_tf32(d[i], al[mt], bh[nt]);
      }
    }
    if (++tiles_done == kFlushTiles) {
      tiles_done = 0;
#pragma unroll
      for (int i = 0; i < NTILE; ++i)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          atomicAdd(&acc64[(i * 4 + r) * 32 + lane], (double)d[i][r]);
          d[i][r] = 0.0f;
        }
    }
    __syncthreads();  // the tile's columns are consumed before the next tile overwrites them
  }
#pragma unroll
  for (int i = 0; i < NTILE; ++i)
#pragma unroll
    for (int r = 0; r < 4; ++r) atomicAdd(&acc64[(i * 4 + r) * 32 + lane], (double)d[i][r]);
  if (nonfinite) atomicAdd(&nonfinite_block, nonfinite);
  __syncthreads();
  // Sum the warps' fragments and add the upper triangle of G to the record.
  for (int e = threadIdx.x; e < NTILE * 4 * 32; e += blockDim.x) {
    const int i = e / 128, r = (e / 32) % 4, ln = e % 32;
    const int row = tile_mt<D>(i) * 16 + (ln >> 2) + (r >= 2 ? 8 : 0);
    const int colx = tile_nt<D>(i) * 8 + 2 * (ln & 3) + (r & 1);
    if (row > colx) continue;
    atomicAdd(&acc[row * NC - row * (row - 1) / 2 + (colx - row)], acc64[e]);
  }
  if (threadIdx.x == 0 && nonfinite_block) atomicAdd(&acc[P::NREC], (double)nonfinite_block);
}

template <int D, typename S>
size_t stats_smem() {
  using P = StatsPlan<D>;
  return 2 * sizeof(uint32_t) * kTileSites * P::LD + sizeof(double) * P::NTILE * 4 * 32;
}

// Resident blocks per SM for a kernel and its dynamic shared memory (cached; the
// attribute that allows more than 48 KB is set once per kernel).
template <typename K>
cudaError_t stats_grid(K kernel, size_t smem, long long tiles, int *grid) {
  static std::mutex mu;
  static std::map<const void *, int> cache;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find((const void *)kernel);
    if (it != cache.end()) {
      per_sm = it->second;
    } else {
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kStatsBlock, smem);
      if (e != cudaSuccess) return e;
      cache[(const void *)kernel] = per_sm;
    }
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long cap = (long long)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  *grid = (int)(tiles < cap ? tiles : cap);
  return cudaSuccess;
}

template <int D, typename S, int PARITY, bool PAIRROW, bool ISO>
cudaError_t launch_one(const S *p, long long plane, int nx, int ny, int nz, float rho0, double *acc,
                       cudaStream_t s) {
  auto kernel = stats_kernel<D, S, PARITY, PAIRROW, ISO>;
  const size_t smem = stats_smem<D, S>();
  const long long tiles = (plane + kTileSites - 1) / kTileSites;
  int grid = 0;
  const cudaError_t e = stats_grid(kernel, smem, tiles, &grid);
  if (e != cudaSuccess) return e;
  kernel<<<grid, kStatsBlock, smem, s>>>(p, plane, nx, ny, nz, rho0, acc);
  return cudaGetLastError();
}

template <int D, typename S, bool ISO>
cudaError_t launch_typed(int parity, const void *f, long long plane, int nx, int ny, int nz,
                         float rho0, double *acc, cudaStream_t s) {
  const S *p = static_cast<const S *>(f);
  const bool pairrow = nx % 2 == 0;
  if (parity == 0)
    return pairrow ? launch_one<D, S, 0, true, ISO>(p, plane, nx, ny, nz, rho0, acc, s)
                   : launch_one<D, S, 0, false, ISO>(p, plane, nx, ny, nz, rho0, acc, s);
  return pairrow ? launch_one<D, S, 1, true, ISO>(p, plane, nx, ny, nz, rho0, acc, s)
                 : launch_one<D, S, 1, false, ISO>(p, plane, nx, ny, nz, rho0, acc, s);
}

}  // namespace

cudaError_t launch_stats(int D, int storage, bool iso, int parity, const void *f, long long plane, int nx,
                         int ny, int nz, float rho0, double *acc, cudaStream_t s) {
  if (D == 19) {  // D3Q19 (lattice code 19)
    if (storage == 0) return launch_typed<19, float, false>(parity, f, plane, nx, ny, nz, rho0, acc, s);
    if (storage == 1)
      return launch_typed<19, __nv_bfloat16, false>(parity, f, plane, nx, ny, nz, rho0, acc, s);
    return launch_typed<19, __half, false>(parity, f, plane, nx, ny, nz, rho0, acc, s);
  }
  if (D == 3 && iso) {
    if (storage == 0) return launch_typed<3, float, true>(parity, f, plane, nx, ny, nz, rho0, acc, s);
    if (storage == 1)
      return launch_typed<3, __nv_bfloat16, true>(parity, f, plane, nx, ny, nz, rho0, acc, s);
    return launch_typed<3, __half, true>(parity, f, plane, nx, ny, nz, rho0, acc, s);
  }
  if (D == 3) {
    if (storage == 0) return launch_typed<3, float, false>(parity, f, plane, nx, ny, nz, rho0, acc, s);
    if (storage == 1)
      return launch_typed<3, __nv_bfloat16, false>(parity, f, plane, nx, ny, nz, rho0, acc, s);
    return launch_typed<3, __half, false>(parity, f, plane, nx, ny, nz, rho0, acc, s);
  }
  if (storage == 0) return launch_typed<2, float, false>(parity, f, plane, nx, ny, nz, rho0, acc, s);
  if (storage == 1)
    return launch_typed<2, __nv_bfloat16, false>(parity, f, plane, nx, ny, nz, rho0, acc, s);
  return launch_typed<2, __half, false>(parity, f, plane, nx, ny, nz, rho0, acc, s);
}

}  // namespace flbm
