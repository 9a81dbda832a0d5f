// Statistics reduction over one lattice state: the diagnostics of Sec. III (spatial
// means <u_a>, <u_a u_b> for the equipartition tests, Eq. for <u_a^2> = kBT/rho0) and
// the central-moment means and covariances whose equilibrium form is C^eq (Sec. II-B,
// "Structural properties"), plus mass and momentum for the conservation checks.
//
// Every one of these sums is an entry of the Gram matrix G of the per-site columns
// (gram.cuh: layout, BF16 four-pass tensor-core accumulation, output record; k_0 = rho
// and the central moments k_1..k_D, which vanish identically, are rebuilt or set to zero
// by the host, api.cu). Persistent blocks of kStatsBlock threads walk tiles of
// 2 kStatsBlock sites: each thread computes the columns of two sites with the packed
// FP32x2 algebra of the step (cm.cuh) and stages them in its warp's rows (one row per
// pair, BF16 hi/lo words); each warp then accumulates the Gram fragments of its rows.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "cm.cuh"
#include "d3q19.cuh"
#include "gram.cuh"
#include "internal.h"

namespace flbm {

int stats_nacc(int Q) { return Q == 9 ? StatsPlan<2>::NREC : StatsPlan<3>::NREC; }

namespace {

using gram::kTileSites;

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
      load19_pairs<S, PARITY>(f, plane, addr2(x0, y, z, nx, ny, nz), F);
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

// Columns of the two sites of a pair (lane x: site s, lane y: site s + 1). PAIRROW: nx is
// even, so s (even) and s + 1 share a row and load as pairs; on odd parity the pair is the
// step's (cm.cuh, load_pairs: sites s + 1 and s + 2 of the row), which covers the same sites.
template <int D, typename S, int PARITY, bool PAIRROW, bool ISO>
__device__ __forceinline__ void pair_columns(const S *__restrict__ f, long long plane, int nx, int ny, int nz,
                                             float rho0, long long s, long long N,
                                             float2 (&col)[StatsPlan<D>::NC], unsigned &nonfinite) {
  float2 F[3][3][3];
  bool valid[2] = {s < N, s + 1 < N};
  if (PAIRROW) {
    if (valid[0]) {
      const uint32_t r = (uint32_t)s / (uint32_t)nx, q = r / (uint32_t)ny;
      const int x0 = (int)((uint32_t)s - r * (uint32_t)nx), y = (int)(r - q * (uint32_t)ny), z = (int)q;
      load_pairs<D, S, PARITY>(f, plane, addr2(x0, y, z, nx, ny, nz), F);
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
  gram::moment_columns<D, ISO>(F, drho, rho, ux, uy, uz, valid[0], valid[1], col, nonfinite);
}

template <int D, typename S, int PARITY, bool PAIRROW, bool ISO>
__global__ void __launch_bounds__(kStatsBlock, PAIRROW ? 4 : 3) stats_kernel(const S *__restrict__ f, long long plane,
                                                               int nx, int ny, int nz, float rho0,
                                                               double *__restrict__ acc, long long site0,
                                                               long long site1) {
  constexpr int NC = StatsPlan<D>::NC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const gram::Smem<D> sm = gram::smem_layout<D>(smem_raw);
  __shared__ unsigned int nonfinite_block;
  if (threadIdx.x == 0) nonfinite_block = 0u;
  gram::zero_acc64<D>(sm);
  __syncthreads();  // sums zeroed before any warp flushes (warps do not meet again in the loop)
  gram::Warp<D> gw;
  gw.init();

  unsigned nonfinite = 0u;
  const long long N = site1;  // sites [site0, site1) of the array (plane = its Q-stride)
  int tiles_done = 0;
  for (long long base = site0 + (long long)blockIdx.x * kTileSites; base < N;
       base += (long long)gridDim.x * kTileSites) {
    {
      float2 col[NC];
      if constexpr (D == 19) {
#pragma unroll
        for (int c = 0; c < NC; ++c) col[c] = make_float2(0.0f, 0.0f);
        pair_columns19<S, PARITY, PAIRROW>(f, plane, nx, ny, nz, rho0, base + 2 * threadIdx.x, N, col,
                                           nonfinite);
      } else {
        pair_columns<D, S, PARITY, PAIRROW, ISO>(f, plane, nx, ny, nz, rho0, base + 2 * threadIdx.x, N, col,
                                                 nonfinite);
      }
      // The thread's site pair in the warp's own rows; the rows are consumed (second
      // __syncwarp) before the next tile overwrites them.
      gram::stage_columns<D>(sm, col);
      __syncwarp();
      gw.tile(sm);
      __syncwarp();
    }
    if (++tiles_done == gram::kFlushTiles) {
      tiles_done = 0;
      gw.flush(sm);
    }
  }
  gw.flush(sm);
  if (nonfinite) atomicAdd(&nonfinite_block, nonfinite);
  __syncthreads();
  gram::finish<D>(sm, nonfinite_block, acc);
}

template <int D, typename S>
size_t stats_smem() {
  return gram::smem_bytes<D>();
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
                       cudaStream_t s, long long site0, long long nsites) {
  auto kernel = stats_kernel<D, S, PARITY, PAIRROW, ISO>;
  const size_t smem = stats_smem<D, S>();
  const long long tiles = (nsites + kTileSites - 1) / kTileSites;
  if (tiles == 0) return cudaSuccess;
  int grid = 0;
  const cudaError_t e = stats_grid(kernel, smem, tiles, &grid);
  if (e != cudaSuccess) return e;
  kernel<<<grid, kStatsBlock, smem, s>>>(p, plane, nx, ny, nz, rho0, acc, site0, site0 + nsites);
  return cudaGetLastError();
}

template <int D, typename S, bool ISO>
cudaError_t launch_typed(int parity, const void *f, long long plane, int nx, int ny, int nz,
                         float rho0, double *acc, cudaStream_t s, long long site0, long long nsites) {
  const S *p = static_cast<const S *>(f);
  // Pairs (s, s + 1) share a row when nx is even and every tile starts on an even site.
  const bool pairrow = nx % 2 == 0 && site0 % 2 == 0;
  if (parity == 0)
    return pairrow ? launch_one<D, S, 0, true, ISO>(p, plane, nx, ny, nz, rho0, acc, s, site0, nsites)
                   : launch_one<D, S, 0, false, ISO>(p, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
  return pairrow ? launch_one<D, S, 1, true, ISO>(p, plane, nx, ny, nz, rho0, acc, s, site0, nsites)
                 : launch_one<D, S, 1, false, ISO>(p, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
}

}  // namespace

cudaError_t launch_stats(int D, int storage, bool iso, int parity, const void *f, long long plane, int nx,
                         int ny, int nz, float rho0, double *acc, cudaStream_t s, long long site0,
                         long long nsites) {
  if (D == 19) {  // D3Q19 (lattice code 19)
    if (storage == 0) return launch_typed<19, float, false>(parity, f, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
    if (storage == 1)
      return launch_typed<19, __nv_bfloat16, false>(parity, f, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
    return launch_typed<19, __half, false>(parity, f, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
  }
  if (D == 3 && iso) {
    if (storage == 0) return launch_typed<3, float, true>(parity, f, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
    if (storage == 1)
      return launch_typed<3, __nv_bfloat16, true>(parity, f, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
    return launch_typed<3, __half, true>(parity, f, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
  }
  if (D == 3) {
    if (storage == 0) return launch_typed<3, float, false>(parity, f, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
    if (storage == 1)
      return launch_typed<3, __nv_bfloat16, false>(parity, f, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
    return launch_typed<3, __half, false>(parity, f, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
  }
  if (storage == 0) return launch_typed<2, float, false>(parity, f, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
  if (storage == 1)
    return launch_typed<2, __nv_bfloat16, false>(parity, f, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
  return launch_typed<2, __half, false>(parity, f, plane, nx, ny, nz, rho0, acc, s, site0, nsites);
}

}  // namespace flbm
