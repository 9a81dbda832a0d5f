// Statistics reduction over one lattice state: the diagnostics of Sec. III (spatial
// means <u_a>, <u_a u_b> for the equipartition tests, Eq. for <u_a^2> = kBT/rho0) and
// the central-moment means and covariances whose equilibrium form is C^eq (Sec. II-B,
// "Structural properties"), plus mass and momentum for the conservation checks.
//
// Every one of these sums is an entry of the Gram matrix G of the per-site columns
// (gram.cuh: staging layout, BF16 hi/lo products on the tcgen05 tensor cores with a TMEM
// accumulator, output record; k_0 = rho and the central moments k_1..k_D, which vanish
// identically, are rebuilt or set to zero by the host, api.cu). Persistent blocks of
// kStatsBlock threads walk tiles of 2 kStatsBlock sites: each thread computes the columns
// of two sites with the packed FP32x2 algebra of the step (cm.cuh) and writes their BF16
// hi/lo words into its warp's operand rows; one thread per block multiplies the tile.
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

// The populations of a thread's site pair, as loaded for one tile and consumed by the
// next: F19 for D3Q19 (lattice code 19), the 3x3x3 tile otherwise.
template <int D>
struct PairPops {
  float2 F[3][3][3];
};
template <>
struct PairPops<19> {
  float2 F[19];
};

// Loads the pair's populations (lane x: site s, lane y: site s + 1; zeros for a site
// beyond N). PAIRROW: nx is even, so s (even) and s + 1 share a row and load as pairs; on
// odd parity the pair is the step's (cm.cuh, load_pairs: sites s + 1 and s + 2 of the
// row), which covers the same sites.
template <int D, typename S, int PARITY, bool PAIRROW>
__device__ __forceinline__ void load_pair(const S *__restrict__ f, long long plane, int nx, int ny, int nz,
                                          long long s, long long N, PairPops<D> &P) {
  constexpr int NP = D == 19 ? 19 : 27;
  float2 *F = reinterpret_cast<float2 *>(&P.F);
  if (PAIRROW) {
    if (s < N) {
      const uint32_t r = (uint32_t)s / (uint32_t)nx, q = r / (uint32_t)ny;
      const int x0 = (int)((uint32_t)s - r * (uint32_t)nx), y = (int)(r - q * (uint32_t)ny), z = (int)q;
      if constexpr (D == 19)
        load19_pairs<S, PARITY>(f, plane, addr2(x0, y, z, nx, ny, nz), P.F);
      else
        load_pairs<D, S, PARITY>(f, plane, addr2(x0, y, z, nx, ny, nz), P.F);
    } else {
#pragma unroll
      for (int a = 0; a < NP; ++a) F[a] = make_float2(0.0f, 0.0f);
    }
  } else {
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const long long sl = s + l;
      float Fl[NP];
      if (sl < N) {
        const uint32_t r = (uint32_t)sl / (uint32_t)nx, q = r / (uint32_t)ny;
        const int x = (int)((uint32_t)sl - r * (uint32_t)nx), y = (int)(r - q * (uint32_t)ny), z = (int)q;
        if constexpr (D == 19)
          load19<S, PARITY>(f, plane, neighbourhood(x, y, z, nx, ny, nz), Fl);
        else
          load_logical<D, S, PARITY>(f, plane, neighbourhood(x, y, z, nx, ny, nz),
                                     *reinterpret_cast<float(*)[3][3][3]>(Fl));
      } else {
#pragma unroll
        for (int a = 0; a < NP; ++a) Fl[a] = 0.0f;
      }
#pragma unroll
      for (int a = 0; a < NP; ++a) set_lane(F[a], l, Fl[a]);
    }
  }
}

// The columns of the pair from its populations. D3Q19: [1, rho - rho0, j, u, k_4 .. k_18,
// 0 ...] from the generated transforms of d3q19_gen.cuh; D2Q9 / D3Q27: gram::moment_columns.
template <int D, bool ISO>
__device__ __forceinline__ void pair_columns(PairPops<D> &P, float rho0, bool v0, bool v1,
                                             float2 (&col)[StatsPlan<D>::NC], unsigned &nonfinite) {
  if constexpr (D == 19) {
    float2 r[19], rho, ux, uy, uz;
    d3q19_macros(P.F, rho0, r, rho, ux, uy, uz);
    const float2 drho = r[0];
    d3q19_central(r, rho, ux, uy, uz);
    col[0] = make_float2(v0 ? 1.0f : 0.0f, v1 ? 1.0f : 0.0f);
    col[1] = drho;
    col[2] = vmul(rho, ux);
    col[3] = vmul(rho, uy);
    col[4] = vmul(rho, uz);
    col[5] = ux;
    col[6] = uy;
    col[7] = uz;
#pragma unroll
    for (int v = 4; v < 19; ++v) col[8 + v - 4] = r[v];
#pragma unroll
    for (int c = 8 + 15; c < StatsPlan<D>::NC; ++c) col[c] = make_float2(0.0f, 0.0f);
    float2 sum = col[1];
#pragma unroll
    for (int c = 2; c < 8 + 15; ++c) sum = vadd(sum, col[c]);
    const bool valid[2] = {v0, v1};
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      if (valid[l] && !isfinite(lane(sum, l))) {
        ++nonfinite;
#pragma unroll
        for (int c = 0; c < 8 + 15; ++c) set_lane(col[c], l, 0.0f);
      }
    }
  } else {
    float2 drho, rho, ux, uy, uz;
    site_central_moments<D>(P.F, rho0, drho, rho, ux, uy, uz);
    gram::moment_columns<D, ISO>(P.F, drho, rho, ux, uy, uz, v0, v1, col, nonfinite);
  }
}

// One block walks tiles of kTileSites sites: every thread transforms its site pair
// (loaded during the previous tile) and stages the split columns; each warp then arrives
// once on the pipeline's "staged" mbarrier and thread 0 multiplies the tile (gram.cuh,
// Pipeline). Before a thread overwrites the staging rows it waits for the MMAs that read
// them (one phase of each mbarrier per tile; every wait bounded), so the loads and
// arithmetic of the next tile proceed while the tensor cores work.
template <int D, typename S, int PARITY, bool PAIRROW, bool ISO>
__global__ void __launch_bounds__(kStatsBlock, gram::blocks_per_sm<D>()) stats_kernel(const S *__restrict__ f, long long plane,
                                                               int nx, int ny, int nz, float rho0,
                                                               double *__restrict__ out, long long site0,
                                                               long long site1) {
  constexpr int NC = StatsPlan<D>::NC;
  extern __shared__ unsigned char smem_raw[];
  __shared__ unsigned int flags[2];  // non-finite count of the block, failure flag
  gram::Pipeline<D> pl;
  pl.init(smem_raw, flags);

  unsigned nonfinite = 0u;
  const long long N = site1;  // sites [site0, site1) of the array (plane = its Q-stride)
  const long long stride = (long long)gridDim.x * kTileSites;
  // Software pipelining: the populations of the thread's pair in the next tile are loaded
  // as soon as the current ones are consumed, so the loads are in flight while the thread
  // splits and stages its columns and waits for the tensor cores.
  PairPops<D> pp;
  if (site0 + (long long)blockIdx.x * kTileSites < N)
    load_pair<D, S, PARITY, PAIRROW>(f, plane, nx, ny, nz, site0 + (long long)blockIdx.x * kTileSites + 2 * threadIdx.x,
                                     N, pp);
  for (long long base = site0 + (long long)blockIdx.x * kTileSites; base < N; base += stride) {
    const long long s = base + 2 * threadIdx.x;
    float2 col[NC];
    pair_columns<D, ISO>(pp, rho0, s < N, s + 1 < N, col, nonfinite);
    if (base + stride < N) load_pair<D, S, PARITY, PAIRROW>(f, plane, nx, ny, nz, s + stride, N, pp);
    pl.tile(col);
  }
  pl.end(nonfinite, flags, out);
}

template <int D, typename S>
size_t stats_smem() {
  return gram::Plan<D>::SMEM;
}

// Persistent grid: `per_sm` blocks per SM, the residency the kernel is built for (its
// launch bounds, 52 KB of shared memory and 128 of the SM's 512 TMEM columns per block),
// at most one block per tile. The attribute that allows more than 48 KB of dynamic shared
// memory is set once per kernel and device.
template <typename K>
cudaError_t stats_grid(K kernel, size_t smem, long long tiles, int per_sm, int *grid) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, bool> ready;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(mu);
    bool &done = ready[std::make_pair(dev, (const void *)kernel)];
    if (!done) {
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      done = true;
    }
  }
  const long long cap = (long long)(sms > 0 ? sms : 1) * per_sm;
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
  const cudaError_t e = stats_grid(kernel, smem, tiles, gram::blocks_per_sm<D>(), &grid);
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
