// Pipelined fused step: the same update as step.cu (same per-site algebra, collide.cuh),
// with the population reads decoupled from the arithmetic.
//
// Persistent blocks walk the lattice rows (y, z) with a stride of gridDim.x; one row of
// nx sites is one tile and each thread owns two sites of it (x0 = 2 t, x0 + 1). For
// every tile the Q population rows it reads are fetched by the bulk-copy engine
// (cp.async.bulk, one contiguous row per population) into one of two shared-memory
// stages, two tiles ahead of the arithmetic, with completion counted on an mbarrier per
// stage. The threads read their populations from shared memory, release the stage (the
// next-but-one tile is fetched into it at once), collide in registers and store with
// ordinary writes. The noise loop is the rolled one (collide.cuh) to keep the persistent
// loop's code within the instruction cache.
//
// Streaming stays the in-place AA pattern (step.cu): on even steps a tile reads its own
// row; on odd steps population i of row (y, z) comes from slot opposite(i) of row
// (y - c_iy, z - c_iz), shifted by -c_ix in x, which the threads resolve with periodic
// indexing inside the staged row. Prefetching is race-free because the slots a row reads
// are exactly the slots that row's own collisions write, so no other tile touches them.
//
// Requirements (else the caller uses step.cu): nx even, nx <= 512, a population row a
// multiple of 16 bytes, and two stages of Q rows fitting in shared memory.
#include <cuda_runtime.h>

#include <map>
#include <tuple>
#include <mutex>
#include <utility>

#include "async.cuh"
#include "collide.cuh"
#include "internal.h"

namespace flbm {
namespace {

constexpr int kPipeMaxThreads = 256;

template <int D, typename S, int PARITY>
__device__ __forceinline__ void load_row_tile(const S *st, int nx, int x0, float2 (&F)[3][3][3]) {
  constexpr int z0 = (D == 3) ? -1 : 0, z1 = (D == 3) ? 1 : 0;
#pragma unroll
  for (int dz = z0; dz <= z1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = Lat<D>::index(dx, dy, dz);
        const S *row = st + i * nx;  // slot i: the row holding f_i of this tile
        float2 v;
        if (PARITY == 0 || dx == 0) {
          v = Storage2<S>::load(row + x0);
        } else if (dx == 1) {  // f_i(x) sits at x - 1 of the staged row
          v.x = Storage<S>::load(row + (x0 == 0 ? nx - 1 : x0 - 1));
          v.y = Storage<S>::load(row + x0);
        } else {  // f_i(x) sits at x + 1
          v.x = Storage<S>::load(row + x0 + 1);
          v.y = Storage<S>::load(row + (x0 + 2 == nx ? 0 : x0 + 2));
        }
        F[dz + 1][dy + 1][dx + 1] = v;
      }
}

// Warp 0: fetch the Q rows tile `r` reads into stage buffer `st`, counted on `bar`. Lane 0
// arrives with the expected byte count first; then the lanes issue the Q row copies.
template <int D, typename S, int PARITY>
__device__ __forceinline__ void fetch_tile(const S *f, long long plane, int nx, int ny, int nz, long long r,
                                           S *st, uint64_t *bar, int lane) {
  constexpr int Q = Lat<D>::Q;
  const uint32_t row_bytes = (uint32_t)(nx * sizeof(S));
  const int y = (int)(r % ny), z = (int)(r / ny);
  if (lane == 0) mbar_arrive_expect_tx(bar, Q * row_bytes);
  __syncwarp(__activemask());
  const int lanes = blockDim.x < 32 ? (int)blockDim.x : 32;  // small rows: fewer than 32 threads
  for (int i = lane; i < Q; i += lanes) {
    const S *src;
    if (PARITY == 0) {
      src = f + i * plane + ((long long)z * ny + y) * nx;
    } else {
      int yy = y - Lat<D>::cy(i), zz = z - Lat<D>::cz(i);
      yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
      zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
      src = f + opposite<D>(i) * plane + ((long long)zz * ny + yy) * nx;
    }
    bulk_copy_g2s(st + i * nx, src, row_bytes, bar);
  }
}

template <int D, typename S, int PARITY, bool NOISE, bool SHEAR>
__global__ void __launch_bounds__(kPipeMaxThreads, 2) step_pipe_kernel(const StepArgs a) {
  constexpr int Q = Lat<D>::Q;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const long long rows = (long long)ny * nz;
  S *stage0 = reinterpret_cast<S *>(smem_raw);
  S *stage1 = stage0 + Q * nx;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + 2 * Q * nx * sizeof(S));
  S *__restrict__ f = static_cast<S *>(a.f);
  const int tid = threadIdx.x;
  const int x0 = 2 * tid;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const long long r0 = blockIdx.x, stride = gridDim.x;
  const int lane = tid & 31;
  if (tid < 32) {
    if (r0 < rows) fetch_tile<D, S, PARITY>(f, a.plane, nx, ny, nz, r0, stage0, &bars[0], lane);
    if (r0 + stride < rows)
      fetch_tile<D, S, PARITY>(f, a.plane, nx, ny, nz, r0 + stride, stage1, &bars[1], lane);
  }
  int j = 0;
  for (long long r = r0; r < rows; r += stride, ++j) {
    const int s = j & 1;
    S *st = s ? stage1 : stage0;
    const bool got = mbar_wait_bounded(&bars[s], (uint32_t)((j >> 1) & 1));
    float2 F[3][3][3];
    if (got) load_row_tile<D, S, PARITY>(st, nx, x0, F);
    // One barrier per tile: every thread holds its populations (the stage is free again),
    // and all threads learn whether any wait gave up.
    if (__syncthreads_or(!got)) {
      // A copy did not complete in time: record it, let the copies still in flight land
      // (bounded), and leave this launch; the host reports FLBM_ETIMEOUT.
      if (tid == 0) {
        atomicExch(a.status, 1);
        mbar_wait_bounded(&bars[s], (uint32_t)((j >> 1) & 1));
        if (r + stride < rows) mbar_wait_bounded(&bars[s ^ 1], (uint32_t)(((j + 1) >> 1) & 1));
      }
      __syncthreads();
      return;
    }
    if (tid < 32 && r + 2 * stride < rows)
      fetch_tile<D, S, PARITY>(f, a.plane, nx, ny, nz, r + 2 * stride, st, &bars[s], lane);
    const int y = (int)(r % ny), z = (int)(r / ny);
    const Addr2 ad = addr2(x0, y, z, nx, ny, nz);
    collide_tile<D, NOISE, float2, true, SHEAR>(F, a.rho0, a.om_t, a.phc_t, (uint32_t)ad.s0, a.step_lo,
                                                a.step_hi, a.ks0, a.ks1);
    store_streamed2<D, S, PARITY>(f, a.plane, ad, F);
  }
}

constexpr size_t kPipeMaxSmem = 200 * 1024;  // largest stage pair pipe_applicable admits

// Persistent grid: resident blocks per SM (for this kernel and shared-memory size) times
// the SM count, at most one block per row. Runtime errors are returned, never left
// pending for a later launch to pick up.
template <typename K>
cudaError_t grid_for(K kernel, int threads, size_t smem, long long rows, int *grid) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void *, size_t>, int> cache;  // blocks per SM, per device
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return cudaGetLastError();
  const auto key = std::make_tuple(cur, (const void *)kernel, smem);
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      per_sm = it->second;
    } else {
      cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPipeMaxSmem);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
      if (e != cudaSuccess) return e;
      cache[key] = per_sm;
    }
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long g = (long long)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  *grid = (int)(g < rows ? g : rows);
  return cudaSuccess;
}

template <int D, typename S, int PARITY, bool NOISE, bool SHEAR>
cudaError_t launch_pipe_typed(const StepArgs &a, cudaStream_t s) {
  constexpr int Q = Lat<D>::Q;
  const int threads = a.nx / 2;
  const size_t smem = 2 * (size_t)Q * a.nx * sizeof(S) + 2 * sizeof(uint64_t);
  auto kernel = step_pipe_kernel<D, S, PARITY, NOISE, SHEAR>;
  int grid = 0;
  const cudaError_t e = grid_for(kernel, threads, smem, (long long)a.ny * a.nz, &grid);
  if (e != cudaSuccess) return e;
  kernel<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int D, typename S, bool SHEAR>
cudaError_t launch_pipe_dispatch(int parity, bool noise, const StepArgs &a, cudaStream_t s) {
  if (parity == 0)
    return noise ? launch_pipe_typed<D, S, 0, true, SHEAR>(a, s) : launch_pipe_typed<D, S, 0, false, SHEAR>(a, s);
  return noise ? launch_pipe_typed<D, S, 1, true, SHEAR>(a, s) : launch_pipe_typed<D, S, 1, false, SHEAR>(a, s);
}

template <int D, typename S>
cudaError_t launch_pipe_shear(bool shear, int parity, bool noise, const StepArgs &a, cudaStream_t s) {
  return shear ? launch_pipe_dispatch<D, S, true>(parity, noise, a, s)
               : launch_pipe_dispatch<D, S, false>(parity, noise, a, s);
}

}  // namespace

bool pipe_applicable(int D, int storage, int nx) {
  const int Q = D == 3 ? 27 : 9;
  const size_t es = storage_bytes(storage);
  if (nx % 2 != 0 || nx / 2 > kPipeMaxThreads || nx < 2) return false;
  if ((nx * es) % 16 != 0) return false;
  return 2 * (size_t)Q * nx * es + 16 <= kPipeMaxSmem;
}

cudaError_t launch_step_pipelined(int D, int storage, int parity, bool noise, bool shear,
                                  const StepArgs &a, cudaStream_t s) {
  if (D == 3) {
    if (storage == 0) return launch_pipe_shear<3, float>(shear, parity, noise, a, s);
    if (storage == 1) return launch_pipe_shear<3, __nv_bfloat16>(shear, parity, noise, a, s);
    return launch_pipe_shear<3, __half>(shear, parity, noise, a, s);
  }
  if (storage == 0) return launch_pipe_shear<2, float>(shear, parity, noise, a, s);
  if (storage == 1) return launch_pipe_shear<2, __nv_bfloat16>(shear, parity, noise, a, s);
  return launch_pipe_shear<2, __half>(shear, parity, noise, a, s);
}

}  // namespace flbm
