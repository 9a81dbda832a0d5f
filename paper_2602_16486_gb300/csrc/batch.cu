// Batched ensembles: many independent periodic lattices (mixed D2Q9 / D3Q27, own size,
// rates, kBT and noise seed) advanced by one persistent kernel.
//
// The host lays every lattice's populations out in one allocation and cuts all lattices
// into tiles of equal site count (two sites per thread; a tile may span rows, never
// lattices). One cooperative launch runs n steps: block b takes the work items
// (step s, tile b + j G) in step-major order, and applies to each the same fused update
// as the single-lattice kernels (collide.cuh: rolled noise loop, packed FP32x2, the AA
// pattern of step.cu) with that lattice's parameters.
//
// There is no grid-wide barrier between steps. Lattices are independent, so a tile of
// lattice L at step s only has to wait until every tile of L has finished step s - 1
// (in-place AA streaming reads and writes neighbour slots across tile boundaries). Each
// lattice has a completion counter; a block announces a finished tile with a release
// (fence, then atomic add) and checks the counter of the next tile's lattice with an
// acquire before starting it. Blocks run ahead into the next step on lattices that are
// done, so the per-step tail of the slowest block no longer idles the machine. Progress
// is guaranteed: all blocks are resident (cooperative launch), each walks its items in
// order, and the lowest pending item only depends on items of the step before it, which
// are all complete.
//
// The per-lattice parameters travel by value in the kernel arguments (constant bank; at
// most kBatchMaxLattices lattices). A tile's lattice is found by a binary search over
// the lattices' first-tile indices in that table, from the block's own counters only,
// so the lattice's parameters stay block-uniform values (uniform registers) instead of
// occupying every thread's registers. All lattices share the step counter in device memory: read at entry and
// advanced by the last block to leave, so that one captured graph of the launch serves
// every call with the same n.
//
// Every wait is bounded: a block that polls longer than wait_polls times (or sees another
// block's failure) sets the status word and leaves; the host reports FLBM_ETIMEOUT.
#include <cuda_runtime.h>

#include "collide.cuh"
#include "internal.h"

namespace flbm {
namespace {


// The collision with lattice L's parameters: its three shear-structure numbers (SHEAR:
// per-mode factors are compile-time constants) or its per-mode arrays; round keys are
// formed from its key.
template <int D, bool SHEAR, bool ROLLED>
__device__ __forceinline__ void collide_lattice(float2 (&F)[3][3][3], const BatchLattice &L, const float *rates,
                                                uint32_t s0, uint32_t dsite, uint32_t step_lo, uint32_t step_hi) {
  const KeyBase keys{L.key0, L.key1};
  if (SHEAR)
    collide_rates<D, true, float2, ROLLED, true>(F, L.rho0, ShearRates<D>{L.sqrt_kbt, L.om_shear, L.phc_shear},
                                                 s0, step_lo, step_hi, keys, dsite);
  else
    collide_rates<D, true, float2, ROLLED, false>(F, L.rho0, ArrayRates{rates, rates + 27}, s0, step_lo, step_hi,
                                                  keys, dsite);
}

// Coordinates of site s of lattice L (32-bit arithmetic: every site index is < 2^32).
__device__ __forceinline__ void site_xyz(const BatchLattice &L, uint32_t s, int &x, int &y, int &z) {
  const uint32_t r = s / (uint32_t)L.nx;
  x = (int)(s - r * (uint32_t)L.nx);
  const uint32_t q = r / (uint32_t)L.ny;
  y = (int)(r - q * (uint32_t)L.ny);
  z = (int)q;
}

// Two sites of lattice L per thread, in tile [first, end). PAIR (nx even): sites
// first + 2 t and first + 2 t + 1 share a row and move as pairs (8-byte accesses).
// Otherwise (nx odd) lane l takes site first + t + l * blockDim.x, so that every access
// of a warp is a contiguous run. Either way the neighbour addresses are recomputed at
// the store rather than kept live across the collision (register pressure).
template <int D, int PARITY, bool SHEAR, bool PAIR, bool ROLLED = true>
__device__ __forceinline__ void batch_sites(const BatchLattice &L, const float *rates, uint32_t first, uint32_t end,
                                            uint32_t step_lo, uint32_t step_hi) {
  float *__restrict__ f = static_cast<float *>(L.f);
  const long long plane = L.plane;
  float2 F[3][3][3];
  if (PAIR) {
    const uint32_t s0 = first + 2u * threadIdx.x;
    if (s0 >= end) return;
    {
      int x0, y, z;
      site_xyz(L, s0, x0, y, z);
      load_logical2<D, float, PARITY>(f, plane, addr2(x0, y, z, L.nx, L.ny, L.nz), F);
    }
    collide_lattice<D, SHEAR, ROLLED>(F, L, rates, s0, 1u, step_lo, step_hi);
    // The neighbour addresses (18 registers) are rebuilt from the site index for the
    // store instead of being kept across the collision; the empty asm hides s0's
    // provenance so that the compiler cannot merge the two computations.
    uint32_t s1 = s0;
    asm volatile("" : "+r"(s1));
    int x0, y, z;
    site_xyz(L, s1, x0, y, z);
    store_streamed2<D, float, PARITY>(f, plane, addr2(x0, y, z, L.nx, L.ny, L.nz), F);
  } else {
    const uint32_t T = blockDim.x;
    const uint32_t s0 = first + threadIdx.x;
    if (s0 >= end) return;
    const bool second = s0 + T < end;
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const uint32_t s = (l == 1 && second) ? s0 + T : s0;  // an absent second lane repeats the first
      int x, y, z;
      site_xyz(L, s, x, y, z);
      float Fl[3][3][3];
      load_logical<D, float, PARITY>(f, plane, neighbourhood(x, y, z, L.nx, L.ny, L.nz), Fl);
#pragma unroll
      for (int a = 0; a < 27; ++a) set_lane((&F[0][0][0])[a], l, (&Fl[0][0][0])[a]);
    }
    collide_lattice<D, SHEAR, ROLLED>(F, L, rates, s0, T, step_lo, step_hi);
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      if (l == 1 && !second) break;
      int x, y, z;
      site_xyz(L, s0 + (uint32_t)l * T, x, y, z);
      float Fl[3][3][3];
#pragma unroll
      for (int a = 0; a < 27; ++a) (&Fl[0][0][0])[a] = lane((&F[0][0][0])[a], l);
      store_streamed<D, float, PARITY>(f, plane, neighbourhood(x, y, z, L.nx, L.ny, L.nz), Fl);
    }
  }
}

template <int PARITY, bool SHEAR>
__device__ __forceinline__ void batch_tile(const BatchLattice &L, const float *rates, uint32_t first, uint32_t end,
                                           uint32_t step_lo, uint32_t step_hi) {
  if (L.D == 3) {
    if (L.nx % 2 == 0)
      batch_sites<3, PARITY, SHEAR, true>(L, rates, first, end, step_lo, step_hi);
    else
      batch_sites<3, PARITY, SHEAR, false>(L, rates, first, end, step_lo, step_hi);
  } else {
    if (L.nx % 2 == 0)
      batch_sites<2, PARITY, SHEAR, true>(L, rates, first, end, step_lo, step_hi);
    else
      batch_sites<2, PARITY, SHEAR, false>(L, rates, first, end, step_lo, step_hi);
  }
}

// Thread 0: waits until lattice `lat` has finished `target` tiles in this launch.
__device__ __forceinline__ bool wait_done(const int *done, int target, int *status, uint32_t polls) {
  const volatile int *d = done;
  for (uint32_t it = 0; it < polls; ++it) {
    if (*d >= target) return true;
    if (*(volatile int *)status != 0) return false;
    __nanosleep(32);
  }
  atomicCAS(status, 0, 2);
  return false;
}

// Lattice of tile t among table entries [lo, hi): the last whose first tile is <= t
// (binary search over the kernel-argument table). Everything here derives from kernel
// arguments and the block's own counters, so the lattice's parameters stay block-uniform
// values rather than occupying every thread's registers.
__device__ __forceinline__ int lattice_of(const BatchArgs &a, int t, int lo, int hi) {
  --hi;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.lats[mid].tile0 <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int tiles_of(const BatchArgs &a, int lat) {
  return (lat + 1 < a.nlat ? a.lats[lat + 1].tile0 : a.ntiles) - a.lats[lat].tile0;
}

template <bool SHEAR>
__global__ void __launch_bounds__(kBatchMaxThreads, 2) batch_kernel(const BatchArgs a) {
  __shared__ int s_ok;
  const long long step0 = *a.step_counter;
  int s = 0, t = blockIdx.x;
  while (s < a.nsteps && t < a.ntiles) {
    const int lat = lattice_of(a, t, 0, a.nlat);
    const BatchLattice &L = a.lats[lat];
    if (threadIdx.x == 0) {
      int ok = 1;
      if (s > 0) ok = wait_done(&a.done[lat], s * tiles_of(a, lat) + a.target_bias, a.status, a.wait_polls);
      __threadfence();  // acquire: the lattice's step s - 1 writes are visible
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    const uint32_t first = (uint32_t)(t - L.tile0) * (uint32_t)a.span;
    const uint32_t end = first + (uint32_t)a.span < L.plane ? first + (uint32_t)a.span : L.plane;
    const unsigned long long step = (unsigned long long)(step0 + s);
    const uint32_t lo = (uint32_t)step, hi = (uint32_t)(step >> 32);
    if (step & 1)
      batch_tile<1, SHEAR>(L, a.rates + 54 * lat, first, end, lo, hi);
    else
      batch_tile<0, SHEAR>(L, a.rates + 54 * lat, first, end, lo, hi);
    __syncthreads();  // every thread's writes of this tile are issued
    if (threadIdx.x == 0) {
      __threadfence();  // release
      atomicAdd(&a.done[lat], 1);
    }
    t += gridDim.x;
    if (t >= a.ntiles) {
      t = blockIdx.x;
      ++s;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.exits, 1u) == gridDim.x - 1 && *(volatile int *)a.status == 0)
      *a.step_counter = step0 + a.nsteps;
  }
}

// One step of the lattices of one type D, table entries [lat_lo, lat_hi), whose tiles
// are tile_base, tile_base + 1, ...: block b takes tile tile_base + b (a plain launch;
// the hardware block scheduler balances the load). One kernel per lattice type keeps
// the D2Q9 blocks at the register count (and occupancy) of D2Q9 alone. The step number
// is read from the device counter plus `k`, so that a captured graph of n such launches
// serves every call with the same n and the same starting parity; PARITY is fixed per
// launch.
template <int D, bool SHEAR, int PARITY, bool ROLLED, int MINB>
__global__ void __launch_bounds__(MINB >= 5 ? 128 : kBatchMaxThreads, MINB)
    batch_step_kernel(const BatchArgs a, int k, int lat_lo, int lat_hi, int tile_base) {
  const int t = tile_base + (int)blockIdx.x;
  const int lat = lattice_of(a, t, lat_lo, lat_hi);
  const BatchLattice &L = a.lats[lat];
  const uint32_t first = (uint32_t)(t - L.tile0) * (uint32_t)a.span;
  const uint32_t end = first + (uint32_t)a.span < L.plane ? first + (uint32_t)a.span : L.plane;
  const unsigned long long step = (unsigned long long)(*a.step_counter + k);
  const float *rates = a.rates + 54 * lat;
  if (L.nx % 2 == 0)
    batch_sites<D, PARITY, SHEAR, true, ROLLED>(L, rates, first, end, (uint32_t)step, (uint32_t)(step >> 32));
  else
    batch_sites<D, PARITY, SHEAR, false, ROLLED>(L, rates, first, end, (uint32_t)step, (uint32_t)(step >> 32));
}

// Advances the shared step counter after the n step launches of one call.
__global__ void batch_advance_kernel(long long *step_counter, int n) { *step_counter += n; }

}  // namespace

cudaError_t batch_max_blocks(bool shear, int threads, int *blocks_per_sm) {
  return shear ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel<true>, threads, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel<false>, threads, 0);
}

// Launch shapes of the per-step form (BatchForm): register cap 128 (up to 256 threads,
// two blocks per SM) or 102 (up to 128 threads, five blocks per SM), D3Q27 noise loop
// unrolled or rolled (D2Q9 has no loop).
template <int D, bool SHEAR, int PARITY>
cudaError_t launch_group(int form, const BatchArgs &a, int k, const BatchGroup &g, int threads, cudaStream_t s) {
  if (g.ntiles <= 0) return cudaSuccess;
  if (form == kBatchStepOcc)
    batch_step_kernel<D, SHEAR, PARITY, false, 5><<<g.ntiles, threads, 0, s>>>(a, k, g.lat_lo, g.lat_hi, g.tile0);
  else if (form == kBatchStepRolled)  // D2Q9 has no noise loop: the same kernel as form 0
    batch_step_kernel<D, SHEAR, PARITY, D == 3, 2><<<g.ntiles, threads, 0, s>>>(a, k, g.lat_lo, g.lat_hi, g.tile0);
  else
    batch_step_kernel<D, SHEAR, PARITY, false, 2><<<g.ntiles, threads, 0, s>>>(a, k, g.lat_lo, g.lat_hi, g.tile0);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_group_any(int form, bool shear, int parity, const BatchArgs &a, int k, const BatchGroup &g,
                             int threads, cudaStream_t s) {
  if (shear)
    return parity ? launch_group<D, true, 1>(form, a, k, g, threads, s)
                  : launch_group<D, true, 0>(form, a, k, g, threads, s);
  return parity ? launch_group<D, false, 1>(form, a, k, g, threads, s)
                : launch_group<D, false, 0>(form, a, k, g, threads, s);
}

cudaError_t launch_batch_steps(int form, bool shear, int parity0, const BatchArgs &a, const BatchGroup &g3,
                               const BatchGroup &g2, int n, int threads, cudaStream_t s) {
  for (int k = 0; k < n; ++k) {
    const int parity = (parity0 + k) & 1;
    cudaError_t e = launch_group_any<3>(form, shear, parity, a, k, g3, threads, s);
    if (e == cudaSuccess) e = launch_group_any<2>(form, shear, parity, a, k, g2, threads, s);
    if (e != cudaSuccess) return e;
  }
  batch_advance_kernel<<<1, 1, 0, s>>>(a.step_counter, n);
  return cudaGetLastError();
}

cudaError_t launch_batch(bool shear, const BatchArgs &a, int grid, int threads, cudaStream_t s) {
  void *args[] = {const_cast<BatchArgs *>(&a)};
  const void *fn = shear ? (const void *)batch_kernel<true> : (const void *)batch_kernel<false>;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(threads), args, 0, s);
}

}  // namespace flbm
