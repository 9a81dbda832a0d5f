// Batched ensembles: many independent periodic lattices (mixed D2Q9 / D3Q27, own size,
// rates, kBT and noise seed) advanced together, each by exactly the fused update of a
// single context (the collision of collide.cuh, packed FP32x2, the AA pattern of step.cu)
// with its own parameters.
//
// The host lays every lattice's populations out in one allocation and cuts all lattices
// into tiles of equal pair-slot count (one slot of two x-adjacent sites per thread; a
// tile may span rows, never lattices). Two launch structures (BatchForm):
//
// Per-step forms (the default): per step one plain launch per lattice type, block b on
// tile tile0 + b, the hardware block scheduler balancing the load; the n launches of a
// call are captured once into a CUDA graph and replayed.
//
// Persistent form: one cooperative launch runs n steps; block b takes the work items
// (step s, tile b + j G) in step-major order. There is no grid-wide barrier between
// steps. Lattices are independent, so a tile of lattice L at step s only has to wait
// until every tile of L has finished step s - 1 (in-place AA streaming reads and writes
// neighbour slots across tile boundaries). Each lattice has a completion counter; a block
// announces a finished tile with a release (fence, then atomic add) and checks the
// counter of the next tile's lattice with an acquire before starting it. Progress is
// guaranteed: all blocks are resident (cooperative launch), each walks its items in
// order, and the lowest pending item only depends on items of the step before it, which
// are all complete. Every wait is bounded: a block that polls longer than wait_polls times
// (or sees another block's failure) sets the status word and leaves; the host reports
// FLBM_ETIMEOUT.
//
// The per-lattice parameters travel by value in the kernel arguments (constant bank; at
// most kBatchMaxLattices lattices). A tile's lattice is found by a binary search over the
// lattices' first-tile indices in that table, from the block's own counters only, so the
// lattice's parameters stay block-uniform values (uniform registers) instead of occupying
// every thread's registers. All lattices share the step counter in device memory, read
// by every launch, so that one captured graph serves every call with the same n (and,
// for the per-step forms, the same starting parity).
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

// Pair slots of lattice L: row r = y + ny z holds ceil(nx / 2) slots, and slot j of it
// is the sites x0 = 2 j and x0 + 1 (only x0 in the last slot of a row when nx is odd).
// Slots are numbered row-major, so consecutive slots are consecutive sites and a warp's
// accesses stay contiguous for every nx.
__device__ __forceinline__ uint32_t pair_slots(const BatchLattice &L) {
  return (uint32_t)((L.nx + 1) >> 1) * (uint32_t)L.ny * (uint32_t)L.nz;
}

__device__ __forceinline__ uint32_t udiv_magic(uint32_t x, uint32_t m, int p) {
  return (uint32_t)(((unsigned long long)x * m) >> p);
}

// Row coordinates of pair slot `slot` (32-bit arithmetic: every site index is < 2^32, so
// slots and rows are < 2^31) and the site index of its first site: 2 slot when nx is even,
// 2 slot - r otherwise. The divisions use the lattice's multiply-shift constants.
__device__ __forceinline__ uint32_t slot_xyz(const BatchLattice &L, uint32_t slot, int &x0, int &y, int &z) {
  const uint32_t hp = (uint32_t)((L.nx + 1) >> 1);
  const uint32_t r = udiv_magic(slot, L.m_hp, L.p_hp());
  x0 = 2 * (int)(slot - r * hp);
  const uint32_t q = udiv_magic(r, L.m_ny, L.p_ny());
  y = (int)(r - q * (uint32_t)L.ny);
  z = (int)q;
  return 2u * slot - ((L.nx & 1) ? r : 0u);
}

// Sites of a pair slot of an odd-nx row: x0 - 1, x0, x0 + 1 and x0 + 2 (periodic), and
// the periodic row / plane offsets as in Addr2. Lane 0 is site x0 and uses s[0..2]; lane
// 1 is x0 + 1 and uses s[1..3]. In the last slot of a row (x0 = nx - 1) lane 1 wraps to
// a real site of the same row: it is loaded and collided (every access stays inside the
// lattice) but never stored.
struct OddPair {
  long long s[4];
  long long dy[3], dz[3];
};

__device__ __forceinline__ OddPair odd_pair(int x0, int y, int z, int nx, int ny, int nz) {
  OddPair a;
  const long long row = ((long long)z * ny + y) * nx;
  int x1 = x0 + 1;
  if (x1 >= nx) x1 -= nx;
  int x2 = x1 + 1;
  if (x2 >= nx) x2 -= nx;
  a.s[0] = row + (x0 == 0 ? nx - 1 : x0 - 1);
  a.s[1] = row + x0;
  a.s[2] = row + x1;
  a.s[3] = row + x2;
  const long long rl = nx, pl = (long long)nx * ny;
  a.dy[0] = (y == 0) ? (long long)(ny - 1) * rl : -rl;
  a.dy[1] = 0;
  a.dy[2] = (y == ny - 1) ? -(long long)(ny - 1) * rl : rl;
  a.dz[0] = (z == 0) ? (long long)(nz - 1) * pl : -pl;
  a.dz[1] = 0;
  a.dz[2] = (z == nz - 1) ? -(long long)(nz - 1) * pl : pl;
  return a;
}

// As load_logical2 for an odd-nx pair: scalar accesses (the pair is not 8-byte aligned).
template <int D, int PARITY>
__device__ __forceinline__ void load_odd_pair(const float *__restrict__ f, long long plane, const OddPair &ad,
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
          const float *b = f + i * plane;
          v.x = b[ad.s[1]];
          v.y = b[ad.s[2]];
        } else {
          // f_i(x) = A[opposite(i)][x - c_i]
          const float *b = f + opposite<D>(i) * plane + ad.dy[1 - dy] + ad.dz[1 - dz];
          v.x = b[ad.s[1 - dx]];
          v.y = b[ad.s[2 - dx]];
        }
        F[dz + 1][dy + 1][dx + 1] = v;
      }
}

// As store_streamed2 for an odd-nx pair; lane 1 only when `two`.
template <int D, int PARITY>
__device__ __forceinline__ void store_odd_pair(float *__restrict__ f, long long plane, const OddPair &ad, bool two,
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
        float *b;
        int k0, k1;
        if (PARITY == 0) {
          b = f + opposite<D>(i) * plane;
          k0 = 1;
          k1 = 2;
        } else {
          // f*_i(x) goes to A[i][x + c_i]
          b = f + i * plane + ad.dy[1 + dy] + ad.dz[1 + dz];
          k0 = 1 + dx;
          k1 = 2 + dx;
        }
        b[ad.s[k0]] = v.x;
        if (two) b[ad.s[k1]] = v.y;
      }
}

// The two sites of pair slot `slot` of lattice L. EVEN (nx even): the sites share a row
// and move as 8-byte pairs (Addr2, as the single-lattice kernels). Otherwise scalar
// accesses through OddPair. Either way the neighbour addresses are recomputed at the
// store rather than kept live across the collision (register pressure).
template <int D, int PARITY, bool SHEAR, bool EVEN, bool ROLLED = true>
__device__ __forceinline__ void batch_sites(const BatchLattice &L, char *pool, const float *rates, uint32_t slot,
                                            uint32_t step_lo, uint32_t step_hi) {
  float *__restrict__ f = reinterpret_cast<float *>(pool + 256ull * L.f256);
  const long long plane = L.plane;
  float2 F[3][3][3];
  uint32_t s0, dsite = 1u;
  {
    int x0, y, z;
    s0 = slot_xyz(L, slot, x0, y, z);
    if (EVEN) {  // the single-lattice pairing: odd steps take sites x0 + 1 and x0 + 2
      const Addr2 ad = addr2(x0, y, z, L.nx, L.ny, L.nz);
      load_pairs<D, float, PARITY>(f, plane, ad, F);
      s0 = pair_site0<PARITY>(ad);
      dsite = pair_dsite<PARITY>(ad);
    } else {
      load_odd_pair<D, PARITY>(f, plane, odd_pair(x0, y, z, L.nx, L.ny, L.nz), F);
    }
  }
  collide_lattice<D, SHEAR, ROLLED>(F, L, rates, s0, dsite, step_lo, step_hi);
  // The empty asm hides the slot's provenance so that the compiler cannot merge the
  // store's address computation with the load's (and keep 18 registers live).
  uint32_t sl = slot;
  asm volatile("" : "+r"(sl));
  int x0, y, z;
  slot_xyz(L, sl, x0, y, z);
  if (EVEN)
    store_pairs<D, float, PARITY>(f, plane, addr2(x0, y, z, L.nx, L.ny, L.nz), F);
  else
    store_odd_pair<D, PARITY>(f, plane, odd_pair(x0, y, z, L.nx, L.ny, L.nz), x0 + 1 < L.nx, F);
}

// Pair slot first + threadIdx.x of tile [first, end) of lattice L.
template <int PARITY, bool SHEAR>
__device__ __forceinline__ void batch_tile(const BatchLattice &L, char *pool, const float *rates, uint32_t first,
                                           uint32_t end,
                                           uint32_t step_lo, uint32_t step_hi) {
  const uint32_t slot = first + threadIdx.x;
  if (slot >= end) return;
  if (L.D() == 3) {
    if (L.nx % 2 == 0)
      batch_sites<3, PARITY, SHEAR, true>(L, pool, rates, slot, step_lo, step_hi);
    else
      batch_sites<3, PARITY, SHEAR, false>(L, pool, rates, slot, step_lo, step_hi);
  } else {
    if (L.nx % 2 == 0)
      batch_sites<2, PARITY, SHEAR, true>(L, pool, rates, slot, step_lo, step_hi);
    else
      batch_sites<2, PARITY, SHEAR, false>(L, pool, rates, slot, step_lo, step_hi);
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
    const uint32_t per = (uint32_t)a.tile_slots[L.D() == 3 ? 1 : 0];
    const uint32_t first = (uint32_t)(t - L.tile0) * per;
    const uint32_t slots = pair_slots(L);
    const uint32_t end = first + per < slots ? first + per : slots;
    const unsigned long long step = (unsigned long long)(step0 + s);
    const uint32_t lo = (uint32_t)step, hi = (uint32_t)(step >> 32);
    if (step & 1)
      batch_tile<1, SHEAR>(L, a.pool, a.rates + 54 * lat, first, end, lo, hi);
    else
      batch_tile<0, SHEAR>(L, a.pool, a.rates + 54 * lat, first, end, lo, hi);
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
  const uint32_t per = (uint32_t)a.tile_slots[D == 3 ? 1 : 0];
  const uint32_t first = (uint32_t)(t - L.tile0) * per;
  const uint32_t slots = pair_slots(L);
  const uint32_t end = first + per < slots ? first + per : slots;
  const uint32_t slot = first + threadIdx.x;
  if (slot >= end) return;
  const unsigned long long step = (unsigned long long)(*a.step_counter + k);
  const float *rates = a.rates + 54 * lat;
  char *pool = a.pool;
  if (L.nx % 2 == 0)
    batch_sites<D, PARITY, SHEAR, true, ROLLED>(L, pool, rates, slot, (uint32_t)step, (uint32_t)(step >> 32));
  else
    batch_sites<D, PARITY, SHEAR, false, ROLLED>(L, pool, rates, slot, (uint32_t)step, (uint32_t)(step >> 32));
}

// Advances the shared step counter after the n step launches of one call.
__global__ void batch_advance_kernel(long long *step_counter, int n) { *step_counter += n; }

}  // namespace

cudaError_t batch_max_blocks(bool shear, int threads, int *blocks_per_sm) {
  return shear ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel<true>, threads, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel<false>, threads, 0);
}

// Launch shapes of the per-step form (BatchForm): register cap 128 (up to 256 threads,
// two blocks per SM), or up to 128 threads with five (D3Q27, 102 registers) or ten (D2Q9,
// 51 registers: its lighter update gains from the extra warps) blocks per SM; D3Q27
// noise loop unrolled or rolled (D2Q9 has no loop).
template <int D, bool SHEAR, int PARITY>
cudaError_t launch_group(int form, const BatchArgs &a, int k, const BatchGroup &g, int threads, cudaStream_t s) {
  if (g.ntiles <= 0) return cudaSuccess;
  if (form == kBatchStepOcc)  // D3Q27: five blocks per SM; the lighter D2Q9 update: ten
    batch_step_kernel<D, SHEAR, PARITY, false, D == 3 ? 5 : 10><<<g.ntiles, threads, 0, s>>>(a, k, g.lat_lo,
                                                                                         g.lat_hi, g.tile0);
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

cudaError_t launch_batch_steps(int form3, int threads3, int form2, int threads2, bool shear, int parity0,
                               const BatchArgs &a, const BatchGroup &g3, const BatchGroup &g2, int n,
                               cudaStream_t s) {
  for (int k = 0; k < n; ++k) {
    const int parity = (parity0 + k) & 1;
    cudaError_t e = launch_group_any<3>(form3, shear, parity, a, k, g3, threads3, s);
    if (e == cudaSuccess) e = launch_group_any<2>(form2, shear, parity, a, k, g2, threads2, s);
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
