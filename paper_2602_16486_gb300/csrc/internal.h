// Host-side internals shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace flbm {

constexpr int kStepBlock = 128;   // threads per block of the step kernels (x direction)
constexpr int kStatsBlock = 128;  // threads (= sites per tile) of the statistics kernel

// Arguments of one fused step launch (passed by value, lives in the constant bank).
struct StepArgs {
  void *f;            // populations (deviations), Q planes of `plane` elements
  long long plane;    // nx * ny * nz
  int nx, ny, nz;
  float rho0;
  uint32_t key0, key1;        // noise key (seed)
  uint32_t ks0[10], ks1[10];  // Philox round keys: key0 + r 0x9E3779B9, key1 + r 0xBB67AE85
  uint32_t step_lo, step_hi;  // step number of this update
  // Planes updated: z_lo .. z_lo + nz_grid - 1 (the whole box: 0 and nz; a slab of a
  // decomposed lattice: its owned planes between two ghost planes), and the global index of
  // local site 0 (0 for a whole box), added to the local site index that keys the noise.
  int z_lo, nz_grid;
  uint32_t site_base;
  int *status;        // device word: nonzero after a bounded wait gave up (pipelined kernel)
  float om[27];       // 1 - Lambda_v (conserved modes: unused)
  float phc[27];      // sqrt(kBT Lambda_v (2 - Lambda_v) b_v / cs^2); phi_v = sqrt(rho) phc_v
  float om_t[27];     // om and phc times the mode's tile scale (lattice.cuh, tile_scale): the
  float phc_t[27];    // constants the D2Q9 / D3Q27 collision takes (isotropic modes 4-6: 1)
};

// ---- batched ensembles (batch.cu) ----------------------------------------------------
constexpr int kBatchMaxThreads = 256;  // largest tile: 512 sites (two per thread)

constexpr int kBatchMaxLattices = 512;  // bound of the by-value lattice table below
constexpr uint32_t kBatchWaitPolls = 1u << 22;  // polls of about a microsecond each

struct BatchLattice {  // one lattice of a batch (FP32 storage); lives in the kernel arguments
  uint32_t f256;   // populations at pool + 256 f256 bytes (the batch's allocation)
  uint32_t plane;  // nx * ny * nz (< 2^32)
  int nx, ny, nz;
  uint32_t dpp;    // D | p_hp << 8 | p_ny << 16 (lattice dimension and the shifts below)
  float rho0;
  uint32_t key0, key1;                  // noise key (seed)
  float sqrt_kbt, om_shear, phc_shear;  // rates in the paper's structure (ShearRates)
  int tile0;                            // index of the lattice's first tile
  // Division by the row's pair-slot count and by ny as a multiply-high and a shift:
  // q = (x * m) >> p with p = 31 + ceil(log2 d), m = ceil(2^p / d), exact for x < 2^31.
  uint32_t m_hp, m_ny;
  __host__ __device__ int D() const { return (int)(dpp & 0xFFu); }
  __host__ __device__ int p_hp() const { return (int)((dpp >> 8) & 0xFFu); }
  __host__ __device__ int p_ny() const { return (int)((dpp >> 16) & 0xFFu); }
};
// (m, p) of the division by d >= 1 described at BatchLattice.
inline void batch_magic(uint32_t d, uint32_t *m, int *p) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  *p = 31 + l;
  *m = (uint32_t)(((1ull << *p) + d - 1) / d);
}
struct BatchArgs {
  const float *rates;        // general rates: om[27] then phc[27] per lattice (device)
  char *pool;                // the allocation holding every lattice's populations
  int nlat, ntiles, nsteps;  // lattices, tiles (all lattices), steps of this launch
  int tile_slots[2];         // pair slots (two x-adjacent sites) per tile = threads per block:
                             // [0] the D2Q9 lattices, [1] the D3Q27 lattices
  long long *step_counter;   // device: completed steps of every lattice
  int *done;                 // device, one per lattice, zero at launch: tiles finished
  unsigned int *exits;       // device, zero at launch: blocks that have left
  int *status;               // nonzero after a bounded wait gave up
  int target_bias;           // added to every completion target (0; a test hook raises it)
  uint32_t wait_polls;       // bound of each wait, in polls
  BatchLattice lats[kBatchMaxLattices];
};
static_assert(sizeof(BatchArgs) <= 32764, "batch kernel arguments exceed the parameter space");
cudaError_t batch_max_blocks(bool shear, int threads, int *blocks_per_sm);
cudaError_t launch_batch(bool shear, const BatchArgs &a, int grid, int threads, cudaStream_t s);
// The lattices of one type: table entries [lat_lo, lat_hi) owning tiles
// [tile0, tile0 + ntiles).
struct BatchGroup {
  int lat_lo, lat_hi, tile0, ntiles;
};
// Launch forms of a batch (values of flbm_batch_set_shape's `form`).
enum BatchForm {
  kBatchStep = 0,        // per-step launches, 128-register cap, unrolled D3Q27 noise
  kBatchPersistent = 1,  // one cooperative launch, per-lattice completion counters
  kBatchStepOcc = 2,     // per-step launches, five (D3Q27) / ten (D2Q9) blocks of <= 128 per SM
  kBatchStepRolled = 3,  // per-step launches, 128-register cap, rolled D3Q27 noise
  kBatchFormMax = 3
};
// n steps as plain launches (per step one launch per lattice type, block = tile, each
// type in its own per-step form and block size), then the step-counter update.
cudaError_t launch_batch_steps(int form3, int threads3, int form2, int threads2, bool shear, int parity0,
                               const BatchArgs &a, const BatchGroup &g3, const BatchGroup &g2, int n,
                               cudaStream_t s);

// Statistics accumulators, in doubles: see stats.cu for the layout.
int stats_nacc(int Q);
inline int stats_record_len(int Q) { return stats_nacc(Q) + 1; }  // + non-finite count

// Step-kernel variants (the autotuner's search space; all compute the same update):
// one site per thread; two sites per thread (nx even) with the noise loop unrolled or
// rolled; or the bulk-copy pipelined persistent kernel (step_pipe.cu; needs
// pipe_applicable). `shear` selects the specialisation for the paper's rate structure
// (rate 1 for every non-conserved mode but the shear ones).
enum StepVariant {
  kStepAuto = 0,
  kStepOneSite = 1,
  kStepPair = 2,
  kStepPairRolled = 3,
  kStepPipelined = 4,
  kStepPairOcc = 5,        // as 2, register cap for five blocks per SM (D3Q27)
  kStepPairRolledOcc = 6,  // as 3, register cap for five blocks per SM (D3Q27)
  kStepPairOccRows = 7,    // as 5, blocks of kRowBlockRows rows x 32 pair slots (short rows)
  kStepPairRows = 8,       // as 2, blocks of kRowBlockRows rows x 32 pair slots (short rows)
  kStepVariantMax = 8
};
constexpr int kRowBlockRows = 4;  // rows per block of variants 7 and 8 (one row per warp)
bool pipe_applicable(int D, int storage, int nx);
// lattice: the public lattice id (0 D2Q9, 1 D3Q27, 2 D3Q27 isotropic, 3 D3Q19).
cudaError_t launch_step(int lattice, int storage, int variant, int parity, bool noise, bool shear,
                        const StepArgs &a, cudaStream_t s);
// Per translation unit (step_16.cu, step_iso.cu).
cudaError_t launch_step_16(int D, int storage, int variant, int parity, bool noise, bool shear, const StepArgs &a,
                           cudaStream_t s);
cudaError_t launch_step_iso(int storage, int variant, int parity, bool noise, bool shear, const StepArgs &a,
                            cudaStream_t s);
cudaError_t launch_step_d3q19(int storage, int variant, int parity, bool noise, bool shear, const StepArgs &a,
                              cudaStream_t s);
cudaError_t launch_step_pipelined(int D, int storage, int parity, bool noise, bool shear,
                                  const StepArgs &a, cudaStream_t s);
// The raw-moment collision (step_raw.cu): D 2 or 3, variants 1 (one site) and 2 (pairs).
cudaError_t launch_step_raw(int D, int storage, int variant, int parity, bool noise, const StepArgs &a,
                            cudaStream_t s);
// Statistics of the sites [site0, site0 + nsites) of the array (the whole box: 0, plane).
cudaError_t launch_stats(int D, int storage, bool iso, int parity, const void *f, long long plane, int nx,
                         int ny, int nz, float rho0, double *acc, cudaStream_t s, long long site0,
                         long long nsites);
// site_base: global index of local site 0 (keys the density perturbation).
cudaError_t launch_init(int D, int storage, void *f, long long plane, int nx, int ny, int nz,
                        double rho0, double ux, double uy, double uz, double amp,
                        uint64_t perturb_seed, uint32_t site_base, cudaStream_t s);
cudaError_t launch_gather_plane(int D, int storage, int parity, const void *f, long long plane,
                                int nx, int ny, int nz, double rho0, int q, double *out,
                                cudaStream_t s);
cudaError_t launch_scatter_plane(int D, int storage, int parity, void *f, long long plane, int nx,
                                 int ny, int nz, double rho0, int q, const double *in,
                                 cudaStream_t s);
cudaError_t launch_gather_sites(int D, int storage, int parity, const void *f, long long plane,
                                int nx, int ny, int nz, double rho0, const long long *sites,
                                long long n, double *out, cudaStream_t s);

// Modal norms b_v of the device bases (host copy, computed from the same tensor
// structure the kernels use) and the storage element size.
double mode_bnorm(int D, int v);
// b_v of the lattice's basis (lattice 2: the isotropic D3Q27 variant, modes 4-6 rotated).
double mode_bnorm_lattice(int lattice, int v);
// Tile scale of mode v of a public lattice (1 for D3Q19, whose collision has no tile).
float mode_tile_scale(int lattice, int v);
size_t storage_bytes(int storage);

}  // namespace flbm
