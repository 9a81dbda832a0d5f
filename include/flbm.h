/*
 * flbm.h - C ABI of the GB300 (sm_103a) fluctuating central-moment lattice Boltzmann
 * library: the fused collide-and-stream step of De Rosis & Zhou, "A fluctuating
 * lattice Boltzmann formulation based on orthogonal central moments" (arXiv:2602.16486),
 * for D2Q9 and D3Q27 on periodic boxes.
 *
 * Conventions shared by every call
 *  - Every function returns an int status (enum flbm_status); no C++ exception ever
 *    crosses this boundary. On failure flbm_last_error() describes the cause.
 *  - Out-pointers are written only when the call returns FLBM_OK (flbm_stats and
 *    flbm_fetch_samples also write on FLBM_ENUMERIC, see there).
 *  - The library owns everything it allocates. A device buffer or stream handed in by
 *    the caller (flbm_create_ex) stays owned by the caller and must outlive the context.
 *  - All device work of a context is issued on one CUDA stream (its own, or the
 *    caller's). flbm_step and flbm_sample only enqueue work and never synchronise;
 *    calls that return host data synchronise that stream.
 *  - Populations cross the ABI in logical order, FP64, laid out [q][z][y][x] with x
 *    fastest and q in the paper's velocity order (Sec. II-B for D2Q9, Sec. II-C for
 *    D3Q27), whatever the storage type or the in-place streaming parity.
 *  - Sites are numbered site = x + nx * (y + ny * z).
 *  - A context is not thread safe: one host thread at a time may call into it.
 */
#ifndef FLBM_H
#define FLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct flbm_ctx flbm_ctx;
typedef struct flbm_batch flbm_batch;

/* Lattices: D2Q9 (Sec. II-B) and D3Q27 (Sec. II-C). FLBM_D3Q27_ISO is D3Q27 with its
 * normal-stress modes 4-6 replaced by their trace and two deviators,
 *   M4' = M4 + M5 + M6,  M5' = M4 - M5,  M6' = M4 + M5 - 2 M6   (norms 2/3, 4/9, 4/3),
 * an orthogonal basis of the same space. The paper relaxes modes 4-6 at rate 1 (Sec. II-C),
 * which makes the viscosity of extensional flow differ from that of shear; with the
 * deviators at the shear rate (Lambda_5 = Lambda_6 = Lambda_7..9) the variant has one
 * viscosity, and Lambda_4 is the bulk rate. Statistics report k_4..k_6 in this basis.
 * Step variants 3, 4 and 6 run as 2, 2 and 5 for it. Not available in batches.
 * FLBM_D3Q19 is the reduced lattice of Sec. II-C ("Lattice-agnostic construction and the
 * D3Q19 example"): rest, axis and face-diagonal velocities (weights 1/3, 1/18, 1/36) in the
 * order of the first 19 D3Q27 velocities, the printed 19-mode basis and norms, Lambda_7..9
 * the shear rates, and the equilibrium whose central moments are (rho, 0, ..., 0). Step
 * variants 3, 4 and 6 run as 2, 2 and 5 for it. Not available in batches. */
enum flbm_lattice { FLBM_D2Q9 = 0, FLBM_D3Q27 = 1, FLBM_D3Q27_ISO = 2, FLBM_D3Q19 = 3 };

/* Storage of the deviations d_i = f_i - w_i * rho0 in device memory. All moment
 * arithmetic is FP32 whatever the storage; statistics accumulate in FP64. */
enum flbm_storage { FLBM_FP32 = 0, FLBM_BF16 = 1, FLBM_FP16 = 2 };

enum flbm_status {
  FLBM_OK = 0,
  FLBM_EINVAL = 1,   /* invalid argument or handle                                   */
  FLBM_ENOMEM = 2,   /* device or host allocation failed                             */
  FLBM_ECUDA = 3,    /* a CUDA runtime call failed (message in flbm_last_error)       */
  FLBM_ENUMERIC = 4, /* the sampled state holds non-finite values                     */
  FLBM_ETIMEOUT = 5, /* a device-side bounded wait gave up (persistent kernels, the
                        tensor-core statistics reduction); the result is not valid     */
  FLBM_ESTATE = 6    /* call not valid in the current state (e.g. sample buffer full) */
};

/* Statistics of one state, taken before the collision of step `step` (the state
 * after `step` completed steps). k_v are the central moments T(u(x)) f(x) of every
 * site in the paper's mode order (Sec. II-B / II-C); means divide by `sites`.
 * Entries beyond q (k_mean) or q*q (k_cov, row-major q x q) are zero. */
typedef struct flbm_stats_t {
  int64_t step;        /* completed steps when the sample was taken                */
  int64_t sites;       /* nx * ny * nz                                              */
  int64_t nonfinite;   /* sites whose rho, u or k is not finite (left out of sums)  */
  int32_t lattice;     /* enum flbm_lattice                                         */
  int32_t q;           /* 9 or 27                                                   */
  double mass;         /* sum_x rho(x)                                              */
  double mom[3];       /* sum_x rho u (x)                                           */
  double u_mean[3];    /* <u_a>                                                     */
  double uu[6];        /* <u_a u_b>: xx, yy, zz, xy, xz, yz                         */
  double k_mean[27];   /* <k_v>                                                     */
  double k_cov[27 * 27]; /* <k_v k_w> (raw second moments, symmetric)              */
} flbm_stats_t;

/* Bytes of device memory the populations of one lattice occupy (in-place streaming:
 * one copy, Q * sites * sizeof(storage)). 0 for invalid arguments. */
size_t flbm_required_bytes(int lattice, const int64_t dims[3], int storage);

/*
 * flbm_create - build a context for one periodic lattice at rest (f = f^eq(rho0, 0)).
 *   lattice : FLBM_D2Q9, FLBM_D3Q27, FLBM_D3Q27_ISO or FLBM_D3Q19.
 *   dims    : {nx, ny, nz}, each >= 1; nz must be 1 for D2Q9; ny, nz <= 65535;
 *             nx * ny * nz < 2^32 (the site index keys the noise).
 *   lambda  : Q relaxation rates Lambda_v (Eq. cm_collision) in the paper's mode order;
 *             entries of the conserved modes (v <= D) are ignored (forced to 1, as in
 *             Sec. II-B and II-C); the others must lie in (0, 2].
 *   kBT     : thermal energy per site, >= 0 (0 disables the noise; Test 1).
 *   rho0    : reference density, > 0 (deviations are stored about w_i * rho0).
 *   seed    : 64-bit key of the counter-based noise (see flbm_step).
 * Storage FP32, a stream and device buffer owned by the library, current CUDA device.
 */
int flbm_create(flbm_ctx **out, int lattice, const int64_t dims[3], const double *lambda,
                double kBT, double rho0, uint64_t seed);

/*
 * flbm_create_ex - as flbm_create, plus
 *   storage     : enum flbm_storage.
 *   cuda_stream : a cudaStream_t to issue all work on, or NULL for a library-owned
 *                 non-blocking stream.
 *   dev_buf     : device memory for the populations (>= flbm_required_bytes, 256-byte
 *                 aligned), owned by the caller, or NULL to let the library allocate.
 *   dev_buf_bytes : size of dev_buf in bytes (ignored when dev_buf is NULL).
 */
int flbm_create_ex(flbm_ctx **out, int lattice, const int64_t dims[3], const double *lambda,
                   double kBT, double rho0, uint64_t seed, int storage, void *cuda_stream,
                   void *dev_buf, size_t dev_buf_bytes);

/* Release the context (synchronises its stream first). NULL is a no-op. */
void flbm_destroy(flbm_ctx *ctx);

/*
 * flbm_init_uniform - reset to step 0 with f = f^eq(rho(x), u0) (the equilibrium of
 * Sec. II-B / II-C, complete Hermite order), where
 *   rho(x) = rho0 * (1 + rho_perturb_amp * (2 U(x) - 1)),
 * U(x) the 23-bit uniform of word 0 of Philox4x32-10 at counter (site, 0, 0, 2^16)
 * under key perturb_seed (the paper runs from rest with uniform rho0: amp = 0).
 *   u0 : {ux, uy, uz} (uz ignored for D2Q9), |u0_a| < 1.
 */
int flbm_init_uniform(flbm_ctx *ctx, const double u0[3], double rho_perturb_amp,
                      uint64_t perturb_seed);

/*
 * flbm_step - enqueue n >= 0 time steps of the fused collide-and-stream update
 * (Sec. II-B "Algorithm of computation"; Eq. cm_collision with Eq. phi_general and the
 * streaming Eq.), numbered step, step+1, ... from the context's current step count.
 * Noise: for step s and site x the normals of the noisy modes v > D come from
 * Philox4x32-10 (key = seed, counter = (site, s mod 2^32, s div 2^32, b)) with the
 * Box-Muller transform: block b = (v - D - 1) / 4 gives four normals. Asynchronous;
 * returns launch errors only.
 */
int flbm_step(flbm_ctx *ctx, int64_t n);

/* Completed steps so far (the step index of the next update). -1 for a NULL ctx. */
int64_t flbm_get_step(const flbm_ctx *ctx);

/*
 * flbm_stats - statistics of the current state (velocity moments, Sec. III Eq. for
 * <u_a^2>; central-moment means and covariances, Sec. II-B C^eq), FP32 per site, the
 * products on the tensor cores (BF16 hi/lo splits of both factors, FP32 accumulation of
 * at most 1024 sites, at most 2^-15 relative error per product and no bias) and FP64
 * sums. Synchronises. Returns FLBM_ENUMERIC (and still fills *out) when some site is
 * not finite, FLBM_ETIMEOUT (out->nonfinite negative) if the reduction's bounded wait
 * for the tensor cores gave up.
 */
int flbm_stats(flbm_ctx *ctx, flbm_stats_t *out);

/*
 * flbm_sample - enqueue the statistics of the current state into the next slot of the
 * context's device-side sample buffer (asynchronous, no host synchronisation).
 * FLBM_ESTATE when the buffer already holds flbm_sample_capacity() samples.
 * flbm_fetch_samples - copy up to max_n recorded samples (oldest first) to out,
 * set *n_out, and empty the buffer. Synchronises. FLBM_ENUMERIC if any fetched sample
 * counted non-finite sites (out is still written).
 * flbm_set_sample_capacity - (re)allocate the buffer for cap >= 1 samples; drops any
 * recorded samples. The default capacity is 1024.
 */
int flbm_sample(flbm_ctx *ctx);
int flbm_fetch_samples(flbm_ctx *ctx, flbm_stats_t *out, int max_n, int *n_out);
int flbm_set_sample_capacity(flbm_ctx *ctx, int cap);
int flbm_sample_capacity(const flbm_ctx *ctx);

/* Logical populations f_i (FP64, [q][z][y][x]) of the whole lattice; count must equal
 * Q * sites. Synchronises. */
int flbm_get_populations(flbm_ctx *ctx, double *host, size_t count);
int flbm_set_populations(flbm_ctx *ctx, const double *host, size_t count);

/* Logical populations of n_sites chosen sites: out[s * Q + i] = f_i(sites[s]).
 * Sites must lie in [0, nx*ny*nz). Synchronises. */
int flbm_get_sites(flbm_ctx *ctx, const int64_t *sites, size_t n_sites, double *out);

/*
 * Checkpoint: a self-describing host blob (header + stored deviations in the context's
 * storage type). flbm_load requires the same lattice, dims and storage and restores
 * populations, step count, rates, kBT, rho0 and seed, so that "run a, save, load, run
 * b" is bitwise equal to "run a + b". Both synchronise.
 */
size_t flbm_checkpoint_bytes(const flbm_ctx *ctx);
int flbm_save(flbm_ctx *ctx, void *host, size_t bytes);
int flbm_load(flbm_ctx *ctx, const void *host, size_t bytes);

/*
 * flbm_stats_noalloc - the statistics of flbm_stats (same kernel, same flbm_stats_t)
 * for a population array the caller owns, with no allocation of any kind. The paper
 * has no counterpart: this entry point exists for callers that cannot allocate GPU
 * memory - an application whose own memory pool owns the whole device-memory budget
 * (a cudaMalloc from elsewhere would fail or break its accounting), or a service that
 * must not change its memory footprint once running. flbm_create cannot serve them,
 * because it allocates its buffers.
 *   lattice, dims, storage, rho0 : as given to flbm_create_ex for this array.
 *   parity          : completed steps mod 2 (flbm_get_step(ctx) & 1): 0 when the array
 *                     holds f_i(x) in slot i at x, 1 after an odd number of AA steps.
 *   dev_populations : the stored deviations, device memory, Q * sites elements of the
 *                     storage type (e.g. the dev_buf handed to flbm_create_ex), 256-byte
 *                     aligned like dev_buf (the kernel reads element pairs); any other
 *                     address is rejected with FLBM_EINVAL before device work.
 *   cuda_stream     : stream to run on (NULL = legacy default stream). The call waits
 *                     for this stream before it returns.
 *   out             : host struct, written on FLBM_OK and FLBM_ENUMERIC; out->step is
 *                     -1 (the array carries no step count).
 * Scratch: the FP64 accumulators live in one statically allocated device array of
 * FLBM_NOALLOC_SCRATCH_DOUBLES doubles (8 KiB), which every GPU that loads the library
 * keeps until the process exits. A lattice whose accumulators would not fit is rejected
 * with FLBM_EINVAL (D2Q9 needs 137 doubles, D3Q27 and D3Q19 529). The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and caches it; make
 * that first call before any stream capture. Every call reuses the same array and zeroes
 * it first, so calls whose GPU work overlaps (other streams, other host threads) race
 * and return wrong sums: serialise them.
 */
#define FLBM_NOALLOC_SCRATCH_DOUBLES 1024
int flbm_stats_noalloc(int lattice, const int64_t dims[3], int storage, int parity, double rho0,
                       const void *dev_populations, void *cuda_stream, flbm_stats_t *out);

/*
 * Step-kernel variant (launch configuration only; every variant computes the same
 * update): 0 = default (2 when nx is even, else 1), 1 = one site per thread, 2 = two
 * sites per thread, 3 = two sites per thread with the noise generated in a rolled loop
 * (smaller code), 4 = a persistent kernel that prefetches each row's populations into
 * shared memory with bulk asynchronous copies (needs nx even, nx <= 512 and a
 * population row a multiple of 16 bytes; else it falls back to 2), 5 and 6 = 2 and 3
 * compiled for more resident blocks per SM to hide latency: five for the 3-D lattices
 * (at most 102 registers), eight for D2Q9 (at most 64); 7 and 8 = 5 and 2 with blocks of
 * four rows of 32 site pairs instead of one row of 128 (for rows shorter than 256 sites,
 * which leave most of a one-row block idle). Variants 2-8 fall back to 1 when nx is odd.
 * The environment variable FLBM_STEP_VARIANT, read by flbm_create, sets the initial
 * choice.
 * flbm_autotune times every applicable variant (7 and 8 only for nx < 256) over
 * trial_steps steps on a copy of the current state (restored afterwards: populations
 * and step count are unchanged), keeps the fastest for this context and caches the
 * choice per (GPU model, lattice, storage, nx parity, size class, noise on/off, rate
 * structure, collision model, nx < 256) for the process; when the environment variable
 * FLBM_AUTOTUNE_CACHE names a file, choices are also read from it (at the first
 * flbm_autotune call of the process) and appended to it (one "key<TAB>variant" line per
 * choice), so later processes skip the trials. Needs one extra copy of the populations
 * in device memory while it runs. Synchronises.
 */
int flbm_set_step_variant(flbm_ctx *ctx, int variant);
int flbm_get_step_variant(const flbm_ctx *ctx);

/*
 * Collision model of a context (default FLBM_COLLISION_CM, the paper's scheme).
 * FLBM_COLLISION_RAW is its raw-moment counterpart, the comparison scheme of the paper:
 * T = M and N = I (Sec. II-C, end of the D3Q27 construction, names this choice as the
 * scheme's raw-moment form), i.e. the same basis, rates, amplitudes phi_v (Eq. phi_general) and normals,
 * applied to the raw moments M f with the equilibrium raw moments M f^eq(rho, u). With
 * every non-conserved rate equal to omega it is the fluctuating BGK step of Sec. II-A:
 * f* = f + omega (f^eq - f) + zeta with zeta_i = w_i sum_v b_v^-1 M_vi phi_v eta_v
 * (Eq. Xi_pop). Available for FLBM_D2Q9 and FLBM_D3Q27 (FLBM_EINVAL otherwise), not for the
 * lattices of a batch (FLBM_ESTATE); step variants 1 and 2 only (others run as 2, odd nx as
 * 1). Statistics still report the central moments of the orthogonal basis. The model is
 * saved in checkpoints. Takes effect at the next flbm_step.
 */
enum flbm_collision { FLBM_COLLISION_CM = 0, FLBM_COLLISION_RAW = 1 };
int flbm_set_collision(flbm_ctx *ctx, int model);
int flbm_get_collision(const flbm_ctx *ctx); /* -1 for a NULL ctx */
int flbm_autotune(flbm_ctx *ctx, int trial_steps, int *chosen);

/* Wait for the context's stream. FLBM_ECUDA carries any asynchronous device error. */
int flbm_sync(flbm_ctx *ctx);

/* Message of the last failing call on this host thread (library-owned, never NULL). */
const char *flbm_last_error(void);

/*
 * Batched ensembles: many independent periodic lattices, each with its own lattice
 * type, size, relaxation rates, kBT, rho0 and noise seed, advanced together by one
 * persistent kernel launch per flbm_batch_step call. Every lattice follows exactly the
 * update of a single context with the same parameters (the same Philox stream keyed on
 * its own seed, step and site); only the launch shape differs. The paper itself runs one
 * lattice at a time; ensembles of independent runs are how its fluctuation statistics
 * are gathered (Sec. III), which this form does in one launch.
 *
 * One spec per lattice (plain data, copied by flbm_batch_create):
 *   lattice, dims, lambda, kBT, rho0, seed : as for flbm_create (lambda holds Q rates).
 */
typedef struct flbm_lattice_spec {
  int32_t lattice;
  int32_t reserved; /* must be 0 */
  int64_t dims[3];
  double lambda[27];
  double kBT;
  double rho0;
  uint64_t seed;
} flbm_lattice_spec;

#define FLBM_BATCH_MAX_LATTICES 512

/*
 * flbm_batch_create - build n lattices (1 <= n <= FLBM_BATCH_MAX_LATTICES), all at rest
 * and at step 0, with FP32 storage in one device allocation.
 *   out         : receives the batch handle (release with flbm_batch_destroy).
 *   specs       : n specs, host memory, read during the call only.
 *   cuda_stream : cudaStream_t for all of the batch's work, or NULL for a stream the
 *                 batch creates and owns. Graph capture needs a stream other than the
 *                 legacy default stream.
 * Errors: FLBM_EINVAL (bad spec: the message names its index), FLBM_ENOMEM, FLBM_ECUDA.
 */
int flbm_batch_create(flbm_batch **out, const flbm_lattice_spec *specs, int n, void *cuda_stream);
void flbm_batch_destroy(flbm_batch *b);
int flbm_batch_size(const flbm_batch *b);

/*
 * flbm_batch_lattice - borrowed context of lattice i (owned by the batch; valid until
 * flbm_batch_destroy; NULL for a bad index). It shares the batch's stream, and the
 * read and exchange calls work on it as on any context: flbm_stats, flbm_sample,
 * flbm_fetch_samples, flbm_get_populations, flbm_set_populations, flbm_get_sites,
 * flbm_save. flbm_init_uniform works while the batch is at step 0; flbm_load only
 * restores a checkpoint taken at the batch's current step. flbm_step,
 * flbm_set_step_variant and flbm_autotune return FLBM_ESTATE on it (the batch steps
 * all of its lattices together), and flbm_destroy ignores it.
 */
flbm_ctx *flbm_batch_lattice(flbm_batch *b, int i);

/*
 * flbm_batch_stats - the statistics of lattice i of the batch, exactly as flbm_stats on
 * flbm_batch_lattice(b, i): velocity moments (Sec. III, <u_a^2>) and central-moment means
 * and raw second moments (Sec. II-B, C^eq) of one member of the ensemble; the paper gathers
 * its fluctuation statistics over such ensembles of independent runs (Sec. III).
 *   i   : 0 <= i < flbm_batch_size(b), else FLBM_EINVAL.
 *   out : host struct; written on FLBM_OK and on FLBM_ENUMERIC (some site not finite).
 * Waits for the batch's stream (the statistics of the state after every step enqueued
 * so far).
 */
int flbm_batch_stats(flbm_batch *b, int i, flbm_stats_t *out);

/*
 * flbm_batch_step - enqueue n >= 0 steps of every lattice. Never synchronises. Every
 * launch form (see flbm_batch_set_shape) computes the same update (bitwise):
 *   per-step forms: per step one plain launch per lattice type over all of its tiles
 *     (block = tile), then a one-thread update of the device step counter;
 *   persistent form: one cooperative launch of co-resident blocks that walk (step, tile)
 *     items in order; a tile of lattice L waits (bounded) for all of L's tiles of the
 *     step before, through per-lattice completion counters, instead of a grid barrier.
 * The n steps are captured once into a CUDA graph per (n, starting parity) and shape and
 * replayed, where the stream allows capture. A bounded wait that gives up ends the
 * persistent launch and makes the next flbm_batch_sync return FLBM_ETIMEOUT (the state
 * is then not valid).
 */
int flbm_batch_step(flbm_batch *b, int64_t n);
int64_t flbm_batch_get_step(const flbm_batch *b);

/*
 * Launch shape: threads per block (64, 128 or 256; every block takes tiles of
 * 2 * threads sites; 0 = the default, 128) and the form:
 *   0 per-step launches, up to 128 registers, D3Q27 noise loop unrolled (default);
 *   1 persistent cooperative launch (rolled noise loop, both lattice types in one kernel);
 *   2 per-step launches compiled for more resident blocks per SM: five for D3Q27 (up
 *     to 102 registers), ten for D2Q9 (up to 51); threads <= 128;
 *   3 per-step launches, up to 128 registers, D3Q27 noise loop rolled (smaller code).
 * flbm_batch_set_shape sets the shape of every lattice type; flbm_batch_get_shape
 * returns the D3Q27 lattices' one. In the per-step forms each lattice type (FLBM_D2Q9,
 * FLBM_D3Q27) launches separately and may take its own threads and per-step form
 * (flbm_batch_set_type_shape: form 0, 2 or 3; FLBM_ESTATE while the batch is in the
 * persistent form, which launches every type alike); flbm_batch_get_type_shape returns a
 * type's shape as launched.
 * flbm_batch_autotune times every (form, threads) pair for all lattices alike and then,
 * in a per-step form, every per-step shape of the D2Q9 lattices with the D3Q27 lattices'
 * shape fixed, over trial_steps steps each (rounded up to even) on a copy of the state
 * (restored afterwards, step count unchanged); keeps the fastest and returns the D3Q27
 * lattices' shape in *threads and *form (either may be NULL). Needs one extra copy of all
 * populations in device memory while it runs. Synchronises.
 */
int flbm_batch_set_shape(flbm_batch *b, int threads, int form);
int flbm_batch_get_shape(const flbm_batch *b, int *threads, int *form);
int flbm_batch_set_type_shape(flbm_batch *b, int lattice, int threads, int form);
int flbm_batch_get_type_shape(const flbm_batch *b, int lattice, int *threads, int *form);
int flbm_batch_autotune(flbm_batch *b, int trial_steps, int *threads, int *form);

/* 1 when the last flbm_batch_step replayed a captured graph, 0 when it launched
 * directly (capture unavailable on this stream or runtime), -1 for a NULL handle. */
int flbm_batch_uses_graph(const flbm_batch *b);

/* Wait for the batch's stream; FLBM_ETIMEOUT if a bounded wait of the persistent form
 * gave up (the flag is cleared, and the step count is reset to the last completed
 * launch: the populations are not valid until re-initialised or loaded), FLBM_ECUDA for
 * an asynchronous device error. */
int flbm_batch_sync(flbm_batch *b);

/*
 * flbm_batch_test_wait_timeout - test hook (the paper has no counterpart): the next
 * flbm_batch_step, if it runs the persistent form, waits for completion counts that are
 * never reached, and each wait gives up after `polls` polls (about a microsecond each),
 * exactly as a real stall would; flbm_batch_sync then returns FLBM_ETIMEOUT. Exercises the
 * timeout path without faulting or hanging the GPU. The hook disarms after one call.
 */
int flbm_batch_test_wait_timeout(flbm_batch *b, uint32_t polls);

/*
 * Domain decomposition. One periodic 3-D lattice (FLBM_D3Q27, FLBM_D3Q27_ISO, FLBM_D3Q19)
 * split along z into slabs of whole planes, for several GPUs (one slab each) or several
 * slabs on one GPU. The update is the fused step of flbm_step with the periodic streaming
 * of Eq. streaming across the whole lattice; the noise is keyed on the global site
 * x + nx (y + ny z), so a decomposed lattice evolves bitwise like the whole one.
 *
 * A slab's device array holds its z_count owned planes between two ghost planes, laid out
 * [q][p][y][x] with p = 0 .. z_count + 1 (p = 1 .. z_count are the global planes z_begin
 * .. z_begin + z_count - 1). With the in-place AA pattern, a step taken from an even step
 * count touches only each site's own slots and needs no exchange. A step taken from an
 * odd step count reads and writes the neighbours' slots, so around it the slots of the
 * velocities with c_z != 0 move across each slab face (9 slots per face site for D3Q27,
 * 5 for D3Q19):
 *   phase 0, before the step: each boundary plane's slots of the velocities leaving through
 *            the face are copied into the neighbour's ghost plane;
 *   phase 1, after the step:  the ghost plane's slots the step wrote are copied back to the
 *            neighbour's boundary plane.
 * No other slot of a boundary plane is touched by the neighbour, so these are the only
 * transfers. Statistics and population reads of a slab in an odd state need phase 0 done.
 */

/* Bytes of a slab's local array (owned and ghost planes); 0 for invalid arguments. */
size_t flbm_slab_required_bytes(int lattice, const int64_t dims[3], int64_t z_count, int storage);

/*
 * flbm_create_slab - context of the owned planes [z_begin, z_begin + z_count) of the
 * lattice dims (global {nx, ny, nz}); other arguments as flbm_create_ex (dev_buf, if
 * given, >= flbm_slab_required_bytes and 256-byte aligned). The context works as any other
 * with these differences: flbm_step advances at most one step per call (the caller
 * exchanges the halo, see flbm_slab_halo, around every step taken from an odd step count);
 * flbm_stats covers the owned planes only (sites = nx ny z_count; add slabs' sums to
 * combine); flbm_get/set_populations, flbm_save/load cover the whole local array, ghost
 * planes included; flbm_autotune is refused (FLBM_ESTATE); step variant 4 runs as 2.
 * Errors: FLBM_EINVAL for D2Q9, a plane range outside [0, nz) or a local array of 2^32
 * sites or more.
 */
int flbm_create_slab(flbm_ctx **out, int lattice, const int64_t dims[3], int64_t z_begin, int64_t z_count,
                     const double *lambda, double kBT, double rho0, uint64_t seed, int storage, void *cuda_stream,
                     void *dev_buf, size_t dev_buf_bytes);

/*
 * flbm_slab_halo - the regions of one halo message of a slab with z_count owned planes
 * (host only; needs no GPU). phase: 0 (before the step) or 1 (after it); side: 0 for the
 * message exchanged with the neighbour below (planes z_begin - 1 ...), 1 with the one above.
 * On return region k (k < *n_regions, at most 9) of the message is the run of *region_len
 * = nx * ny elements starting at element send_offset[k] of this slab's array (what this
 * slab sends), and the matching region of the neighbour's message lands at element
 * recv_offset[k] of this slab's array. Region k of a (phase, side 0) message pairs with
 * region k of the lower neighbour's (phase, side 1) message, and vice versa, so a message
 * is sent and received region by region in this order. Every output array holds 9 entries.
 */
int flbm_slab_halo(int lattice, const int64_t dims[3], int64_t z_count, int phase, int side,
                   int64_t *send_offset, int64_t *recv_offset, int *n_regions, int64_t *region_len);

/*
 * A domain: nslabs slabs of one lattice in this process, planes split as evenly as
 * possible (the first nz mod nslabs slabs one plane thicker), slab k on devices[k] (or
 * every slab on the current device when devices is NULL), each with its own stream; the
 * halo moves by cudaMemcpyAsync between the slabs' arrays (peer copies across devices),
 * ordered by events. Every slab starts at rest at step 0.
 *   flbm_domain_step        : enqueue n steps of the whole lattice (never synchronises).
 *   flbm_domain_stats       : statistics of the whole lattice, the slabs' FP64 sums added;
 *                             synchronises; FLBM_ENUMERIC as flbm_stats.
 *   flbm_domain_get/set_populations : logical FP64 populations of the whole lattice,
 *                             [q][z][y][x]; synchronise.
 *   flbm_domain_slab        : borrowed context of slab k (read-only use; NULL if no such
 *                             slab); flbm_destroy ignores it.
 *   flbm_domain_set_step_variant : as flbm_set_step_variant, for every slab.
 */
typedef struct flbm_domain flbm_domain;
int flbm_domain_create(flbm_domain **out, int lattice, const int64_t dims[3], const double *lambda, double kBT,
                       double rho0, uint64_t seed, int storage, int nslabs, const int *devices);
void flbm_domain_destroy(flbm_domain *d);
int flbm_domain_size(const flbm_domain *d);
flbm_ctx *flbm_domain_slab(flbm_domain *d, int k);
int flbm_domain_init_uniform(flbm_domain *d, const double u0[3], double rho_perturb_amp, uint64_t perturb_seed);
int flbm_domain_step(flbm_domain *d, int64_t n);
int64_t flbm_domain_get_step(const flbm_domain *d);
int flbm_domain_set_step_variant(flbm_domain *d, int variant);
int flbm_domain_stats(flbm_domain *d, flbm_stats_t *out);
int flbm_domain_get_populations(flbm_domain *d, double *host, size_t count);
int flbm_domain_set_populations(flbm_domain *d, const double *host, size_t count);
int flbm_domain_sync(flbm_domain *d);

#ifdef __cplusplus
}
#endif

#endif /* FLBM_H */
