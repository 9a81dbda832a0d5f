// C ABI of the library (declared and documented in include/flbm.h): argument checks,
// context and batch ownership, launch sequencing, graph capture of batch steps, the
// autotuners and host <-> device exchange. Every compute step runs in the kernels of the
// other translation units: the step (step.cu, step_16.cu, step_iso.cu, step19.cu,
// step_pipe.cu), the statistics (stats.cu), initialisation and exchange (state.cu) and
// batches (batch.cu).
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/flbm.h"
#include "internal.h"
#include "lattice.cuh"

using namespace flbm;

struct flbm_ctx {
  int lattice = 0, D = 2, Q = 9, storage = 0;
  int64_t dims[3] = {1, 1, 1};
  long long N = 1;
  double lambda[27] = {};
  double kBT = 0.0, rho0 = 1.0;
  uint64_t seed = 0;
  int64_t step = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void *f = nullptr;
  bool own_f = false;
  size_t f_bytes = 0;
  double *d_acc = nullptr;  // statistics accumulators (stats_record_len doubles)
  double *h_acc = nullptr;  // pinned host mirror of d_acc
  double *d_ring = nullptr;  // sample buffer: ring_cap records
  int ring_cap = 0, ring_count = 0;
  std::vector<int64_t> ring_steps;
  double *d_stage = nullptr;  // FP64 staging for population exchange
  size_t stage_elems = 0;
  long long *d_sites = nullptr;
  size_t sites_cap = 0;
  int variant = 0;  // enum StepVariant; 0 = default choice
  bool shear = false;  // rates follow the paper's structure (collide.cuh, SHEAR)
  bool iso = false;    // the isotropic D3Q27 variant (lattice FLBM_D3Q27_ISO)
  int *d_status = nullptr;  // device status word of the pipelined kernel
  StepArgs args{};
  flbm_batch *owner = nullptr;  // set for a lattice of a batch (borrowed handle)
  bool params_changed = false;  // a lattice of a batch reloaded its parameters
  // One slab of a lattice decomposed along z (flbm_create_slab): dims and N describe the
  // local array, whose planes 1 .. z_count are the global planes z_begin .. z_begin +
  // z_count - 1 and whose planes 0 and z_count + 1 are ghost copies of the neighbours'.
  bool slab = false;
  int64_t gdims[3] = {1, 1, 1};  // the whole lattice
  int64_t z_begin = 0, z_count = 0;
  bool in_domain = false;  // a slab owned by a flbm_domain (stepped by it)
  int model = FLBM_COLLISION_CM;  // enum flbm_collision
};

namespace {

thread_local std::string g_last_error = "no error";

int fail(int status, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return status;
}

#define FLBM_CUDA(call)                                                                   \
  do {                                                                                    \
    const cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return fail(FLBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      return;
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int q_of(int lattice) { return lattice == FLBM_D2Q9 ? 9 : (lattice == FLBM_D3Q19 ? 19 : 27); }
int d_of(int lattice) { return lattice == FLBM_D2Q9 ? 2 : 3; }
// Lattice code of the state, exchange and statistics kernels: 2 (D2Q9), 3 (D3Q27, both
// bases) or 19 (D3Q19).
int klat(int lattice) { return lattice == FLBM_D2Q9 ? 2 : (lattice == FLBM_D3Q19 ? 19 : 3); }
// Lattices whose step kernels exist for variants 1, 2 and 5 only.
bool pair_variants_only(int lattice) { return lattice == FLBM_D3Q27_ISO || lattice == FLBM_D3Q19; }

int check_geometry(int lattice, const int64_t dims[3], int storage) {
  if (lattice != FLBM_D2Q9 && lattice != FLBM_D3Q27 && lattice != FLBM_D3Q27_ISO && lattice != FLBM_D3Q19)
    return fail(FLBM_EINVAL,
                "lattice must be FLBM_D2Q9 (0), FLBM_D3Q27 (1), FLBM_D3Q27_ISO (2) or FLBM_D3Q19 (3), got %d",
                lattice);
  if (!dims) return fail(FLBM_EINVAL, "dims is NULL");
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 1) return fail(FLBM_EINVAL, "dims[%d] = %lld must be >= 1", a, (long long)dims[a]);
  if (lattice == FLBM_D2Q9 && dims[2] != 1)
    return fail(FLBM_EINVAL, "D2Q9 needs dims[2] (nz) == 1, got %lld", (long long)dims[2]);
  if (dims[1] > 65535 || dims[2] > 65535)
    return fail(FLBM_EINVAL, "ny and nz must be <= 65535");
  if (dims[0] > 0x7fffffffLL) return fail(FLBM_EINVAL, "nx must be < 2^31");
  const double n = double(dims[0]) * double(dims[1]) * double(dims[2]);
  if (n >= 4294967296.0) return fail(FLBM_EINVAL, "nx*ny*nz must be < 2^32 (site index keys the noise)");
  if (storage < FLBM_FP32 || storage > FLBM_FP16)
    return fail(FLBM_EINVAL, "storage must be FLBM_FP32, FLBM_BF16 or FLBM_FP16, got %d", storage);
  return FLBM_OK;
}

int check_params(int lattice, const double *lambda, double kBT, double rho0) {
  if (!lambda) return fail(FLBM_EINVAL, "lambda is NULL");
  const int Q = q_of(lattice), D = d_of(lattice);
  for (int v = D + 1; v < Q; ++v)
    if (!(lambda[v] > 0.0 && lambda[v] <= 2.0))
      return fail(FLBM_EINVAL, "lambda[%d] = %g must lie in (0, 2]", v, lambda[v]);
  if (!(kBT >= 0.0) || !std::isfinite(kBT)) return fail(FLBM_EINVAL, "kBT = %g must be finite and >= 0", kBT);
  if (!(rho0 > 0.0) || !std::isfinite(rho0)) return fail(FLBM_EINVAL, "rho0 = %g must be finite and > 0", rho0);
  return FLBM_OK;
}

// Per-mode constants of the collision: om_v = 1 - L_v and
// phc_v = sqrt(kBT L_v (2 - L_v) b_v / cs^2) (Eq. phi_general without the sqrt(rho)).
void fill_args(flbm_ctx *c) {
  StepArgs &a = c->args;
  a.f = c->f;
  a.plane = c->N;
  a.nx = int(c->dims[0]);
  a.ny = int(c->dims[1]);
  a.nz = int(c->dims[2]);
  a.rho0 = float(c->rho0);
  a.status = c->d_status;
  a.z_lo = c->slab ? 1 : 0;
  a.nz_grid = c->slab ? int(c->z_count) : a.nz;
  // Global index of local site 0: nx ny (z_begin - 1), taken mod 2^32 (the ghost plane
  // below z_begin = 0 wraps; it is never updated).
  a.site_base = c->slab ? uint32_t(uint64_t(int64_t(c->dims[0] * c->dims[1]) * (c->z_begin - 1))) : 0u;
  a.key0 = uint32_t(c->seed);
  a.key1 = uint32_t(c->seed >> 32);
  for (int r = 0; r < 10; ++r) {  // Weyl key schedule of Philox4x32 (Salmon et al., SC'11)
    a.ks0[r] = a.key0 + uint32_t(r) * 0x9E3779B9u;
    a.ks1[r] = a.key1 + uint32_t(r) * 0xBB67AE85u;
  }
  for (int v = 0; v < 27; ++v) {
    a.om[v] = 0.0f;
    a.phc[v] = 0.0f;
    a.om_t[v] = 0.0f;
    a.phc_t[v] = 0.0f;
  }
  for (int v = c->D + 1; v < c->Q; ++v) {
    const double L = c->lambda[v];
    a.om[v] = float(1.0 - L);
    a.phc[v] = float(std::sqrt(c->kBT * L * (2.0 - L) * mode_bnorm_lattice(c->lattice, v) * 3.0));
    // Scales are powers of two: the products are exact.
    a.om_t[v] = a.om[v] * mode_tile_scale(c->lattice, v);
    a.phc_t[v] = a.phc[v] * mode_tile_scale(c->lattice, v);
  }
  // The paper's structure: rate 1 for every non-conserved mode except the shear modes
  // (isotropic variant: except the second-order modes 4-9).
  c->iso = c->lattice == FLBM_D3Q27_ISO;
  c->shear = true;
  for (int v = c->D + 1; v < c->Q; ++v) {
    const bool is_shear = c->iso ? (v <= 9) : (c->D == 3) ? (v >= 7 && v <= 9) : (v == 4 || v == 5);
    if (!is_shear && c->lambda[v] != 1.0) c->shear = false;
  }
}

void release(flbm_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->own_f && c->f) cudaFree(c->f);
  if (c->d_acc) cudaFree(c->d_acc);
  if (c->h_acc) cudaFreeHost(c->h_acc);
  if (c->d_ring) cudaFree(c->d_ring);
  if (c->d_stage) cudaFree(c->d_stage);
  if (c->d_sites) cudaFree(c->d_sites);
  if (c->d_status) cudaFree(c->d_status);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

int ensure_stage(flbm_ctx *c, size_t elems) {
  if (c->stage_elems >= elems) return FLBM_OK;
  if (c->d_stage) {
    cudaStreamSynchronize(c->stream);
    cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_elems = 0;
  }
  if (cudaMalloc(&c->d_stage, elems * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(FLBM_ENOMEM, "cannot allocate %zu bytes of staging memory", elems * sizeof(double));
  }
  c->stage_elems = elems;
  return FLBM_OK;
}

// Host struct from one record: the upper triangle of the Gram matrix G of the per-site
// column c = [1, rho - rho0, j, u, k_{D+1} .. k_{Q-1}, 0 ...] (NC columns; stats.cu),
// then the non-finite count. k_0 = rho = rho0 + (rho - rho0) is rebuilt in FP64; the
// central moments k_1..k_D vanish identically and are reported as 0.
// Sites the statistics cover: the whole box, or a slab's owned planes.
long long stat_site0(const flbm_ctx *c) { return c->slab ? (long long)(c->dims[0] * c->dims[1]) : 0; }
long long stat_sites(const flbm_ctx *c) {
  return c->slab ? (long long)(c->dims[0] * c->dims[1] * c->z_count) : c->N;
}

void fill_stats(const flbm_ctx *c, const double *acc, int64_t step, flbm_stats_t *out) {
  const int Q = c->Q, D = c->D;
  const int NC = D == 3 ? 32 : 16;
  auto G = [&](int a, int b) {
    if (a > b) std::swap(a, b);
    return acc[a * NC - a * (a - 1) / 2 + (b - a)];
  };
  std::memset(out, 0, sizeof(*out));
  out->step = step;
  out->sites = stat_sites(c);
  out->lattice = c->lattice;
  out->q = Q;
  out->nonfinite = (int64_t)llround(acc[NC * (NC + 1) / 2]);
  const double inv = 1.0 / double(stat_sites(c));
  const double rho0 = c->rho0, cnt = G(0, 0), sd = G(0, 1);
  out->mass = rho0 * cnt + sd;
  for (int a = 0; a < 3; ++a) {
    out->mom[a] = G(0, 2 + a);
    out->u_mean[a] = G(0, 5 + a) * inv;
  }
  const int uu_pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  for (int e = 0; e < 6; ++e) out->uu[e] = G(5 + uu_pairs[e][0], 5 + uu_pairs[e][1]) * inv;
  // column of mode v >= D + 1
  auto kc = [&](int v) { return 8 + v - D - 1; };
  out->k_mean[0] = (rho0 * cnt + sd) * inv;
  for (int v = D + 1; v < Q; ++v) out->k_mean[v] = G(0, kc(v)) * inv;
  out->k_cov[0] = (rho0 * rho0 * cnt + 2.0 * rho0 * sd + G(1, 1)) * inv;
  for (int v = D + 1; v < Q; ++v) {
    const double k0v = (rho0 * G(0, kc(v)) + G(1, kc(v))) * inv;
    out->k_cov[v] = k0v;
    out->k_cov[v * Q] = k0v;
    for (int w = v; w < Q; ++w) {
      const double vw = G(kc(v), kc(w)) * inv;
      out->k_cov[v * Q + w] = vw;
      out->k_cov[w * Q + v] = vw;
    }
  }
}

// Status of a statistics record: FLBM_ETIMEOUT when the reduction's bounded wait on the
// tensor cores gave up (it marks the non-finite count negative), FLBM_ENUMERIC when
// sites hold non-finite values, else FLBM_OK.
int stats_result(const flbm_stats_t *out, long long step) {
  if (out->nonfinite < 0)
    return fail(FLBM_ETIMEOUT, "a bounded wait of the statistics reduction gave up; the record is not valid");
  if (out->nonfinite > 0) {
    if (step >= 0)
      return fail(FLBM_ENUMERIC, "%lld sites hold non-finite values at step %lld", (long long)out->nonfinite,
                  step);
    return fail(FLBM_ENUMERIC, "%lld sites hold non-finite values", (long long)out->nonfinite);
  }
  return FLBM_OK;
}

int enqueue_stats(flbm_ctx *c, double *acc_dev) {
  FLBM_CUDA(cudaMemsetAsync(acc_dev, 0, sizeof(double) * stats_record_len(c->Q), c->stream));
  FLBM_CUDA(launch_stats(klat(c->lattice), c->storage, c->iso, int(c->step & 1), c->f, c->N, int(c->dims[0]),
                         int(c->dims[1]), int(c->dims[2]), float(c->rho0), acc_dev, c->stream, stat_site0(c),
                         stat_sites(c)));
  return FLBM_OK;
}

// Variant actually launched: the choice, or the default (two sites per thread where nx
// is even, else one site per thread); the pipelined choice falls back where it does not
// apply.
int resolve_variant(const flbm_ctx *c) {
  if (c->model == FLBM_COLLISION_RAW)  // raw-moment kernels: one site or two per thread
    return c->dims[0] % 2 != 0 || c->variant == kStepOneSite ? int(kStepOneSite) : int(kStepPair);
  const bool pipe = pipe_applicable(c->D, c->storage, int(c->dims[0]));
  int v = c->variant;
  if (v == kStepAuto) v = kStepPair;
  if (v == kStepPipelined && (!pipe || c->slab)) v = kStepPair;  // the pipelined kernel walks whole boxes
  if (pair_variants_only(c->lattice)) {  // unrolled two-site kernels only
    if (v == kStepPairRolled || v == kStepPipelined) v = kStepPair;
    if (v == kStepPairRolledOcc) v = kStepPairOcc;
  }
  if (v != kStepOneSite && c->dims[0] % 2 != 0) v = kStepOneSite;
  return v;
}

// Reads and clears the device status word (after a synchronisation).
int check_status(flbm_ctx *c) {
  int h = 0;
  FLBM_CUDA(cudaMemcpy(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    FLBM_CUDA(cudaMemset(c->d_status, 0, sizeof(int)));
    return fail(FLBM_ETIMEOUT, "a bounded wait in the pipelined step kernel gave up; the state is not valid");
  }
  return FLBM_OK;
}

struct CkptHeader {
  char magic[8];
  int32_t version, lattice, storage, q;  // version 2 adds `model` (version 1: central moments)
  int64_t dims[3];
  int64_t step;
  uint64_t seed;
  double kBT, rho0;
  double lambda[27];
  uint64_t payload_bytes;
  int32_t model, pad;
};
const char kMagic[8] = {'F', 'L', 'B', 'M', 'C', 'K', 'P', '1'};

}  // namespace

extern "C" {

size_t flbm_required_bytes(int lattice, const int64_t dims[3], int storage) {
  const std::string saved = g_last_error;
  if (check_geometry(lattice, dims, storage) != FLBM_OK) return 0;
  g_last_error = saved;
  return size_t(q_of(lattice)) * size_t(dims[0] * dims[1] * dims[2]) * storage_bytes(storage);
}

int flbm_create_ex(flbm_ctx **out, int lattice, const int64_t dims[3], const double *lambda,
                   double kBT, double rho0, uint64_t seed, int storage, void *cuda_stream,
                   void *dev_buf, size_t dev_buf_bytes) {
  if (!out) return fail(FLBM_EINVAL, "out is NULL");
  int st = check_geometry(lattice, dims, storage);
  if (st != FLBM_OK) return st;
  st = check_params(lattice, lambda, kBT, rho0);
  if (st != FLBM_OK) return st;
  const size_t need = flbm_required_bytes(lattice, dims, storage);
  if (dev_buf) {
    if (dev_buf_bytes < need)
      return fail(FLBM_EINVAL, "dev_buf holds %zu bytes, %zu needed", dev_buf_bytes, need);
    if (reinterpret_cast<uintptr_t>(dev_buf) % 256 != 0)
      return fail(FLBM_EINVAL, "dev_buf must be 256-byte aligned");
  }
  int dev = 0;
  FLBM_CUDA(cudaGetDevice(&dev));

  flbm_ctx *c = new (std::nothrow) flbm_ctx();
  if (!c) return fail(FLBM_ENOMEM, "host allocation failed");
  c->lattice = lattice;
  c->D = d_of(lattice);
  c->Q = q_of(lattice);
  c->storage = storage;
  for (int a = 0; a < 3; ++a) c->dims[a] = dims[a];
  c->N = (long long)(dims[0] * dims[1] * dims[2]);
  for (int v = 0; v < c->Q; ++v) c->lambda[v] = (v <= c->D) ? 1.0 : lambda[v];
  c->kBT = kBT;
  c->rho0 = rho0;
  c->seed = seed;
  c->device = dev;
  c->f_bytes = need;

  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      release(c);
      return fail(FLBM_ECUDA, "cudaStreamCreateWithFlags: %s", cudaGetErrorString(e));
    }
    c->own_stream = true;
  }
  if (dev_buf) {
    c->f = dev_buf;
  } else {
    e = cudaMalloc(&c->f, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->f = nullptr;
      release(c);
      return fail(FLBM_ENOMEM, "cannot allocate %zu bytes of population memory", need);
    }
    c->own_f = true;
  }
  const size_t acc_bytes = sizeof(double) * stats_record_len(c->Q);
  e = cudaMalloc(&c->d_acc, acc_bytes);
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_acc, acc_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    release(c);
    return fail(FLBM_ENOMEM, "cannot allocate statistics buffers");
  }
  fill_args(c);
  if (const char *env = std::getenv("FLBM_STEP_VARIANT")) {
    const int v = std::atoi(env);
    if (v >= kStepAuto && v <= kStepVariantMax) c->variant = v;
  }
  // Rest state f = w rho0: every stored deviation is zero (also for BF16/FP16 bits).
  e = cudaMemsetAsync(c->f, 0, need, c->stream);
  if (e != cudaSuccess) {
    release(c);
    return fail(FLBM_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  }
  *out = c;
  return FLBM_OK;
}

int flbm_create(flbm_ctx **out, int lattice, const int64_t dims[3], const double *lambda,
                double kBT, double rho0, uint64_t seed) {
  return flbm_create_ex(out, lattice, dims, lambda, kBT, rho0, seed, FLBM_FP32, nullptr, nullptr, 0);
}

void flbm_destroy(flbm_ctx *ctx) {
  if (!ctx || ctx->owner || ctx->in_domain) return;
  DeviceGuard g(ctx->device);
  release(ctx);
}

int flbm_init_uniform(flbm_ctx *c, const double u0[3], double amp, uint64_t perturb_seed) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (!u0) return fail(FLBM_EINVAL, "u0 is NULL");
  for (int a = 0; a < c->D; ++a)
    if (!(std::fabs(u0[a]) < 1.0)) return fail(FLBM_EINVAL, "|u0[%d]| = %g must be < 1", a, u0[a]);
  if (!(amp >= 0.0 && amp < 1.0)) return fail(FLBM_EINVAL, "rho_perturb_amp = %g must lie in [0, 1)", amp);
  if (c->owner && c->step != 0)
    return fail(FLBM_ESTATE, "a lattice of a batch can be initialised only while the batch is at step 0");
  DeviceGuard g(c->device);
  FLBM_CUDA(launch_init(klat(c->lattice), c->storage, c->f, c->N, int(c->dims[0]), int(c->dims[1]),
                        int(c->dims[2]), c->rho0, u0[0], u0[1], c->D == 3 ? u0[2] : 0.0, amp,
                        perturb_seed, c->args.site_base, c->stream));
  c->step = 0;
  return FLBM_OK;
}

int flbm_step(flbm_ctx *c, int64_t n) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (c->owner) return fail(FLBM_ESTATE, "a lattice of a batch advances with flbm_batch_step");
  if (n < 0) return fail(FLBM_EINVAL, "n = %lld must be >= 0", (long long)n);
  if (c->slab && n > 1)
    return fail(FLBM_EINVAL, "a slab advances one step per flbm_step call (its halo is exchanged around every "
                             "step taken from an odd step count, see flbm_slab_halo)");
  DeviceGuard g(c->device);
  const bool noise = c->kBT > 0.0;
  for (int64_t s = 0; s < n; ++s) {
    c->args.step_lo = uint32_t(uint64_t(c->step));
    c->args.step_hi = uint32_t(uint64_t(c->step) >> 32);
    if (c->model == FLBM_COLLISION_RAW)
      FLBM_CUDA(launch_step_raw(c->D, c->storage, resolve_variant(c), int(c->step & 1), noise, c->args, c->stream));
    else
      FLBM_CUDA(launch_step(c->lattice, c->storage, resolve_variant(c), int(c->step & 1), noise, c->shear,
                            c->args, c->stream));
    ++c->step;
  }
  return FLBM_OK;
}

int64_t flbm_get_step(const flbm_ctx *c) { return c ? c->step : -1; }

int flbm_stats(flbm_ctx *c, flbm_stats_t *out) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (!out) return fail(FLBM_EINVAL, "out is NULL");
  DeviceGuard g(c->device);
  int st = enqueue_stats(c, c->d_acc);
  if (st != FLBM_OK) return st;
  FLBM_CUDA(cudaMemcpyAsync(c->h_acc, c->d_acc, sizeof(double) * stats_record_len(c->Q),
                            cudaMemcpyDeviceToHost, c->stream));
  FLBM_CUDA(cudaStreamSynchronize(c->stream));
  const int status = check_status(c);
  if (status != FLBM_OK) return status;
  fill_stats(c, c->h_acc, c->step, out);
  return stats_result(out, (long long)c->step);
}

int flbm_set_sample_capacity(flbm_ctx *c, int cap) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (cap < 1) return fail(FLBM_EINVAL, "capacity must be >= 1");
  DeviceGuard g(c->device);
  FLBM_CUDA(cudaStreamSynchronize(c->stream));
  if (c->d_ring) cudaFree(c->d_ring);
  c->d_ring = nullptr;
  c->ring_cap = c->ring_count = 0;
  c->ring_steps.clear();
  if (cudaMalloc(&c->d_ring, sizeof(double) * size_t(stats_record_len(c->Q)) * size_t(cap)) != cudaSuccess) {
    cudaGetLastError();
    c->d_ring = nullptr;
    return fail(FLBM_ENOMEM, "cannot allocate a sample buffer of %d records", cap);
  }
  c->ring_cap = cap;
  return FLBM_OK;
}

int flbm_sample_capacity(const flbm_ctx *c) { return c ? (c->d_ring ? c->ring_cap : 1024) : -1; }

int flbm_sample(flbm_ctx *c) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (!c->d_ring) {
    const int st = flbm_set_sample_capacity(c, 1024);
    if (st != FLBM_OK) return st;
  }
  if (c->ring_count >= c->ring_cap)
    return fail(FLBM_ESTATE, "sample buffer full (%d samples); fetch first", c->ring_cap);
  DeviceGuard g(c->device);
  double *slot = c->d_ring + size_t(c->ring_count) * size_t(stats_record_len(c->Q));
  const int st = enqueue_stats(c, slot);
  if (st != FLBM_OK) return st;
  c->ring_steps.push_back(c->step);
  ++c->ring_count;
  return FLBM_OK;
}

int flbm_fetch_samples(flbm_ctx *c, flbm_stats_t *out, int max_n, int *n_out) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (!n_out || (!out && max_n > 0) || max_n < 0) return fail(FLBM_EINVAL, "bad output arguments");
  DeviceGuard g(c->device);
  const int n = c->ring_count < max_n ? c->ring_count : max_n;
  const size_t len = size_t(stats_record_len(c->Q));
  std::vector<double> h(len * size_t(n > 0 ? n : 1));
  if (n > 0)
    FLBM_CUDA(cudaMemcpyAsync(h.data(), c->d_ring, sizeof(double) * len * size_t(n),
                              cudaMemcpyDeviceToHost, c->stream));
  FLBM_CUDA(cudaStreamSynchronize(c->stream));
  int64_t bad = 0;
  bool timeout = false;
  for (int k = 0; k < n; ++k) {
    fill_stats(c, h.data() + len * size_t(k), c->ring_steps[size_t(k)], &out[k]);
    if (out[k].nonfinite < 0)
      timeout = true;
    else
      bad += out[k].nonfinite;
  }
  c->ring_count = 0;
  c->ring_steps.clear();
  *n_out = n;
  if (timeout)
    return fail(FLBM_ETIMEOUT, "a bounded wait of the statistics reduction gave up; a fetched record is not valid");
  if (bad > 0) return fail(FLBM_ENUMERIC, "fetched samples count %lld non-finite sites", (long long)bad);
  return FLBM_OK;
}

int flbm_get_populations(flbm_ctx *c, double *host, size_t count) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (!host) return fail(FLBM_EINVAL, "host is NULL");
  if (count != size_t(c->Q) * size_t(c->N))
    return fail(FLBM_EINVAL, "count = %zu, expected Q * sites = %zu", count, size_t(c->Q) * size_t(c->N));
  DeviceGuard g(c->device);
  int st = ensure_stage(c, size_t(c->N));
  if (st != FLBM_OK) return st;
  for (int q = 0; q < c->Q; ++q) {
    FLBM_CUDA(launch_gather_plane(klat(c->lattice), c->storage, int(c->step & 1), c->f, c->N, int(c->dims[0]),
                                  int(c->dims[1]), int(c->dims[2]), c->rho0, q, c->d_stage, c->stream));
    FLBM_CUDA(cudaMemcpyAsync(host + size_t(q) * size_t(c->N), c->d_stage, sizeof(double) * size_t(c->N),
                              cudaMemcpyDeviceToHost, c->stream));
    FLBM_CUDA(cudaStreamSynchronize(c->stream));
  }
  return FLBM_OK;
}

int flbm_set_populations(flbm_ctx *c, const double *host, size_t count) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (!host) return fail(FLBM_EINVAL, "host is NULL");
  if (count != size_t(c->Q) * size_t(c->N))
    return fail(FLBM_EINVAL, "count = %zu, expected Q * sites = %zu", count, size_t(c->Q) * size_t(c->N));
  DeviceGuard g(c->device);
  int st = ensure_stage(c, size_t(c->N));
  if (st != FLBM_OK) return st;
  for (int q = 0; q < c->Q; ++q) {
    FLBM_CUDA(cudaMemcpyAsync(c->d_stage, host + size_t(q) * size_t(c->N), sizeof(double) * size_t(c->N),
                              cudaMemcpyHostToDevice, c->stream));
    FLBM_CUDA(launch_scatter_plane(klat(c->lattice), c->storage, int(c->step & 1), c->f, c->N, int(c->dims[0]),
                                   int(c->dims[1]), int(c->dims[2]), c->rho0, q, c->d_stage, c->stream));
  }
  FLBM_CUDA(cudaStreamSynchronize(c->stream));
  return FLBM_OK;
}

int flbm_get_sites(flbm_ctx *c, const int64_t *sites, size_t n, double *out) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (n == 0) return FLBM_OK;
  if (!sites || !out) return fail(FLBM_EINVAL, "sites or out is NULL");
  for (size_t k = 0; k < n; ++k)
    if (sites[k] < 0 || sites[k] >= c->N)
      return fail(FLBM_EINVAL, "sites[%zu] = %lld out of range [0, %lld)", k, (long long)sites[k], c->N);
  DeviceGuard g(c->device);
  if (c->sites_cap < n) {
    FLBM_CUDA(cudaStreamSynchronize(c->stream));
    if (c->d_sites) cudaFree(c->d_sites);
    c->d_sites = nullptr;
    c->sites_cap = 0;
    if (cudaMalloc(&c->d_sites, n * sizeof(long long)) != cudaSuccess) {
      cudaGetLastError();
      return fail(FLBM_ENOMEM, "cannot allocate the site list");
    }
    c->sites_cap = n;
  }
  int st = ensure_stage(c, n * size_t(c->Q));
  if (st != FLBM_OK) return st;
  static_assert(sizeof(long long) == sizeof(int64_t), "site index width");
  FLBM_CUDA(cudaMemcpyAsync(c->d_sites, sites, n * sizeof(long long), cudaMemcpyHostToDevice, c->stream));
  FLBM_CUDA(launch_gather_sites(klat(c->lattice), c->storage, int(c->step & 1), c->f, c->N, int(c->dims[0]),
                                int(c->dims[1]), int(c->dims[2]), c->rho0, c->d_sites, (long long)n,
                                c->d_stage, c->stream));
  FLBM_CUDA(cudaMemcpyAsync(out, c->d_stage, n * size_t(c->Q) * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
  FLBM_CUDA(cudaStreamSynchronize(c->stream));
  return FLBM_OK;
}

size_t flbm_checkpoint_bytes(const flbm_ctx *c) { return c ? sizeof(CkptHeader) + c->f_bytes : 0; }

int flbm_save(flbm_ctx *c, void *host, size_t bytes) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (!host) return fail(FLBM_EINVAL, "host is NULL");
  if (bytes < flbm_checkpoint_bytes(c))
    return fail(FLBM_EINVAL, "checkpoint needs %zu bytes, got %zu", flbm_checkpoint_bytes(c), bytes);
  DeviceGuard g(c->device);
  CkptHeader h{};
  std::memcpy(h.magic, kMagic, 8);
  h.version = 2;
  h.model = c->model;
  h.lattice = c->lattice;
  h.storage = c->storage;
  h.q = c->Q;
  for (int a = 0; a < 3; ++a) h.dims[a] = c->dims[a];
  h.step = c->step;
  h.seed = c->seed;
  h.kBT = c->kBT;
  h.rho0 = c->rho0;
  for (int v = 0; v < 27; ++v) h.lambda[v] = c->lambda[v];
  h.payload_bytes = c->f_bytes;
  std::memcpy(host, &h, sizeof(h));
  FLBM_CUDA(cudaMemcpyAsync(static_cast<char *>(host) + sizeof(h), c->f, c->f_bytes,
                            cudaMemcpyDeviceToHost, c->stream));
  FLBM_CUDA(cudaStreamSynchronize(c->stream));
  return FLBM_OK;
}

int flbm_load(flbm_ctx *c, const void *host, size_t bytes) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (!host) return fail(FLBM_EINVAL, "host is NULL");
  // Version 1 headers end before `model`.
  constexpr size_t kHeaderV1 = offsetof(CkptHeader, model);
  if (bytes < kHeaderV1) return fail(FLBM_EINVAL, "blob too small for a checkpoint header");
  CkptHeader h{};
  std::memcpy(&h, host, kHeaderV1);
  const size_t hbytes = h.version == 1 ? kHeaderV1 : sizeof(CkptHeader);
  if (h.version == 2 && bytes >= sizeof(CkptHeader)) std::memcpy(&h, host, sizeof(h));
  if (std::memcmp(h.magic, kMagic, 8) != 0 || (h.version != 1 && h.version != 2))
    return fail(FLBM_EINVAL, "not a checkpoint blob");
  if (h.version == 1) h.model = FLBM_COLLISION_CM;
  if (h.model != FLBM_COLLISION_CM && (h.model != FLBM_COLLISION_RAW || c->owner))
    return fail(FLBM_EINVAL, "checkpoint collision model %d is not available for this context", h.model);
  if (h.lattice != c->lattice || h.storage != c->storage || h.dims[0] != c->dims[0] ||
      h.dims[1] != c->dims[1] || h.dims[2] != c->dims[2] || h.payload_bytes != c->f_bytes)
    return fail(FLBM_EINVAL, "checkpoint lattice, dims or storage differ from the context");
  if (bytes < hbytes + h.payload_bytes) return fail(FLBM_EINVAL, "checkpoint blob truncated");
  const int st = check_params(h.lattice, h.lambda, h.kBT, h.rho0);
  if (st != FLBM_OK) return st;
  if (c->owner && h.step != c->step)
    return fail(FLBM_ESTATE, "checkpoint of step %lld, the batch is at step %lld", (long long)h.step,
                (long long)c->step);
  DeviceGuard g(c->device);
  FLBM_CUDA(cudaMemcpyAsync(c->f, static_cast<const char *>(host) + hbytes, c->f_bytes,
                            cudaMemcpyHostToDevice, c->stream));
  FLBM_CUDA(cudaStreamSynchronize(c->stream));
  c->step = h.step;
  c->seed = h.seed;
  c->kBT = h.kBT;
  c->rho0 = h.rho0;
  c->model = h.model;
  for (int v = 0; v < c->Q; ++v) c->lambda[v] = (v <= c->D) ? 1.0 : h.lambda[v];
  fill_args(c);
  c->params_changed = true;
  return FLBM_OK;
}

int flbm_set_step_variant(flbm_ctx *c, int variant) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (c->owner) return fail(FLBM_ESTATE, "a lattice of a batch has no step variant of its own");
  if (variant < kStepAuto || variant > kStepVariantMax)
    return fail(FLBM_EINVAL, "variant %d is not one of 0..%d", variant, int(kStepVariantMax));
  c->variant = variant;
  return FLBM_OK;
}

int flbm_get_step_variant(const flbm_ctx *c) { return c ? resolve_variant(c) : -1; }

int flbm_set_collision(flbm_ctx *c, int model) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (model != FLBM_COLLISION_CM && model != FLBM_COLLISION_RAW)
    return fail(FLBM_EINVAL, "collision model %d is not FLBM_COLLISION_CM (0) or FLBM_COLLISION_RAW (1)", model);
  if (c->owner) return fail(FLBM_ESTATE, "the lattices of a batch use the central-moment collision");
  if (model == FLBM_COLLISION_RAW && c->lattice != FLBM_D2Q9 && c->lattice != FLBM_D3Q27)
    return fail(FLBM_EINVAL, "the raw-moment collision is available for FLBM_D2Q9 and FLBM_D3Q27 only");
  c->model = model;
  return FLBM_OK;
}

int flbm_get_collision(const flbm_ctx *c) { return c ? c->model : -1; }

int flbm_autotune(flbm_ctx *c, int trial_steps, int *chosen) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  if (c->owner) return fail(FLBM_ESTATE, "a lattice of a batch is tuned with flbm_batch_autotune");
  if (c->slab) return fail(FLBM_ESTATE, "a slab is not tuned alone (its steps need halo exchanges)");
  if (trial_steps < 2) return fail(FLBM_EINVAL, "trial_steps must be >= 2");
  DeviceGuard g(c->device);
  // Cache: one choice per (device, lattice, storage, nx parity, size class, noise, rate
  // structure, collision model, rows shorter than one block).
  cudaDeviceProp prop;
  FLBM_CUDA(cudaGetDeviceProperties(&prop, c->device));
  int size_class = 0;
  for (long long n = c->N; n > 1; n >>= 1) ++size_class;
  char key[320];
  std::snprintf(key, sizeof(key), "%s|%d|%d|%d|%d|%d|%d|%d|%d", prop.name, c->lattice, c->storage,
                int(c->dims[0] % 2), size_class, c->kBT > 0.0 ? 1 : 0, c->shear ? 1 : 0, c->model,
                c->dims[0] < 2 * kStepBlock ? 1 : 0);
  static std::mutex mu;
  static std::map<std::string, int> cache;
  static bool file_read = false;
  const char *cache_file = std::getenv("FLBM_AUTOTUNE_CACHE");
  {
    std::lock_guard<std::mutex> lock(mu);
    if (cache_file && *cache_file && !file_read) {
      // One "key<TAB>variant" line per choice; malformed lines are skipped.
      file_read = true;
      if (FILE *fh = std::fopen(cache_file, "r")) {
        char line[512];
        while (std::fgets(line, sizeof(line), fh)) {
          char *tab = std::strchr(line, '\t');
          if (!tab) continue;
          *tab = '\0';
          const int v = std::atoi(tab + 1);
          if (v >= kStepOneSite && v <= kStepVariantMax) cache[line] = v;
        }
        std::fclose(fh);
      }
    }
    auto it = cache.find(key);
    if (it != cache.end()) {
      c->variant = it->second;
      if (chosen) *chosen = it->second;
      return FLBM_OK;
    }
  }
  // Trial steps run on a copy of the state, which is restored afterwards; the step
  // counter is left unchanged, so tuning does not alter the simulation.
  void *backup = nullptr;
  if (cudaMalloc(&backup, c->f_bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(FLBM_ENOMEM, "cannot allocate %zu bytes for the autotuner's state copy", c->f_bytes);
  }
  int st = FLBM_OK;
  float best = 1e30f;
  int best_v = resolve_variant(c);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int64_t step0 = c->step;
  const int saved_variant = c->variant;
  do {
    if (cudaMemcpyAsync(backup, c->f, c->f_bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      st = fail(FLBM_ECUDA, "autotune set-up: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    const int candidates[8] = {kStepOneSite, kStepPair,    kStepPairRolled,  kStepPipelined,
                               kStepPairOcc, kStepPairRolledOcc, kStepPairOccRows, kStepPairRows};
    for (int v : candidates) {
      if (pair_variants_only(c->lattice) &&
          (v == kStepPairRolled || v == kStepPipelined || v == kStepPairRolledOcc))
        continue;
      // Blocks of four rows only where a row is shorter than a one-row block's 256 sites.
      if ((v == kStepPairOccRows || v == kStepPairRows) && c->dims[0] >= 2 * kStepBlock) continue;
      if (v != kStepOneSite && c->dims[0] % 2 != 0) continue;
      if (v == kStepPipelined && !pipe_applicable(c->D, c->storage, int(c->dims[0]))) continue;
      c->variant = v;
      if ((st = flbm_step(c, 2)) != FLBM_OK) break;  // warm-up (both parities)
      cudaEventRecord(e0, c->stream);
      if ((st = flbm_step(c, trial_steps)) != FLBM_OK) break;
      cudaEventRecord(e1, c->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = fail(FLBM_ECUDA, "autotune timing failed");
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_v = v;
      }
      c->step = step0;
      if (cudaMemcpyAsync(c->f, backup, c->f_bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
        st = fail(FLBM_ECUDA, "autotune restore failed");
        break;
      }
    }
  } while (false);
  cudaStreamSynchronize(c->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(backup);
  c->step = step0;
  if (st != FLBM_OK) {
    c->variant = saved_variant;
    return st;
  }
  c->variant = best_v;
  {
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = best_v;
    if (cache_file && *cache_file)
      if (FILE *fh = std::fopen(cache_file, "a")) {
        std::fprintf(fh, "%s\t%d\n", key, best_v);
        std::fclose(fh);
      }
  }
  if (chosen) *chosen = best_v;
  return FLBM_OK;
}

int flbm_sync(flbm_ctx *c) {
  if (!c) return fail(FLBM_EINVAL, "ctx is NULL");
  DeviceGuard g(c->device);
  FLBM_CUDA(cudaStreamSynchronize(c->stream));
  return check_status(c);
}

const char *flbm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ---- batched ensembles -------------------------------------------------------------------
// The batch owns one population allocation cut into its lattices' arrays (256-byte
// aligned), one context per lattice (borrowed by the caller through flbm_batch_lattice,
// sharing the batch's stream), the tile table and general-rate table of the persistent
// kernel (batch.cu), its step counter, barrier words and status word.
struct flbm_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void *pool = nullptr;
  size_t pool_bytes = 0;
  std::vector<flbm_ctx *> members;
  std::vector<int> order;  // kernel table entry -> member (D3Q27 lattices first)
  BatchGroup g3{}, g2{};   // the two lattice types' table entries and tiles
  bool shear = true;       // every lattice follows the paper's rate structure
  int threads = 128;       // block size of the D3Q27 lattices (all in the persistent form)
  int form = kBatchStep;    // enum BatchForm: per-step launches or one persistent launch
  int threads2 = 128;      // the D2Q9 lattices' block size and per-step form (the
  int form2 = kBatchStep;  // persistent form launches every type alike)
  int grid = 0;            // co-resident blocks (cooperative launch)
  int tiles_for = 0, tiles_for2 = 0;  // block sizes the tiling was built for
  int ntiles = 0;
  float *d_rates = nullptr;  // om[27], phc[27] per lattice
  long long *d_step = nullptr;
  int *d_done = nullptr;           // per lattice: tiles finished in the running launch
  unsigned int *d_exits = nullptr;  // blocks that have left the running launch
  int *d_status = nullptr;
  int64_t step = 0;
  BatchArgs *args = nullptr;  // by-value kernel arguments (large: heap)
  bool graphs_ok = true;      // capture worked (or was not tried yet)
  uint32_t test_wait_polls = 0;  // armed by flbm_batch_test_wait_timeout for one launch
  bool last_graph = false;
  std::map<int64_t, cudaGraphExec_t> graphs;  // per (n, form, start parity), current shape
};

namespace {

constexpr int kBatchDefaultThreads = 128;

void batch_drop_graphs(flbm_batch *b) {
  for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
}

void batch_release(flbm_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop_graphs(b);
  for (flbm_ctx *c : b->members) {
    c->owner = nullptr;
    release(c);
  }
  if (b->pool) cudaFree(b->pool);
  if (b->d_rates) cudaFree(b->d_rates);
  if (b->d_step) cudaFree(b->d_step);
  if (b->d_done) cudaFree(b->d_done);
  if (b->d_exits) cudaFree(b->d_exits);
  if (b->d_status) cudaFree(b->d_status);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b->args;
  delete b;
}

// Kernel arguments from the lattices' contexts: geometry, keys, the paper-structure
// triple (sqrt kBT, 1 - L_shear, phc_shear) and the general-rate table.
int batch_params(flbm_batch *b) {
  const int n = int(b->members.size());
  std::vector<float> rates(size_t(n) * 54, 0.0f);
  b->shear = true;
  for (int i = 0; i < n; ++i) {
    flbm_ctx *c = b->members[size_t(b->order[size_t(i)])];
    const StepArgs &a = c->args;
    BatchLattice &L = b->args->lats[i];
    L.f256 = uint32_t((static_cast<char *>(c->f) - static_cast<char *>(b->pool)) / 256);
    L.plane = uint32_t(c->N);
    L.nx = a.nx;
    L.ny = a.ny;
    L.nz = a.nz;
    uint32_t m = 0;
    int p_hp = 0, p_ny = 0;
    batch_magic(uint32_t((a.nx + 1) / 2), &L.m_hp, &p_hp);
    batch_magic(uint32_t(a.ny), &m, &p_ny);
    L.m_ny = m;
    L.dpp = uint32_t(c->D) | (uint32_t(p_hp) << 8) | (uint32_t(p_ny) << 16);
    L.rho0 = a.rho0;
    L.key0 = a.key0;
    L.key1 = a.key1;
    const int ref = c->D == 3 ? 7 : 5;  // a shear mode with b = 1/9
    L.sqrt_kbt = float(std::sqrt(c->kBT));
    L.om_shear = a.om[ref];
    L.phc_shear = a.phc[ref];
    for (int v = 0; v < 27; ++v) {
      rates[size_t(i) * 54 + size_t(v)] = a.om_t[v];  // the collision's (tile-scaled) constants
      rates[size_t(i) * 54 + 27 + size_t(v)] = a.phc_t[v];
    }
    // The shear form needs the paper's structure and one rate shared by the shear modes.
    bool ok = c->shear;
    if (c->D == 3)
      ok = ok && a.om[8] == a.om[7] && a.om[9] == a.om[7] && a.phc[8] == a.phc[7] && a.phc[9] == a.phc[7];
    else
      ok = ok && a.om[4] == a.om[5] && a.phc[4] == 2.0f * a.phc[5];
    if (!ok) b->shear = false;
    c->params_changed = false;
  }
  FLBM_CUDA(cudaMemcpyAsync(b->d_rates, rates.data(), rates.size() * sizeof(float), cudaMemcpyHostToDevice,
                            b->stream));
  FLBM_CUDA(cudaStreamSynchronize(b->stream));  // `rates` is a local
  return FLBM_OK;
}

// The D2Q9 lattices' block size and form as launched: their own in the per-step forms,
// the batch's in the persistent one.
int batch_threads2(const flbm_batch *b) { return b->form == kBatchPersistent ? b->threads : b->threads2; }
int batch_form2(const flbm_batch *b) { return b->form == kBatchPersistent ? b->form : b->form2; }

// Tiling for the block sizes (tiles of `threads` pair slots, never spanning lattices; a
// row of nx sites holds ceil(nx / 2) slots; lattice i owns tiles [tile0_i, tile0_{i+1}))
// and the grid of co-resident blocks.
int batch_shape(flbm_batch *b) {
  if (b->tiles_for == b->threads && b->tiles_for2 == batch_threads2(b)) return FLBM_OK;
  long long total = 0;
  const int nl = int(b->members.size());
  int n3 = 0;  // table entries 0 .. n3-1 are the D3Q27 lattices
  while (n3 < nl && b->members[size_t(b->order[size_t(n3)])]->D == 3) ++n3;
  long long tiles3 = 0;
  for (int i = 0; i < nl; ++i) {
    if (i == n3) tiles3 = total;
    b->args->lats[i].tile0 = int(total);
    const flbm_ctx *m = b->members[size_t(b->order[size_t(i)])];
    const long long slots = (m->dims[0] + 1) / 2 * m->dims[1] * m->dims[2];
    const long long per_tile = m->D == 3 ? b->threads : batch_threads2(b);
    total += (slots + per_tile - 1) / per_tile;
    if (total > 0x3fffffffLL) return fail(FLBM_EINVAL, "too many tiles");
  }
  if (n3 == nl) tiles3 = total;
  b->g3 = BatchGroup{0, n3, 0, int(tiles3)};
  b->g2 = BatchGroup{n3, nl, int(tiles3), int(total - tiles3)};
  FLBM_CUDA(cudaStreamSynchronize(b->stream));
  batch_drop_graphs(b);
  b->tiles_for = 0;
  b->ntiles = int(total);
  int per_sm = 0, sms = 0;
  FLBM_CUDA(batch_max_blocks(b->shear, b->threads, &per_sm));
  FLBM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  if (per_sm < 1) return fail(FLBM_ECUDA, "the batch kernel cannot be resident with %d threads", b->threads);
  const long long g = (long long)per_sm * sms;
  b->grid = int(g < b->ntiles ? g : b->ntiles);
  b->tiles_for = b->threads;
  b->tiles_for2 = batch_threads2(b);
  return FLBM_OK;
}

// Enqueue n steps: the persistent form resets the completion counters and makes one
// cooperative launch; the per-step form makes n plain launches and a counter update.
int batch_enqueue(flbm_batch *b, int64_t n) {
  b->args->rates = b->d_rates;
  b->args->pool = static_cast<char *>(b->pool);
  b->args->nlat = int(b->members.size());
  b->args->ntiles = b->ntiles;
  b->args->tile_slots[1] = b->threads;
  b->args->tile_slots[0] = batch_threads2(b);
  b->args->nsteps = int(n);
  b->args->step_counter = b->d_step;
  b->args->done = b->d_done;
  b->args->exits = b->d_exits;
  b->args->status = b->d_status;
  b->args->target_bias = b->test_wait_polls ? (1 << 30) : 0;
  b->args->wait_polls = b->test_wait_polls ? b->test_wait_polls : kBatchWaitPolls;
  if (b->form != kBatchPersistent) {
    FLBM_CUDA(launch_batch_steps(b->form, b->threads, batch_form2(b), batch_threads2(b), b->shear, int(b->step & 1),
                                 *b->args, b->g3, b->g2, int(n), b->stream));
    return FLBM_OK;
  }
  FLBM_CUDA(cudaMemsetAsync(b->d_done, 0, b->members.size() * sizeof(int), b->stream));
  FLBM_CUDA(cudaMemsetAsync(b->d_exits, 0, sizeof(unsigned int), b->stream));
  FLBM_CUDA(launch_batch(b->shear, *b->args, b->grid, b->threads, b->stream));
  return FLBM_OK;
}

// The captured graph of n steps in the current form, or nullptr where capture is
// unavailable.
cudaGraphExec_t batch_graph(flbm_batch *b, int64_t n) {
  if (!b->graphs_ok) return nullptr;
  const int64_t key = n * 2 + (b->form == kBatchPersistent ? 0 : int64_t(b->step & 1));
  auto it = b->graphs.find(key);
  if (it != b->graphs.end()) return it->second;
  if (b->graphs.size() >= 16) batch_drop_graphs(b);
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    b->graphs_ok = false;
    return nullptr;
  }
  const int st = batch_enqueue(b, n);
  const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (st == FLBM_OK && e == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess) {
    cudaGraphDestroy(g);
    b->graphs[key] = exec;
    return exec;
  }
  cudaGetLastError();
  if (g) cudaGraphDestroy(g);
  b->graphs_ok = false;
  return nullptr;
}

}  // namespace

extern "C" {

int flbm_batch_create(flbm_batch **out, const flbm_lattice_spec *specs, int n, void *cuda_stream) {
  if (!out) return fail(FLBM_EINVAL, "out is NULL");
  if (!specs) return fail(FLBM_EINVAL, "specs is NULL");
  if (n < 1 || n > kBatchMaxLattices)
    return fail(FLBM_EINVAL, "n = %d must lie in [1, %d]", n, int(kBatchMaxLattices));
  static_assert(FLBM_BATCH_MAX_LATTICES == kBatchMaxLattices, "header and kernel bounds differ");
  std::vector<size_t> offset(static_cast<size_t>(n), 0);
  size_t total = 0;
  for (int i = 0; i < n; ++i) {
    const flbm_lattice_spec &s = specs[i];
    if (s.reserved != 0) return fail(FLBM_EINVAL, "specs[%d].reserved must be 0", i);
    if (s.lattice == FLBM_D3Q27_ISO || s.lattice == FLBM_D3Q19)
      return fail(FLBM_EINVAL, "specs[%d]: only FLBM_D2Q9 and FLBM_D3Q27 lattices are available in batches", i);
    int st = check_geometry(s.lattice, s.dims, FLBM_FP32);
    if (st == FLBM_OK) st = check_params(s.lattice, s.lambda, s.kBT, s.rho0);
    if (st != FLBM_OK) return fail(st, "specs[%d]: %s", i, g_last_error.c_str());
    offset[size_t(i)] = total;
    total += (flbm_required_bytes(s.lattice, s.dims, FLBM_FP32) + 255) / 256 * 256;
  }
  int dev = 0;
  FLBM_CUDA(cudaGetDevice(&dev));
  int coop = 0;
  FLBM_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return fail(FLBM_ECUDA, "device %d does not support cooperative launches", dev);

  flbm_batch *b = new (std::nothrow) flbm_batch();
  if (!b) return fail(FLBM_ENOMEM, "host allocation failed");
  b->args = new (std::nothrow) BatchArgs();
  if (!b->args) {
    delete b;
    return fail(FLBM_ENOMEM, "host allocation failed");
  }
  b->device = dev;
  b->threads = kBatchDefaultThreads;
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      batch_release(b);
      return fail(FLBM_ECUDA, "cudaStreamCreateWithFlags: %s", cudaGetErrorString(e));
    }
    b->own_stream = true;
  }
  e = cudaMalloc(&b->pool, total);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_rates, size_t(n) * 54 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_step, sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_done, size_t(n) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_exits, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_release(b);
    return fail(FLBM_ENOMEM, "cannot allocate %zu bytes of batch memory", total);
  }
  b->pool_bytes = total;
  if (cudaMemsetAsync(b->d_step, 0, sizeof(long long), b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_done, 0, size_t(n) * sizeof(int), b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_exits, 0, sizeof(unsigned int), b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream) != cudaSuccess) {
    batch_release(b);
    return fail(FLBM_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(cudaGetLastError()));
  }
  for (int i = 0; i < n; ++i) {
    const flbm_lattice_spec &s = specs[i];
    flbm_ctx *c = nullptr;
    const size_t need = flbm_required_bytes(s.lattice, s.dims, FLBM_FP32);
    const int st = flbm_create_ex(&c, s.lattice, s.dims, s.lambda, s.kBT, s.rho0, s.seed, FLBM_FP32, b->stream,
                                  static_cast<char *>(b->pool) + offset[size_t(i)], need);
    if (st != FLBM_OK) {
      const std::string msg = g_last_error;
      batch_release(b);
      return fail(st, "lattice %d: %s", i, msg.c_str());
    }
    c->owner = b;
    c->variant = kStepPair;
    b->members.push_back(c);
  }
  for (int i = 0; i < n; ++i)
    if (b->members[size_t(i)]->D == 3) b->order.push_back(i);
  for (int i = 0; i < n; ++i)
    if (b->members[size_t(i)]->D == 2) b->order.push_back(i);
  int st = batch_params(b);
  if (st == FLBM_OK) st = batch_shape(b);
  if (st != FLBM_OK) {
    const std::string msg = g_last_error;
    batch_release(b);
    return fail(st, "%s", msg.c_str());
  }
  *out = b;
  return FLBM_OK;
}

void flbm_batch_destroy(flbm_batch *b) {
  if (!b) return;
  DeviceGuard g(b->device);
  batch_release(b);
}

int flbm_batch_size(const flbm_batch *b) { return b ? int(b->members.size()) : -1; }

flbm_ctx *flbm_batch_lattice(flbm_batch *b, int i) {
  if (!b || i < 0 || i >= int(b->members.size())) {
    fail(FLBM_EINVAL, "no lattice %d in this batch", i);
    return nullptr;
  }
  return b->members[size_t(i)];
}

int flbm_batch_stats(flbm_batch *b, int i, flbm_stats_t *out) {
  if (!b) return fail(FLBM_EINVAL, "batch is NULL");
  if (i < 0 || i >= int(b->members.size()))
    return fail(FLBM_EINVAL, "no lattice %d in this batch of %d", i, int(b->members.size()));
  if (!out) return fail(FLBM_EINVAL, "out is NULL");
  return flbm_stats(b->members[size_t(i)], out);
}

int flbm_batch_step(flbm_batch *b, int64_t n) {
  if (!b) return fail(FLBM_EINVAL, "batch is NULL");
  if (n < 0 || n > 0x7fffffff) return fail(FLBM_EINVAL, "n = %lld must lie in [0, 2^31)", (long long)n);
  if (n == 0) return FLBM_OK;
  DeviceGuard g(b->device);
  bool changed = false;
  for (flbm_ctx *c : b->members) changed = changed || c->params_changed;
  if (changed) {
    int st = batch_params(b);
    if (st != FLBM_OK) return st;
    batch_drop_graphs(b);
    b->tiles_for = b->tiles_for2 = 0;  // the kernel form (shear) may have changed: new grid
  }
  int st = batch_shape(b);
  if (st != FLBM_OK) return st;
  // An armed test hook changes the kernel arguments of this one launch: no graph.
  cudaGraphExec_t exec = b->test_wait_polls ? nullptr : batch_graph(b, n);
  b->last_graph = exec != nullptr;
  if (exec) {
    FLBM_CUDA(cudaGraphLaunch(exec, b->stream));
  } else {
    st = batch_enqueue(b, n);
    if (st != FLBM_OK) return st;
  }
  b->test_wait_polls = 0;
  b->step += n;
  for (flbm_ctx *c : b->members) c->step = b->step;
  return FLBM_OK;
}

int64_t flbm_batch_get_step(const flbm_batch *b) { return b ? b->step : -1; }

int flbm_batch_set_shape(flbm_batch *b, int threads, int form) {
  if (!b) return fail(FLBM_EINVAL, "batch is NULL");
  if (threads == 0) threads = kBatchDefaultThreads;
  if (threads != 64 && threads != 128 && threads != 256)
    return fail(FLBM_EINVAL, "threads = %d must be 64, 128 or 256 (or 0)", threads);
  if (form < 0 || form > kBatchFormMax) return fail(FLBM_EINVAL, "form = %d is not one of 0..%d", form, int(kBatchFormMax));
  if (form == kBatchStepOcc && threads > 128)
    return fail(FLBM_EINVAL, "form 2 (five blocks per SM) takes at most 128 threads per block");
  if (threads != b->threads || form != b->form || threads != b->threads2 || form != b->form2) batch_drop_graphs(b);
  b->threads = b->threads2 = threads;
  b->form = b->form2 = form;
  return FLBM_OK;
}

int flbm_batch_get_shape(const flbm_batch *b, int *threads, int *form) {
  if (!b) return fail(FLBM_EINVAL, "batch is NULL");
  if (threads) *threads = b->threads;
  if (form) *form = b->form;
  return FLBM_OK;
}

int flbm_batch_set_type_shape(flbm_batch *b, int lattice, int threads, int form) {
  if (!b) return fail(FLBM_EINVAL, "batch is NULL");
  if (lattice != FLBM_D2Q9 && lattice != FLBM_D3Q27)
    return fail(FLBM_EINVAL, "lattice %d is not FLBM_D2Q9 (0) or FLBM_D3Q27 (1)", lattice);
  if (b->form == kBatchPersistent)
    return fail(FLBM_ESTATE, "the persistent form launches every lattice type alike (use flbm_batch_set_shape)");
  if (threads == 0) threads = kBatchDefaultThreads;
  if (threads != 64 && threads != 128 && threads != 256)
    return fail(FLBM_EINVAL, "threads = %d must be 64, 128 or 256 (or 0)", threads);
  if (form < 0 || form > kBatchFormMax || form == kBatchPersistent)
    return fail(FLBM_EINVAL, "form = %d is not a per-step form (0, 2 or 3)", form);
  if (form == kBatchStepOcc && threads > 128)
    return fail(FLBM_EINVAL, "form 2 (five blocks per SM) takes at most 128 threads per block");
  int &t = lattice == FLBM_D3Q27 ? b->threads : b->threads2;
  int &f = lattice == FLBM_D3Q27 ? b->form : b->form2;
  if (threads != t || form != f) batch_drop_graphs(b);
  t = threads;
  f = form;
  return FLBM_OK;
}

int flbm_batch_get_type_shape(const flbm_batch *b, int lattice, int *threads, int *form) {
  if (!b) return fail(FLBM_EINVAL, "batch is NULL");
  if (lattice != FLBM_D2Q9 && lattice != FLBM_D3Q27)
    return fail(FLBM_EINVAL, "lattice %d is not FLBM_D2Q9 (0) or FLBM_D3Q27 (1)", lattice);
  if (threads) *threads = lattice == FLBM_D3Q27 ? b->threads : batch_threads2(b);
  if (form) *form = lattice == FLBM_D3Q27 ? b->form : batch_form2(b);
  return FLBM_OK;
}

int flbm_batch_uses_graph(const flbm_batch *b) { return b ? (b->last_graph ? 1 : 0) : -1; }

int flbm_batch_sync(flbm_batch *b) {
  if (!b) return fail(FLBM_EINVAL, "batch is NULL");
  DeviceGuard g(b->device);
  FLBM_CUDA(cudaStreamSynchronize(b->stream));
  int h = 0;
  FLBM_CUDA(cudaMemcpy(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    // The failed launch did not advance the device step counter: take it as the step
    // count, so that the batch stays usable (re-initialise or load checkpoints).
    long long dev_step = 0;
    FLBM_CUDA(cudaMemcpy(&dev_step, b->d_step, sizeof(long long), cudaMemcpyDeviceToHost));
    FLBM_CUDA(cudaMemset(b->d_status, 0, sizeof(int)));
    b->step = dev_step;
    for (flbm_ctx *c : b->members) c->step = dev_step;
    return fail(FLBM_ETIMEOUT, "a bounded wait of the batch kernel gave up; the populations are not valid "
                               "(step count reset to %lld)", dev_step);
  }
  return FLBM_OK;
}

int flbm_batch_test_wait_timeout(flbm_batch *b, uint32_t polls) {
  if (!b) return fail(FLBM_EINVAL, "batch is NULL");
  if (polls == 0) return fail(FLBM_EINVAL, "polls must be >= 1");
  b->test_wait_polls = polls;
  return FLBM_OK;
}

int flbm_batch_autotune(flbm_batch *b, int trial_steps, int *threads_out, int *form_out) {
  if (!b) return fail(FLBM_EINVAL, "batch is NULL");
  if (trial_steps < 2) return fail(FLBM_EINVAL, "trial_steps must be >= 2");
  DeviceGuard g(b->device);
  void *backup = nullptr;
  if (cudaMalloc(&backup, b->pool_bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(FLBM_ENOMEM, "cannot allocate %zu bytes for the autotuner's state copy", b->pool_bytes);
  }
  const int64_t step0 = b->step;
  const long long step0_dev = (long long)step0;
  const int saved_t = b->threads, saved_f = b->form, saved_t2 = b->threads2, saved_f2 = b->form2;
  int best_t = saved_t, best_f = saved_f, best_t2 = saved_t2, best_f2 = saved_f2, st = FLBM_OK;
  float best = 1e30f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // warm-up and capture of the timed shape (an even count keeps the start parity of the
  // timed call, so that it replays the captured graph)
  const int64_t nt = trial_steps + (trial_steps & 1);
  do {
    if (cudaMemcpyAsync(backup, b->pool, b->pool_bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      st = fail(FLBM_ECUDA, "autotune set-up: %s", cudaGetErrorString(cudaGetLastError()));
      break;
    }
    // One trial: the shape (t3, f3) for the D3Q27 lattices (and every lattice in the
    // persistent form) and (t2, f2) for the D2Q9 lattices, timed on the state copy.
    auto trial = [&](int t3, int f3, int t2, int f2, float *ms) -> int {
      b->threads = t3;
      b->form = f3;
      b->threads2 = t2;
      b->form2 = f2;
      batch_drop_graphs(b);
      int r = flbm_batch_step(b, 2);
      if (r == FLBM_OK) r = flbm_batch_step(b, nt);
      if (r == FLBM_OK) {
        cudaEventRecord(e0, b->stream);
        r = flbm_batch_step(b, nt);
      }
      if (r == FLBM_OK) {
        cudaEventRecord(e1, b->stream);
        r = flbm_batch_sync(b);
      }
      if (r != FLBM_OK) return r;
      cudaEventElapsedTime(ms, e0, e1);
      b->step = step0;
      for (flbm_ctx *c : b->members) c->step = step0;
      if (cudaMemcpyAsync(b->pool, backup, b->pool_bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
          cudaMemcpyAsync(b->d_step, &step0_dev, sizeof(long long), cudaMemcpyHostToDevice, b->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(b->stream) != cudaSuccess)
        return fail(FLBM_ECUDA, "autotune restore failed");
      return FLBM_OK;
    };
    // Every lattice alike, then, in a per-step form, the D2Q9 lattices' own shape.
    for (int f = 0; f <= kBatchFormMax && st == FLBM_OK; ++f) {
      for (int t : {64, 128, 256}) {
        if (f == kBatchStepOcc && t > 128) continue;
        float ms = 0.0f;
        if ((st = trial(t, f, t, f, &ms)) != FLBM_OK) break;
        if (ms < best) {
          best = ms;
          best_t = best_t2 = t;
          best_f = best_f2 = f;
        }
      }
    }
    if (st == FLBM_OK && best_f != kBatchPersistent && b->g2.ntiles > 0 && b->g3.ntiles > 0) {
      const int t3 = best_t, f3 = best_f;
      for (int f : {int(kBatchStep), int(kBatchStepOcc), int(kBatchStepRolled)}) {
        for (int t : {64, 128, 256}) {
          if ((f == kBatchStepOcc && t > 128) || (t == t3 && f == f3)) continue;
          float ms = 0.0f;
          if ((st = trial(t3, f3, t, f, &ms)) != FLBM_OK) break;
          if (ms < best) {
            best = ms;
            best_t2 = t;
            best_f2 = f;
          }
        }
        if (st != FLBM_OK) break;
      }
    }
  } while (false);
  cudaStreamSynchronize(b->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(backup);
  b->step = step0;
  for (flbm_ctx *c : b->members) c->step = step0;
  batch_drop_graphs(b);
  if (st != FLBM_OK) {
    b->threads = saved_t;
    b->form = saved_f;
    b->threads2 = saved_t2;
    b->form2 = saved_f2;
    return st;
  }
  b->threads = best_t;
  b->form = best_f;
  b->threads2 = best_t2;
  b->form2 = best_f2;
  if (threads_out) *threads_out = best_t;
  if (form_out) *form_out = best_f;
  return FLBM_OK;
}

}  // extern "C"

// ---- statistics without allocation -----------------------------------------------------
// Scratch of flbm_stats_noalloc: the accumulators of the statistics kernel in a fixed
// device array, so that the call needs no cudaMalloc. Host code may not use the array's
// name as an address; its device address is looked up once per device.
namespace {

static __device__ __align__(256) double g_noalloc_scratch[FLBM_NOALLOC_SCRATCH_DOUBLES];

constexpr int kNoallocMaxDevices = 64;
double *g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of the scratch on the current device (first use: symbol lookup).
int noalloc_scratch(double **out) {
  int dev = 0;
  FLBM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices)
    return fail(FLBM_EINVAL, "device %d beyond the %d devices flbm_stats_noalloc supports", dev,
                kNoallocMaxDevices);
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(FLBM_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return FLBM_OK;
}

}  // namespace

extern "C" int flbm_stats_noalloc(int lattice, const int64_t dims[3], int storage, int parity,
                                  double rho0, const void *dev_populations, void *cuda_stream,
                                  flbm_stats_t *out) {
  int st = check_geometry(lattice, dims, storage);
  if (st != FLBM_OK) return st;
  if (parity != 0 && parity != 1) return fail(FLBM_EINVAL, "parity must be 0 or 1, got %d", parity);
  if (!(rho0 > 0.0) || !std::isfinite(rho0)) return fail(FLBM_EINVAL, "rho0 = %g must be finite and > 0", rho0);
  if (!dev_populations) return fail(FLBM_EINVAL, "dev_populations is NULL");
  // The statistics kernel reads element pairs (8 bytes in FP32) on even-nx lattices, the
  // same kernels flbm_create_ex feeds from a 256-byte aligned dev_buf: require the same.
  if (reinterpret_cast<uintptr_t>(dev_populations) % 256 != 0)
    return fail(FLBM_EINVAL, "dev_populations must be 256-byte aligned");
  if (!out) return fail(FLBM_EINVAL, "out is NULL");
  const int Q = q_of(lattice);
  const int len = stats_record_len(Q);
  if (len > FLBM_NOALLOC_SCRATCH_DOUBLES)
    return fail(FLBM_EINVAL, "the statistics need %d doubles of scratch; the static scratch holds %d",
                len, FLBM_NOALLOC_SCRATCH_DOUBLES);
  double *acc = nullptr;
  st = noalloc_scratch(&acc);
  if (st != FLBM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const long long N = (long long)(dims[0] * dims[1] * dims[2]);
  FLBM_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * size_t(len), s));
  FLBM_CUDA(launch_stats(klat(lattice), storage, lattice == FLBM_D3Q27_ISO, parity, dev_populations, N,
                         int(dims[0]), int(dims[1]),
                         int(dims[2]), float(rho0), acc, s, 0, N));
  double h[FLBM_NOALLOC_SCRATCH_DOUBLES];
  FLBM_CUDA(cudaMemcpyAsync(h, acc, sizeof(double) * size_t(len), cudaMemcpyDeviceToHost, s));
  FLBM_CUDA(cudaStreamSynchronize(s));
  // The host conversion of flbm_stats, fed with a description of this array.
  flbm_ctx view;
  view.lattice = lattice;
  view.D = d_of(lattice);
  view.Q = Q;
  view.N = N;
  view.rho0 = rho0;
  fill_stats(&view, h, -1, out);
  return stats_result(out, -1);
}

// ---- domain decomposition along z -------------------------------------------------------
// A lattice split into slabs of whole planes (flbm_create_slab, flbm_domain_*). Each slab
// keeps its owned planes between two ghost planes. With the in-place AA pattern a step
// taken from an even step count reads and writes only the site's own slots, so it needs
// no exchange; a step taken from an odd count reads slot opposite(i) of x - c_i and
// writes slot i of x + c_i, which crosses the slab faces for the velocities with c_z != 0.
// Around such a step the slots of those velocities move between the owned boundary planes
// and the neighbours' ghost planes: before it (phase 0) each boundary plane's slots of the
// velocities leaving through the face are copied into the neighbour's ghost plane; after
// it (phase 1) the ghost plane's slots written by the step go back to their owner. No
// other slot of a boundary plane is read or written by the neighbour, so the copies need
// no further ordering with the neighbour's own step. The noise is keyed on the global
// site, so a decomposed lattice steps bitwise like the whole one.
namespace {

int check_slab(int lattice, const int64_t dims[3], int64_t z_begin, int64_t z_count, int storage) {
  int st = check_geometry(lattice, dims, storage);
  if (st != FLBM_OK) return st;
  if (lattice == FLBM_D2Q9)
    return fail(FLBM_EINVAL, "slabs split a 3-D lattice along z; D2Q9 is not decomposed");
  if (z_begin < 0 || z_begin >= dims[2])
    return fail(FLBM_EINVAL, "z_begin = %lld outside [0, %lld)", (long long)z_begin, (long long)dims[2]);
  if (z_count < 1 || z_begin + z_count > dims[2])
    return fail(FLBM_EINVAL, "z_count = %lld must lie in [1, nz - z_begin]", (long long)z_count);
  if (z_count + 2 > 65535) return fail(FLBM_EINVAL, "a slab holds at most 65533 planes");
  if (double(dims[0]) * double(dims[1]) * double(z_count + 2) >= 4294967296.0)
    return fail(FLBM_EINVAL, "a slab's local array (owned and ghost planes) must hold < 2^32 sites");
  return FLBM_OK;
}

// Slots of the velocities with c_z = +1 (dir > 0) or -1 (dir < 0), in index order.
int z_slots(int lattice, int dir, int *out) {
  const int Q = q_of(lattice);
  int n = 0;
  for (int i = 0; i < Q; ++i) {
    const int cz = Lat<3>::cz(i);  // D3Q19 takes the first 19 D3Q27 velocities
    if ((dir > 0 && cz == 1) || (dir < 0 && cz == -1)) out[n++] = i;
  }
  return n;
}

}  // namespace

extern "C" {

size_t flbm_slab_required_bytes(int lattice, const int64_t dims[3], int64_t z_count, int storage) {
  const std::string saved = g_last_error;
  if (!dims || check_slab(lattice, dims, 0, z_count, storage) != FLBM_OK) return 0;
  g_last_error = saved;
  return size_t(q_of(lattice)) * size_t(dims[0] * dims[1] * (z_count + 2)) * storage_bytes(storage);
}

int flbm_slab_halo(int lattice, const int64_t dims[3], int64_t z_count, int phase, int side,
                   int64_t *send_offset, int64_t *recv_offset, int *n_regions, int64_t *region_len) {
  int st = check_slab(lattice, dims, 0, z_count, FLBM_FP32);
  if (st != FLBM_OK) return st;
  if (phase != 0 && phase != 1) return fail(FLBM_EINVAL, "phase must be 0 or 1, got %d", phase);
  if (side != 0 && side != 1) return fail(FLBM_EINVAL, "side must be 0 (lower) or 1 (upper), got %d", side);
  if (!send_offset || !recv_offset || !n_regions || !region_len) return fail(FLBM_EINVAL, "NULL output");
  const int64_t pl = dims[0] * dims[1];          // sites per plane
  const int64_t N = pl * (z_count + 2);          // sites of the local array
  const int64_t top = z_count, ghost_hi = z_count + 1;
  // (plane sent, slot set sent, plane received, slot set received); slot sets by c_z sign.
  int64_t p_send, p_recv;
  int d_send, d_recv;
  if (phase == 0) {  // owned boundary plane -> neighbour's ghost plane
    if (side == 0) { p_send = 1; d_send = +1; p_recv = 0; d_recv = -1; }
    else           { p_send = top; d_send = -1; p_recv = ghost_hi; d_recv = +1; }
  } else {           // ghost plane -> its owner's boundary plane
    if (side == 0) { p_send = 0; d_send = -1; p_recv = 1; d_recv = +1; }
    else           { p_send = ghost_hi; d_send = +1; p_recv = top; d_recv = -1; }
  }
  int ss[27], rs[27];
  const int ns = z_slots(lattice, d_send, ss), nr = z_slots(lattice, d_recv, rs);
  if (ns != nr) return fail(FLBM_EINVAL, "internal: slot sets differ in size");
  for (int k = 0; k < ns; ++k) {
    send_offset[k] = int64_t(ss[k]) * N + p_send * pl;
    recv_offset[k] = int64_t(rs[k]) * N + p_recv * pl;
  }
  *n_regions = ns;
  *region_len = pl;
  return FLBM_OK;
}

int flbm_create_slab(flbm_ctx **out, int lattice, const int64_t dims[3], int64_t z_begin, int64_t z_count,
                     const double *lambda, double kBT, double rho0, uint64_t seed, int storage, void *cuda_stream,
                     void *dev_buf, size_t dev_buf_bytes) {
  if (!out) return fail(FLBM_EINVAL, "out is NULL");
  if (!dims) return fail(FLBM_EINVAL, "dims is NULL");
  int st = check_slab(lattice, dims, z_begin, z_count, storage);
  if (st != FLBM_OK) return st;
  const int64_t local[3] = {dims[0], dims[1], z_count + 2};
  flbm_ctx *c = nullptr;
  st = flbm_create_ex(&c, lattice, local, lambda, kBT, rho0, seed, storage, cuda_stream, dev_buf, dev_buf_bytes);
  if (st != FLBM_OK) return st;
  c->slab = true;
  for (int a = 0; a < 3; ++a) c->gdims[a] = dims[a];
  c->z_begin = z_begin;
  c->z_count = z_count;
  fill_args(c);
  *out = c;
  return FLBM_OK;
}

}  // extern "C"

struct flbm_domain {
  int lattice = 1, Q = 27, storage = 0;
  int64_t dims[3] = {1, 1, 1};
  double rho0 = 1.0;
  std::vector<flbm_ctx *> slabs;
  std::vector<cudaEvent_t> done;  // per slab: its last work that neighbours wait for
  int64_t step = 0;
  bool ghosts_filled = false;  // phase-0 copies made for the current (odd) state
};

namespace {

void domain_release(flbm_domain *d) {
  if (!d) return;
  for (size_t k = 0; k < d->slabs.size(); ++k) {
    flbm_ctx *c = d->slabs[k];
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    if (k < d->done.size() && d->done[k]) cudaEventDestroy(d->done[k]);
    c->in_domain = false;
    release(c);
  }
  delete d;
}

int domain_record(flbm_domain *d) {
  for (size_t k = 0; k < d->slabs.size(); ++k) {
    DeviceGuard g(d->slabs[k]->device);
    FLBM_CUDA(cudaEventRecord(d->done[k], d->slabs[k]->stream));
  }
  return FLBM_OK;
}

// Slab k's stream waits for the last recorded work of its two neighbours (periodic in z).
int domain_wait_neighbours(flbm_domain *d, size_t k) {
  const size_t n = d->slabs.size(), lo = (k + n - 1) % n, hi = (k + 1) % n;
  DeviceGuard g(d->slabs[k]->device);
  FLBM_CUDA(cudaStreamWaitEvent(d->slabs[k]->stream, d->done[lo], 0));
  if (hi != lo) FLBM_CUDA(cudaStreamWaitEvent(d->slabs[k]->stream, d->done[hi], 0));
  return FLBM_OK;
}

// Copies of one message: `from`'s send regions of (phase, side) into `to`'s receive
// regions of (phase, 1 - side), on `stream`.
int domain_copy(const flbm_domain *d, const flbm_ctx *from, const flbm_ctx *to, int phase, int side,
                cudaStream_t stream) {
  int64_t so[27], ro_unused[27], so_unused[27], ro[27], len = 0, len2 = 0;
  int n = 0, n2 = 0;
  int st = flbm_slab_halo(d->lattice, d->dims, from->z_count, phase, side, so, ro_unused, &n, &len);
  if (st == FLBM_OK) st = flbm_slab_halo(d->lattice, d->dims, to->z_count, phase, 1 - side, so_unused, ro, &n2, &len2);
  if (st != FLBM_OK) return st;
  const size_t es = storage_bytes(d->storage);
  for (int k = 0; k < n; ++k) {
    const char *src = static_cast<const char *>(from->f) + size_t(so[k]) * es;
    char *dst = static_cast<char *>(to->f) + size_t(ro[k]) * es;
    FLBM_CUDA(cudaMemcpyAsync(dst, src, size_t(len) * es, cudaMemcpyDefault, stream));
  }
  return FLBM_OK;
}

// Phase 0: every slab fills its ghost planes from its neighbours' boundary planes.
int domain_fill_ghosts(flbm_domain *d) {
  int st = domain_record(d);
  const size_t n = d->slabs.size();
  for (size_t k = 0; k < n && st == FLBM_OK; ++k) {
    st = domain_wait_neighbours(d, k);
    flbm_ctx *me = d->slabs[k], *lo = d->slabs[(k + n - 1) % n], *hi = d->slabs[(k + 1) % n];
    DeviceGuard g(me->device);
    if (st == FLBM_OK) st = domain_copy(d, lo, me, 0, 1, me->stream);  // lower's top -> my lower ghost
    if (st == FLBM_OK) st = domain_copy(d, hi, me, 0, 0, me->stream);  // upper's bottom -> my upper ghost
  }
  if (st == FLBM_OK) st = domain_record(d);
  if (st == FLBM_OK) d->ghosts_filled = true;
  return st;
}

// Phase 1: every slab returns the ghost slots its step wrote to their owners.
int domain_return_ghosts(flbm_domain *d) {
  const size_t n = d->slabs.size();
  int st = FLBM_OK;
  for (size_t k = 0; k < n && st == FLBM_OK; ++k) {
    flbm_ctx *me = d->slabs[k], *lo = d->slabs[(k + n - 1) % n], *hi = d->slabs[(k + 1) % n];
    DeviceGuard g(me->device);
    st = domain_copy(d, me, lo, 1, 0, me->stream);        // my lower ghost -> lower's top plane
    if (st == FLBM_OK) st = domain_copy(d, me, hi, 1, 1, me->stream);  // my upper ghost -> upper's bottom
  }
  if (st == FLBM_OK) st = domain_record(d);
  return st;
}

int domain_view(const flbm_domain *d, flbm_ctx *view) {
  view->lattice = d->lattice;
  view->D = 3;
  view->Q = d->Q;
  view->N = (long long)(d->dims[0] * d->dims[1] * d->dims[2]);
  view->rho0 = d->rho0;
  return FLBM_OK;
}

}  // namespace

extern "C" {

int flbm_domain_create(flbm_domain **out, int lattice, const int64_t dims[3], const double *lambda, double kBT,
                       double rho0, uint64_t seed, int storage, int nslabs, const int *devices) {
  if (!out) return fail(FLBM_EINVAL, "out is NULL");
  if (!dims) return fail(FLBM_EINVAL, "dims is NULL");
  if (nslabs < 1 || nslabs > dims[2])
    return fail(FLBM_EINVAL, "nslabs = %d must lie in [1, nz = %lld]", nslabs, (long long)dims[2]);
  int st = check_slab(lattice, dims, 0, (dims[2] + nslabs - 1) / nslabs, storage);
  if (st != FLBM_OK) return st;
  st = check_params(lattice, lambda, kBT, rho0);
  if (st != FLBM_OK) return st;
  int cur = 0;
  FLBM_CUDA(cudaGetDevice(&cur));
  flbm_domain *d = new (std::nothrow) flbm_domain();
  if (!d) return fail(FLBM_ENOMEM, "host allocation failed");
  d->lattice = lattice;
  d->Q = q_of(lattice);
  d->storage = storage;
  d->rho0 = rho0;
  for (int a = 0; a < 3; ++a) d->dims[a] = dims[a];
  // Planes split as evenly as possible, the first nz mod nslabs slabs one plane thicker.
  int64_t z = 0;
  for (int k = 0; k < nslabs; ++k) {
    const int64_t zc = dims[2] / nslabs + (k < dims[2] % nslabs ? 1 : 0);
    const int dev = devices ? devices[k] : cur;
    flbm_ctx *c = nullptr;
    {
      DeviceGuard g(dev);
      if (!g.ok) {
        domain_release(d);
        return fail(FLBM_EINVAL, "cannot make device %d current", dev);
      }
      st = flbm_create_slab(&c, lattice, dims, z, zc, lambda, kBT, rho0, seed, storage, nullptr, nullptr, 0);
      cudaEvent_t e = nullptr;
      if (st == FLBM_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        release(c);
        st = fail(FLBM_ECUDA, "cudaEventCreate failed");
      }
      if (st != FLBM_OK) {
        const std::string msg = g_last_error;
        domain_release(d);
        return fail(st, "slab %d: %s", k, msg.c_str());
      }
      c->in_domain = true;
      d->slabs.push_back(c);
      d->done.push_back(e);
    }
    z += zc;
  }
  const int rs = domain_record(d);
  if (rs != FLBM_OK) {
    domain_release(d);
    return rs;
  }
  *out = d;
  return FLBM_OK;
}

void flbm_domain_destroy(flbm_domain *d) { domain_release(d); }

int flbm_domain_size(const flbm_domain *d) { return d ? int(d->slabs.size()) : -1; }

flbm_ctx *flbm_domain_slab(flbm_domain *d, int k) {
  if (!d || k < 0 || k >= int(d->slabs.size())) {
    fail(FLBM_EINVAL, "no slab %d in this domain", k);
    return nullptr;
  }
  return d->slabs[size_t(k)];
}

int flbm_domain_init_uniform(flbm_domain *d, const double u0[3], double amp, uint64_t perturb_seed) {
  if (!d) return fail(FLBM_EINVAL, "domain is NULL");
  for (flbm_ctx *c : d->slabs) {
    const int st = flbm_init_uniform(c, u0, amp, perturb_seed);
    if (st != FLBM_OK) return st;
  }
  d->step = 0;
  d->ghosts_filled = false;
  return domain_record(d);
}

int flbm_domain_step(flbm_domain *d, int64_t n) {
  if (!d) return fail(FLBM_EINVAL, "domain is NULL");
  if (n < 0) return fail(FLBM_EINVAL, "n = %lld must be >= 0", (long long)n);
  for (int64_t s = 0; s < n; ++s) {
    const bool odd = (d->step & 1) != 0;
    int st = FLBM_OK;
    if (odd && !d->ghosts_filled) st = domain_fill_ghosts(d);
    for (size_t k = 0; k < d->slabs.size() && st == FLBM_OK; ++k) {
      st = domain_wait_neighbours(d, k);
      if (st == FLBM_OK) st = flbm_step(d->slabs[k], 1);
    }
    if (st == FLBM_OK) st = odd ? domain_return_ghosts(d) : domain_record(d);
    if (st != FLBM_OK) return st;
    d->ghosts_filled = false;
    ++d->step;
  }
  return FLBM_OK;
}

int64_t flbm_domain_get_step(const flbm_domain *d) { return d ? d->step : -1; }

int flbm_domain_set_step_variant(flbm_domain *d, int variant) {
  if (!d) return fail(FLBM_EINVAL, "domain is NULL");
  for (flbm_ctx *c : d->slabs) {
    const int st = flbm_set_step_variant(c, variant);
    if (st != FLBM_OK) return st;
  }
  return FLBM_OK;
}

int flbm_domain_sync(flbm_domain *d) {
  if (!d) return fail(FLBM_EINVAL, "domain is NULL");
  for (flbm_ctx *c : d->slabs) {
    const int st = flbm_sync(c);
    if (st != FLBM_OK) return st;
  }
  return FLBM_OK;
}

int flbm_domain_stats(flbm_domain *d, flbm_stats_t *out) {
  if (!d) return fail(FLBM_EINVAL, "domain is NULL");
  if (!out) return fail(FLBM_EINVAL, "out is NULL");
  // An odd state's owned sites read their arriving populations from the ghost planes.
  if ((d->step & 1) && !d->ghosts_filled) {
    const int st = domain_fill_ghosts(d);
    if (st != FLBM_OK) return st;
  }
  const size_t len = size_t(stats_record_len(d->Q));
  std::vector<double> sum(len, 0.0);
  for (size_t k = 0; k < d->slabs.size(); ++k) {
    flbm_ctx *c = d->slabs[k];
    DeviceGuard g(c->device);
    int st = domain_wait_neighbours(d, k);
    if (st == FLBM_OK) st = enqueue_stats(c, c->d_acc);
    if (st != FLBM_OK) return st;
    FLBM_CUDA(cudaMemcpyAsync(c->h_acc, c->d_acc, sizeof(double) * len, cudaMemcpyDeviceToHost, c->stream));
    FLBM_CUDA(cudaStreamSynchronize(c->stream));
    // Every entry of the record is a plain sum over sites (Gram entries and the
    // non-finite count): the slabs' records add in FP64.
    for (size_t i = 0; i < len; ++i) sum[i] += c->h_acc[i];
  }
  flbm_ctx view;
  domain_view(d, &view);
  fill_stats(&view, sum.data(), d->step, out);
  return stats_result(out, (long long)d->step);
}

int flbm_domain_get_populations(flbm_domain *d, double *host, size_t count) {
  if (!d) return fail(FLBM_EINVAL, "domain is NULL");
  if (!host) return fail(FLBM_EINVAL, "host is NULL");
  const size_t pl = size_t(d->dims[0] * d->dims[1]), N = pl * size_t(d->dims[2]);
  if (count != size_t(d->Q) * N) return fail(FLBM_EINVAL, "count = %zu, expected Q * sites = %zu", count, size_t(d->Q) * N);
  if ((d->step & 1) && !d->ghosts_filled) {
    const int st = domain_fill_ghosts(d);
    if (st != FLBM_OK) return st;
  }
  for (size_t k = 0; k < d->slabs.size(); ++k) {
    flbm_ctx *c = d->slabs[k];
    const size_t nl = size_t(c->N);
    std::vector<double> loc(size_t(d->Q) * nl);
    int st = domain_wait_neighbours(d, k);
    if (st == FLBM_OK) st = flbm_get_populations(c, loc.data(), loc.size());
    if (st != FLBM_OK) return st;
    for (int q = 0; q < d->Q; ++q)
      std::memcpy(host + size_t(q) * N + size_t(c->z_begin) * pl, loc.data() + size_t(q) * nl + pl,
                  sizeof(double) * pl * size_t(c->z_count));
  }
  return FLBM_OK;
}

int flbm_domain_set_populations(flbm_domain *d, const double *host, size_t count) {
  if (!d) return fail(FLBM_EINVAL, "domain is NULL");
  if (!host) return fail(FLBM_EINVAL, "host is NULL");
  const size_t pl = size_t(d->dims[0] * d->dims[1]), N = pl * size_t(d->dims[2]);
  if (count != size_t(d->Q) * N) return fail(FLBM_EINVAL, "count = %zu, expected Q * sites = %zu", count, size_t(d->Q) * N);
  // Each slab takes its owned planes and, in its ghost planes, the neighbouring planes of
  // the whole lattice (periodic): every slot the scatter writes then holds its true value,
  // whichever slab owns it in the current AA state.
  for (flbm_ctx *c : d->slabs) {
    const size_t nl = size_t(c->N);
    std::vector<double> loc(size_t(d->Q) * nl);
    for (int64_t p = 0; p < c->z_count + 2; ++p) {
      const int64_t zg = ((c->z_begin + p - 1) % d->dims[2] + d->dims[2]) % d->dims[2];
      for (int q = 0; q < d->Q; ++q)
        std::memcpy(loc.data() + size_t(q) * nl + size_t(p) * pl, host + size_t(q) * N + size_t(zg) * pl,
                    sizeof(double) * pl);
    }
    const int st = flbm_set_populations(c, loc.data(), loc.size());
    if (st != FLBM_OK) return st;
  }
  d->ghosts_filled = false;
  return domain_record(d);
}

}  // extern "C"
