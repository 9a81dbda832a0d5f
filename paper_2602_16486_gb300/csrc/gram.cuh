// Gram-matrix accumulation of the statistics (Sec. III diagnostics and the mode
// covariances of Sec. II-B) for the statistics kernel (stats.cu).
//
// Every recorded sum is an entry of G = sum_x c(x) c(x)^T over the per-site column
//   c = [1, rho - rho0, j_x, j_y, j_z, u_x, u_y, u_z, k_{D+1} .. k_{Q-1}, 0 ...]
// (NC = 32 entries for D3Q27 and D3Q19, 16 for D2Q9). G is a dense contraction over the
// sites, so it runs on the fifth-generation tensor cores (tcgen05): BF16 inputs, FP32
// accumulators in tensor memory (TMEM), K running over sites. Each input is split into
// x_hi = bf16(x) and x_lo = bf16(x - x_hi) (both rounded to nearest; x - x_hi is exact in
// FP32), and every product is formed as hi*hi + hi*lo + lo*hi + lo*lo: what is left out is
// the rounding of x_lo, below 2^-16 of x with either sign, so the products carry no bias
// and at most 2^-15 relative error each. BF16 keeps FP32's exponent range, so no column
// needs scaling.
//
// Operands. A warp's 32 threads hold 64 sites (two per thread). The warp stages them as
// X = [X_hi; X_lo], 2 NC rows (one per column and part) by 64 sites, K-major: row r is one
// 128-byte line of 64 BF16 values, with the 128-byte swizzle (16-byte chunk q of row r at
// chunk position q ^ (r mod 8)), i.e. the canonical SWIZZLE_128B K-major layout of the
// tensor-core shared-memory descriptor. The four warps' regions are contiguous, so 128
// consecutive rows are the regions of 128 / (2 NC) warps. One MMA of shape M = N = 128,
// K = 16 takes those 128 rows as both A and B: D = A B^T holds, in its diagonal blocks of
// 2 NC x 2 NC, exactly the Gram matrices X X^T of those warps (the off-diagonal blocks mix
// different warps' sites at the same K index and are never read). Every MMA of a tile
// accumulates into the same 128 x 128 FP32 accumulator (128 TMEM columns), so the
// diagonal blocks sum the Grams of all staged sites. Every warp arrives on a "staged"
// mbarrier after its lanes have written their rows; one thread waits for it, issues the
// tile's MMAs (4 K-steps per 128-row group) and commits them to a "done" mbarrier, on
// which the warps wait before they overwrite the staging rows. Apart from the flushes no
// block-wide barrier sits in the loop, so a warp runs ahead into the loads and arithmetic
// of its next pair while the tensor cores work. After every kFlushTiles tiles (at the wait
// that precedes the next staging) the warps read their quadrant of the accumulator
// (tcgen05.ld), add hi and lo column halves and leave the rows in FP32 scratch (the idle
// staging rows); each entry of the upper triangle then sums its few contributions in FP32
// and is added once, by the thread that owns it, to the block's FP64 sums (no atomics:
// GB300's FP64 pipe is narrow). The next tile's first MMA overwrites the accumulator. At
// the end the block adds its sums to the output record with one FP64 atomic per entry.
// Output record: the upper triangle of G in FP64, row-major, then the number of
// non-finite sites (a bounded wait that gave up adds kStatsTimeoutMark to that count).
#pragma once

#include <cuda_runtime.h>

#include "async.cuh"
#include "cm.cuh"
#include "internal.h"

namespace flbm {

template <int D>  // D: 2 (D2Q9), 3 (D3Q27) or 19 (D3Q19)
struct StatsPlan {
  static constexpr int NC = D == 2 ? 16 : 32;  // columns, padded to a power of two
  // Columns in use: 1, rho - rho0, j (3), u (3) and the non-conserved modes.
  static constexpr int USED = 8 + (D == 2 ? 6 : D == 19 ? 15 : 23);
  static constexpr int NREC = NC * (NC + 1) / 2;
};

namespace gram {

constexpr int kWarps = kStatsBlock / 32;   // warps per block (one TMEM lane quadrant each)
constexpr int kTileSites = 2 * kStatsBlock;  // two sites per thread
constexpr int kRowBytes = 128;             // one staged row: 64 sites in BF16
constexpr uint32_t kTmemCols = 128;        // the 128 x 128 FP32 accumulator
// 52 KB per block: four blocks fit the SM's 228 KB of shared memory, five do not (each
// block holds 128 of the SM's 512 TMEM columns).
constexpr size_t kSmemFloor = 52 * 1024;
// Resident blocks per SM the kernel is built for (launch bounds and grid): three for the
// 3-D lattices, whose prefetched populations need up to 170 registers, four for D2Q9.
template <int D>
__host__ __device__ constexpr int blocks_per_sm() {
  return D == 2 ? 4 : 3;
}
constexpr int kFlushTiles = 8;  // FP32 sums over at most 8 tiles (1024 sites per accumulator entry)
// Added to the non-finite count of the record when a bounded wait gave up (the host
// reports FLBM_ETIMEOUT for a negative count).
constexpr double kStatsTimeoutMark = -1099511627776.0;  // -2^40

template <int D>
struct Plan {
  using SP = StatsPlan<D>;
  static constexpr int NC = SP::NC;
  static constexpr int ROWS = 2 * NC;                  // hi rows, then lo rows
  static constexpr int REGION = ROWS * kRowBytes;      // one warp's staging: 8 KB or 4 KB
  static constexpr int BUF = kWarps * REGION;          // the block's staging
  static constexpr int GROUPS = kWarps * ROWS / 128;   // 128-row MMA operands per tile
  static constexpr int ACC = StatsPlan<D>::NREC;       // FP64 sums, in record order
  // Shared memory: 1024 bytes of alignment slack, the staging rows, the sums, the two
  // mbarriers and the TMEM address; at least kSmemFloor, so that at most four blocks (4 x
  // 128 TMEM columns) share an SM.
  static constexpr size_t NEED = 1024 + BUF + sizeof(double) * ACC + 32;
  static constexpr size_t SMEM = NEED > kSmemFloor ? NEED : kSmemFloor;
};

// bf16x2 of (a, b): a in the low half (the lower K index), b in the high half; rounded to
// nearest.
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte swizzle: start
// address (16-byte units, bits 0-13), leading byte offset (unused by this layout; 16 B),
// stride byte offset between 8-row groups = 8 x 128 B (bits 32-45), the fixed value 1 in
// bits 46-48, base offset 0 (1024-byte aligned atoms), layout 2 = SWIZZLE_128B (bits 61-63).
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: D in FP32 (bits 4-5 = 1), A and B in BF16 (bits
// 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 in bits 17-22, M / 16 in
// bits 24-28; M = N = 128.
constexpr uint32_t kIdescBf16M128N128 = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) |
                                        ((128u >> 4) << 24);

// D (TMEM) = A B^T (+ D when accumulate), A and B from shared memory; issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(kIdescBf16M128N128), "r"(accumulate)
      : "memory");
}

// The mbarrier completes a phase when every MMA issued before by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

// One arrival on an mbarrier (release semantics at CTA scope).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy shared-memory writes become visible to the tensor cores (async proxy).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Warp-wide (all 32 lanes): allocate kTmemCols columns, address written to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t *slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
               "r"(kTmemCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp-wide; the warp's quadrant).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// Columns of a pair (lane x: first site, lane y: second) from its central moments: F as
// left by site_central_moments (entry (0,0,0) = rho; Q = 27 or 9), drho = rho - rho0.
// v0 / v1: the site exists. A site whose column holds a NaN or an infinity makes the sum
// of its entries non-finite (the entries are far below overflow); such a site
// contributes a zero column (select, not multiply: it may hold NaN) and is counted.
template <int D, bool ISO, int NC>
__device__ __forceinline__ void moment_columns(const float2 (&F)[3][3][3], float2 drho, float2 rho, float2 ux,
                                               float2 uy, float2 uz, bool v0, bool v1, float2 (&col)[NC],
                                               unsigned &nonfinite) {
  constexpr int Q = Lat<D>::Q;
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
  col[0] = make_float2(v0 ? 1.0f : 0.0f, v1 ? 1.0f : 0.0f);
  col[1] = drho;
  col[2] = vmul(rho, ux);
  col[3] = vmul(rho, uy);
  col[4] = vmul(rho, uz);
  col[5] = ux;
  col[6] = uy;
  col[7] = uz;
#pragma unroll
  for (int v = D + 1; v < Q; ++v) col[8 + v - D - 1] = k[v];
#pragma unroll
  for (int c = 8 + Q - D - 1; c < NC; ++c) col[c] = make_float2(0.0f, 0.0f);
  float2 sum = col[1];
#pragma unroll
  for (int c = 2; c < 8 + Q - D - 1; ++c) sum = vadd(sum, col[c]);
  const bool valid[2] = {v0, v1};
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    if (valid[l] && !isfinite(lane(sum, l))) {
      ++nonfinite;
#pragma unroll
      for (int c = 0; c < NC; ++c) set_lane(col[c], l, 0.0f);
    }
  }
}

// The staging offsets of this lane: offs[k] = byte offset, within its warp's region, of
// the lane's bf16x2 word in a row r with r mod 8 = k (chunk lane / 4 at position
// (lane / 4) ^ k, word lane mod 4 of the chunk).
__device__ __forceinline__ void stage_offsets(uint32_t (&offs)[8]) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (uint32_t k = 0; k < 8; ++k) offs[k] = (((lane >> 2) ^ k) << 4) | ((lane & 3u) << 2);
}

// Splits the first USED columns of this thread's site pair (lane x: lower K index) into
// the hi rows 0..USED-1 and the lo rows NC..NC+USED-1 of its warp's region (the other
// rows hold zeros, written once).
template <int D, int USED>
__device__ __forceinline__ void stage_columns(unsigned char *region, const uint32_t (&offs)[8],
                                              const float2 (&col)[StatsPlan<D>::NC]) {
  constexpr int NC = StatsPlan<D>::NC;
#pragma unroll
  for (int c = 0; c < USED; ++c) {
    const float2 x = col[c];
    const uint32_t h = pack_bf16x2(x.x, x.y);
    const float hx = __uint_as_float(h << 16), hy = __uint_as_float(h & 0xFFFF0000u);
    const uint32_t e = pack_bf16x2(x.x - hx, x.y - hy);  // exact differences, rounded to BF16
    *reinterpret_cast<uint32_t *>(region + c * kRowBytes + offs[c & 7]) = h;
    *reinterpret_cast<uint32_t *>(region + (NC + c) * kRowBytes + offs[(NC + c) & 7]) = e;
  }
}

// Issues the tile's MMAs (one thread): GROUPS operands of 128 rows, 4 K-steps of 16 sites
// (32 bytes inside the 128-byte swizzle row) each; the first overwrites the accumulator
// when `fresh`.
template <int D>
__device__ __forceinline__ void issue_tile(uint32_t buf_saddr, uint32_t tmem, bool fresh) {
  using P = Plan<D>;
#pragma unroll
  for (int g = 0; g < P::GROUPS; ++g)
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const uint64_t desc = sw128_kmajor_desc(buf_saddr + (uint32_t)(g * 128 * kRowBytes + kk * 32));
      mma_bf16(tmem, desc, desc, (fresh && g == 0 && kk == 0) ? 0u : 1u);
    }
}

// Accumulator row of this thread: lane l of warp q holds TMEM lane 32 q + l, which is row
// r = (32 q + l) mod 2 NC of a diagonal block starting at column 2 NC (32 q / 2 NC); row r
// is column i = r mod NC of G (hi part for r < NC, lo part otherwise). Its contribution
// slot (32 q + l) / NC (4 slots for NC = 32, 8 for NC = 16) is unique per (block, part, i).
template <int D>
struct Flush {
  using P = Plan<D>;
  static constexpr int NC = P::NC, SLOTS = 128 / NC, NREC = StatsPlan<D>::NREC;
  static constexpr int PER_THREAD = (NREC + kStatsBlock - 1) / kStatsBlock;
  uint32_t taddr;            // this lane's first accumulator column of its diagonal block
  int slot, i;               // contribution slot and G column
  int ent_off[PER_THREAD];   // scratch offset j NC + i of the record entries this thread owns

  __device__ __forceinline__ void init(uint32_t tmem) {
    const int q = threadIdx.x >> 5, grow = threadIdx.x;  // 32 q + lane
    taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((grow / P::ROWS) * P::ROWS);
    slot = grow / NC;
    i = grow % NC;
    // Record entry e = a NC - a (a - 1) / 2 + (b - a) is G(a, b), a <= b (row-major upper
    // triangle); this thread owns e = threadIdx.x + k kStatsBlock.
#pragma unroll
    for (int k = 0; k < PER_THREAD; ++k) {
      const int e = threadIdx.x + k * kStatsBlock;
      int a = 0;
      while (a + 1 < NC && (a + 1) * NC - (a + 1) * a / 2 <= e) ++a;
      const int b = a + (e - (a * NC - a * (a - 1) / 2));
      ent_off[k] = e < NREC ? b * NC + a : -1;
    }
  }

  // Every thread of the block, after the MMAs of the closed period are done: each row goes
  // to the scratch (FP32, [slot][j][i], in the idle staging rows), then the owner of each
  // record entry adds the sum of its slots to the block's FP64 sums. `valid`: warp-uniform;
  // a warp whose wait gave up skips its accumulator reads (the block then reports failure).
  __device__ __forceinline__ void run(float *scratch, double *sums, bool valid) {
    if (valid) {
#pragma unroll
      for (int j0 = 0; j0 < NC; j0 += 16) {
        float hi[16], lo[16];
        tmem_ld16(taddr + (uint32_t)j0, hi);
        tmem_ld16(taddr + (uint32_t)(NC + j0), lo);
#pragma unroll
        for (int k = 0; k < 16; ++k) scratch[(slot * NC + j0 + k) * NC + i] = hi[k] + lo[k];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER_THREAD; ++k) {
      if (ent_off[k] < 0) continue;
      float v = 0.0f;
#pragma unroll
      for (int sl = 0; sl < SLOTS; ++sl) v += scratch[sl * NC * NC + ent_off[k]];
      sums[threadIdx.x + k * kStatsBlock] += (double)v;
    }
    __syncthreads();  // the scratch is staging memory again
  }
};

// After the block's last flush and a barrier: adds its FP64 sums (in record order) and
// its non-finite count, or the timeout mark, to the output record.
template <int D>
__device__ __forceinline__ void finish(const double *sums, unsigned nonfinite_block, bool failed,
                                       double *__restrict__ out) {
  constexpr int NREC = StatsPlan<D>::NREC;
  for (int e = threadIdx.x; e < NREC; e += blockDim.x) atomicAdd(&out[e], sums[e]);
  if (threadIdx.x == 0) {
    double mark = (double)nonfinite_block;
    if (failed) mark += kStatsTimeoutMark;
    if (mark != 0.0) atomicAdd(&out[NREC], mark);
  }
}

// The block's side of the reduction (the statistics kernel, stats.cu): set-up (TMEM,
// mbarriers, sums, the rows of unused columns), one call per tile that stages the thread's
// columns and has one thread multiply the tile, and the end (last flush, record, TMEM
// freed). Every thread of the block makes every call, in the same order.
template <int D>
struct Pipeline {
  using P = Plan<D>;
  static constexpr int NC = P::NC, USED = StatsPlan<D>::USED;
  unsigned char *buf, *region;
  double *sums;
  uint64_t *staged, *bar;  // every warp once per tile / the tile's MMAs are done
  uint32_t tmem, buf_s;
  uint32_t offs[8];
  Flush<D> fl;
  bool ok;
  int t;

  // `raw`: the kernel's dynamic shared memory (P::SMEM bytes); `flags`: two shared words of
  // the kernel (non-finite count, failure flag). Ends with a block barrier.
  __device__ __forceinline__ void init(unsigned char *raw, unsigned int *flags) {
    const uint32_t raw_s = smem_addr(raw);
    buf = raw + (((raw_s + 1023u) & ~1023u) - raw_s);  // 1024-byte aligned swizzle atoms
    sums = reinterpret_cast<double *>(buf + P::BUF);
    staged = reinterpret_cast<uint64_t *>(sums + P::ACC);
    bar = staged + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    const int warp = threadIdx.x >> 5;
    region = buf + warp * P::REGION;
    if (warp == 0) tmem_alloc(tslot);
    if (threadIdx.x == 0) {
      flags[0] = 0u;
      flags[1] = 0u;
      mbar_init(staged, kWarps);
      mbar_init(bar, 1);
      fence_mbar_init();
    }
    for (int e = threadIdx.x; e < P::ACC; e += blockDim.x) sums[e] = 0.0;
    // Rows of the unused columns (hi and lo) stay zero for the whole kernel.
    constexpr int ZR = NC - USED, W = kRowBytes / 4;
    for (int e = threadIdx.x; e < kWarps * 2 * ZR * W; e += blockDim.x) {
      const int w = e / (2 * ZR * W), rr = (e / W) % (2 * ZR), k = e % W;
      const int row = rr < ZR ? USED + rr : NC + USED + (rr - ZR);
      reinterpret_cast<uint32_t *>(buf + w * P::REGION + row * kRowBytes)[k] = 0u;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tmem = *tslot;
    buf_s = smem_addr(buf);
    stage_offsets(offs);
    fl.init(tmem);
    ok = true;
    t = 0;
  }

  // One tile: waits for the previous tile's MMAs (they have read the staging rows; when
  // they closed an accumulation period the accumulator is read now, before this tile's
  // first MMA overwrites it), stages the columns, and thread 0 multiplies the tile once
  // every warp has staged.
  __device__ __forceinline__ void tile(const float2 (&col)[NC]) {
    if (t > 0) {
      if (ok) ok = mbar_wait_bounded(bar, (uint32_t)(t - 1) & 1u);
      if ((t - 1) % kFlushTiles == kFlushTiles - 1) {
        ok = __all_sync(0xFFFFFFFFu, ok);  // the accumulator reads are warp-wide (.sync.aligned)
        tc_fence_after();
        fl.run(reinterpret_cast<float *>(buf), sums, ok);
      }
    }
    stage_columns<D, USED>(region, offs, col);
    fence_async_smem();  // each thread's rows, for the tensor cores
    tc_fence_before();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(staged);  // the warp's rows are staged
    if (threadIdx.x == 0) {
      if (ok) ok = mbar_wait_bounded(staged, (uint32_t)t & 1u);
      tc_fence_after();
      if (ok) issue_tile<D>(buf_s, tmem, t % kFlushTiles == 0);
      mma_commit(bar);
    }
    ++t;
  }

  // After the last tile (t >= 1): the last accumulation period, the record, TMEM freed.
  __device__ __forceinline__ void end(unsigned nonfinite, unsigned int *flags, double *__restrict__ out) {
    if (ok) ok = mbar_wait_bounded(bar, (uint32_t)(t - 1) & 1u);
    ok = __all_sync(0xFFFFFFFFu, ok);
    tc_fence_after();
    if (!ok) {
      flags[1] = 1u;
      mbar_wait_bounded(bar, (uint32_t)(t - 1) & 1u);  // the MMAs in flight, bounded again
    }
    fl.run(reinterpret_cast<float *>(buf), sums, ok);
    tc_fence_before();
    if (nonfinite) atomicAdd(&flags[0], nonfinite);
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
      tc_fence_after();
      tmem_dealloc(tmem);
    }
    finish<D>(sums, flags[0], flags[1] != 0u, out);
  }
};

}  // namespace gram
}  // namespace flbm
