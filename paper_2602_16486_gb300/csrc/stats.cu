// Statistics reduction over one lattice state: the diagnostics of Sec. III (spatial
// means <u_a>, <u_a u_b> for the equipartition tests, Eq. for <u_a^2> = kBT/rho0) and
// the central-moment means and covariances whose equilibrium form is C^eq (Sec. II-B,
// "Structural properties"), plus mass and momentum for the conservation checks.
//
// Per site the kernel recomputes rho, u and the central moments k_v (same factorised
// transform as the step) in FP32 and writes one row of NCOL values
//   [1, rho - rho0, j_x, j_y, j_z, u_x, u_y, u_z, k_0 .. k_{Q-1}]
// to a shared-memory tile of 128 sites. Each accumulator is a product of two columns,
// summed over the tile in FP32 and added to a per-thread FP64 register; one FP64
// atomic per accumulator and block ends the kernel. Sites with a non-finite value are
// left out and counted. Accumulator layout (doubles):
//   [0] number of finite sites         [1] sum (rho - rho0)   [2..4] sum j
//   [5..7] sum u                        [8..13] sum u_a u_b (xx, yy, zz, xy, xz, yz)
//   [14 .. 14+Q) sum k_v                then sum k_v k_w for v <= w (row-major upper)
//   [nacc] number of non-finite sites
#include <cuda_runtime.h>

#include "cm.cuh"
#include "internal.h"

namespace flbm {

int stats_nacc(int Q) { return 14 + Q + Q * (Q + 1) / 2; }

namespace {

// Column pair (p, q) whose product accumulator e sums.
template <int Q>
__device__ __forceinline__ void acc_pair(int e, int &p, int &q) {
  constexpr int kOne = 0, kU = 5, kK = 8;
  if (e == 0) {
    p = kOne;
    q = kOne;
  } else if (e < 8) {
    p = kOne;
    q = e;  // rho - rho0, j, u
  } else if (e < 14) {
    const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
    p = kU + pa[e - 8];
    q = kU + pb[e - 8];
  } else if (e < 14 + Q) {
    p = kOne;
    q = kK + (e - 14);
  } else {
    int r = e - 14 - Q, v = 0;
    while (r >= Q - v) {
      r -= Q - v;
      ++v;
    }
    p = kK + v;
    q = kK + v + r;
  }
}

template <int D, typename S, int PARITY>
__global__ void __launch_bounds__(kStatsBlock) stats_kernel(const S *__restrict__ f, long long plane,
                                                            int nx, int ny, int nz, float rho0,
                                                            double *__restrict__ acc) {
  constexpr int Q = Lat<D>::Q;
  constexpr int NCOL = 8 + Q;
  constexpr int LD = NCOL | 1;
  constexpr int NACC = 14 + Q + Q * (Q + 1) / 2;
  constexpr int PER = (NACC + kStatsBlock - 1) / kStatsBlock;
  __shared__ float tile[kStatsBlock * LD];
  __shared__ unsigned int nonfinite;
  if (threadIdx.x == 0) nonfinite = 0u;
  __syncthreads();

  int pp[PER], qq[PER];
  double sum[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int e = threadIdx.x + r * kStatsBlock;
    pp[r] = qq[r] = 0;
    if (e < NACC) acc_pair<Q>(e, pp[r], qq[r]);
    sum[r] = 0.0;
  }
  const long long N = plane;
  for (long long base = (long long)blockIdx.x * kStatsBlock; base < N;
       base += (long long)gridDim.x * kStatsBlock) {
    const long long s = base + threadIdx.x;
    float col[NCOL];
#pragma unroll
    for (int c = 0; c < NCOL; ++c) col[c] = 0.0f;
    if (s < N) {
      const int x = (int)(s % nx);
      const int y = (int)((s / nx) % ny);
      const int z = (int)(s / ((long long)nx * ny));
      const Neighbourhood nb = neighbourhood(x, y, z, nx, ny, nz);
      float F[3][3][3];
      load_logical<D, S, PARITY>(f, plane, nb, F);
      float drho, rho, ux, uy, uz;
      site_central_moments<D>(F, rho0, drho, rho, ux, uy, uz);
      float k[Q];
      paper_modes<D>(F, k);
      bool ok = isfinite(rho) && isfinite(ux) && isfinite(uy) && isfinite(uz);
#pragma unroll
      for (int v = 0; v < Q; ++v) ok = ok && isfinite(k[v]);
      if (ok) {
        col[0] = 1.0f;
        col[1] = drho;
        col[2] = rho * ux;
        col[3] = rho * uy;
        col[4] = rho * uz;
        col[5] = ux;
        col[6] = uy;
        col[7] = uz;
#pragma unroll
        for (int v = 0; v < Q; ++v) col[8 + v] = k[v];
      } else {
        atomicAdd(&nonfinite, 1u);
      }
    }
#pragma unroll
    for (int c = 0; c < NCOL; ++c) tile[threadIdx.x * LD + c] = col[c];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      float t = 0.0f;
#pragma unroll 8
      for (int j = 0; j < kStatsBlock; ++j) t = fmaf(tile[j * LD + pp[r]], tile[j * LD + qq[r]], t);
      sum[r] += (double)t;
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int e = threadIdx.x + r * kStatsBlock;
    if (e < NACC) atomicAdd(&acc[e], sum[r]);
  }
  __syncthreads();
  if (threadIdx.x == 0 && nonfinite) atomicAdd(&acc[NACC], (double)nonfinite);
}

template <int D, typename S>
cudaError_t launch_typed(int parity, const void *f, long long plane, int nx, int ny, int nz,
                         float rho0, double *acc, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long tiles = (plane + kStatsBlock - 1) / kStatsBlock;
  const long long cap = (long long)(sms > 0 ? sms : 1) * 8;
  const int grid = (int)(tiles < cap ? tiles : cap);
  const S *p = static_cast<const S *>(f);
  if (parity == 0)
    stats_kernel<D, S, 0><<<grid, kStatsBlock, 0, s>>>(p, plane, nx, ny, nz, rho0, acc);
  else
    stats_kernel<D, S, 1><<<grid, kStatsBlock, 0, s>>>(p, plane, nx, ny, nz, rho0, acc);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stats(int D, int storage, int parity, const void *f, long long plane, int nx,
                         int ny, int nz, float rho0, double *acc, cudaStream_t s) {
  if (D == 3) {
    if (storage == 0) return launch_typed<3, float>(parity, f, plane, nx, ny, nz, rho0, acc, s);
    if (storage == 1)
      return launch_typed<3, __nv_bfloat16>(parity, f, plane, nx, ny, nz, rho0, acc, s);
    return launch_typed<3, __half>(parity, f, plane, nx, ny, nz, rho0, acc, s);
  }
  if (storage == 0) return launch_typed<2, float>(parity, f, plane, nx, ny, nz, rho0, acc, s);
  if (storage == 1)
    return launch_typed<2, __nv_bfloat16>(parity, f, plane, nx, ny, nz, rho0, acc, s);
  return launch_typed<2, __half>(parity, f, plane, nx, ny, nz, rho0, acc, s);
}

}  // namespace flbm
