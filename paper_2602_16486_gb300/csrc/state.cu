// State set-up and exchange kernels: the equilibrium initialiser and the conversion
// between the stored AA-pattern deviations and logical FP64 populations.
//
// Equilibrium (Sec. II-B Eq. feq for D2Q9 to fourth order, Sec. II-C for D3Q27 to
// sixth order): on these lattices the complete Hermite expansion equals the product
//   f^eq_i = rho * prod_a g(c_ia, u_a),  g(0, u) = 2/3 - u^2,  g(+-1, u) = (1 +- 3u + 3u^2)/6,
// which is what the initialiser evaluates (FP64, once per run). D3Q19 (lattice code 19)
// has no product form; its equilibrium is the state with central moments (rho, 0, ..., 0),
// built in FP64 with the generated transforms of d3q19_gen.cuh.
#include <cuda_runtime.h>

#include "cm.cuh"
#include "d3q19_gen.cuh"
#include "internal.h"
#include "philox.cuh"

namespace flbm {
namespace {

__device__ __forceinline__ double g1d(int c, double u) {
  return c == 0 ? 2.0 / 3.0 - u * u : (1.0 + 3.0 * c * u + 3.0 * u * u) / 6.0;
}

// Logical slot of population i at site (x, y, z) for the given AA parity:
// even: A[i][x], odd: A[opposite(i)][x - c_i] (periodic).
template <int D>
__device__ __forceinline__ long long logical_slot(int i, int x, int y, int z, int nx, int ny, int nz,
                                                  long long plane, int parity) {
  if (parity == 0) return (long long)i * plane + ((long long)z * ny + y) * nx + x;
  int xx = x - Lat<D>::cx(i), yy = y - Lat<D>::cy(i), zz = z - Lat<D>::cz(i);
  xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
  yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
  zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
  return (long long)opposite<D>(i) * plane + ((long long)zz * ny + yy) * nx + xx;
}

template <int D, typename S>
__global__ void init_kernel(S *__restrict__ f, long long plane, int nx, int ny, int nz, double rho0,
                            double ux, double uy, double uz, double amp, uint32_t key0,
                            uint32_t key1, uint32_t site_base) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= plane) return;
  double rho = rho0;
  if (amp != 0.0) {
    // Tag-1 stream: counter (site, 0, 0, 1 << 16), word 0 -> U in (0, 1).
    const uint4 w = philox4x32_10(make_uint4((uint32_t)s + site_base, 0u, 0u, 1u << 16), key0, key1);
    const double U = (double)uniform01(w.x);
    rho = rho0 * (1.0 + amp * (2.0 * U - 1.0));
  }
  constexpr int Q = Lat<D>::Q;
  if constexpr (D == 19) {
    // r* from k^eq = (rho, 0, ...): rows 4..18 by the inverse shift, r*_0 = rho - rho0,
    // r*_a = rho u_a; then the deviations M^{-1} r*.
    double r[19], d[19];
#pragma unroll
    for (int v = 0; v < 19; ++v) r[v] = 0.0;
    d3q19_raw_from_central(r, rho, ux, uy, uz);
    r[0] = rho - rho0;
    r[1] = rho * ux;
    r[2] = rho * uy;
    r[3] = rho * uz;
    d3q19_pop(r, d);
#pragma unroll
    for (int i = 0; i < 19; ++i) Storage<S>::store(f + (long long)i * plane + s, (float)d[i]);
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      double fe = rho * g1d(Lat<D>::cx(i), ux) * g1d(Lat<D>::cy(i), uy);
      if (D == 3) fe *= g1d(Lat<D>::cz(i), uz);
      Storage<S>::store(f + (long long)i * plane + s, (float)(fe - weight<D>(i) * rho0));
    }
  }
}

template <int D, typename S>
__global__ void gather_plane_kernel(const S *__restrict__ f, long long plane, int nx, int ny, int nz,
                                    double rho0, int parity, int q, double *__restrict__ out) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= plane) return;
  const int x = (int)(s % nx), y = (int)((s / nx) % ny), z = (int)(s / ((long long)nx * ny));
  const long long slot = logical_slot<D>(q, x, y, z, nx, ny, nz, plane, parity);
  out[s] = weight<D>(q) * rho0 + (double)Storage<S>::load(f + slot);
}

template <int D, typename S>
__global__ void scatter_plane_kernel(S *__restrict__ f, long long plane, int nx, int ny, int nz,
                                     double rho0, int parity, int q, const double *__restrict__ in) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= plane) return;
  const int x = (int)(s % nx), y = (int)((s / nx) % ny), z = (int)(s / ((long long)nx * ny));
  const long long slot = logical_slot<D>(q, x, y, z, nx, ny, nz, plane, parity);
  Storage<S>::store(f + slot, (float)(in[s] - weight<D>(q) * rho0));
}

template <int D, typename S>
__global__ void gather_sites_kernel(const S *__restrict__ f, long long plane, int nx, int ny, int nz,
                                    double rho0, int parity, const long long *__restrict__ sites,
                                    long long n, double *__restrict__ out) {
  constexpr int Q = Lat<D>::Q;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * Q) return;
  const long long k = t / Q;
  const int q = (int)(t % Q);
  const long long s = sites[k];
  if (s < 0 || s >= plane) {
    out[t] = __longlong_as_double(0x7ff8000000000000LL);  // NaN for an invalid site index
    return;
  }
  const int x = (int)(s % nx), y = (int)((s / nx) % ny), z = (int)(s / ((long long)nx * ny));
  out[t] = weight<D>(q) * rho0 + (double)Storage<S>::load(f + logical_slot<D>(q, x, y, z, nx, ny, nz, plane, parity));
}

inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename S>
cudaError_t init_typed(int D, void *f, long long plane, int nx, int ny, int nz, double rho0,
                       double ux, double uy, double uz, double amp, uint64_t seed, uint32_t site_base,
                       cudaStream_t s) {
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  S *p = static_cast<S *>(f);
  if (D == 19)
    init_kernel<19, S><<<blocks_for(plane, 256), 256, 0, s>>>(p, plane, nx, ny, nz, rho0, ux, uy, uz, amp, k0, k1,
                                                              site_base);
  else if (D == 3)
    init_kernel<3, S><<<blocks_for(plane, 256), 256, 0, s>>>(p, plane, nx, ny, nz, rho0, ux, uy, uz, amp, k0, k1,
                                                             site_base);
  else
    init_kernel<2, S><<<blocks_for(plane, 256), 256, 0, s>>>(p, plane, nx, ny, nz, rho0, ux, uy, 0.0, amp, k0, k1,
                                                             site_base);
  return cudaGetLastError();
}

template <typename S>
cudaError_t gather_typed(int D, int parity, const void *f, long long plane, int nx, int ny, int nz,
                         double rho0, int q, double *out, cudaStream_t s) {
  const S *p = static_cast<const S *>(f);
  if (D == 19)
    gather_plane_kernel<19, S><<<blocks_for(plane, 256), 256, 0, s>>>(p, plane, nx, ny, nz, rho0, parity, q, out);
  else if (D == 3)
    gather_plane_kernel<3, S><<<blocks_for(plane, 256), 256, 0, s>>>(p, plane, nx, ny, nz, rho0, parity, q, out);
  else
    gather_plane_kernel<2, S><<<blocks_for(plane, 256), 256, 0, s>>>(p, plane, nx, ny, nz, rho0, parity, q, out);
  return cudaGetLastError();
}

template <typename S>
cudaError_t scatter_typed(int D, int parity, void *f, long long plane, int nx, int ny, int nz,
                          double rho0, int q, const double *in, cudaStream_t s) {
  S *p = static_cast<S *>(f);
  if (D == 19)
    scatter_plane_kernel<19, S><<<blocks_for(plane, 256), 256, 0, s>>>(p, plane, nx, ny, nz, rho0, parity, q, in);
  else if (D == 3)
    scatter_plane_kernel<3, S><<<blocks_for(plane, 256), 256, 0, s>>>(p, plane, nx, ny, nz, rho0, parity, q, in);
  else
    scatter_plane_kernel<2, S><<<blocks_for(plane, 256), 256, 0, s>>>(p, plane, nx, ny, nz, rho0, parity, q, in);
  return cudaGetLastError();
}

template <typename S>
cudaError_t sites_typed(int D, int parity, const void *f, long long plane, int nx, int ny, int nz,
                        double rho0, const long long *sites, long long n, double *out, cudaStream_t s) {
  const S *p = static_cast<const S *>(f);
  const int Q = D == 3 ? 27 : (D == 19 ? 19 : 9);
  if (n == 0) return cudaSuccess;
  if (D == 19)
    gather_sites_kernel<19, S><<<blocks_for(n * Q, 256), 256, 0, s>>>(p, plane, nx, ny, nz, rho0, parity, sites, n, out);
  else if (D == 3)
    gather_sites_kernel<3, S><<<blocks_for(n * Q, 256), 256, 0, s>>>(p, plane, nx, ny, nz, rho0, parity, sites, n, out);
  else
    gather_sites_kernel<2, S><<<blocks_for(n * Q, 256), 256, 0, s>>>(p, plane, nx, ny, nz, rho0, parity, sites, n, out);
  return cudaGetLastError();
}

}  // namespace

size_t storage_bytes(int storage) { return storage == 0 ? 4 : 2; }

cudaError_t launch_init(int D, int storage, void *f, long long plane, int nx, int ny, int nz,
                        double rho0, double ux, double uy, double uz, double amp,
                        uint64_t perturb_seed, uint32_t site_base, cudaStream_t s) {
  if (storage == 0)
    return init_typed<float>(D, f, plane, nx, ny, nz, rho0, ux, uy, uz, amp, perturb_seed, site_base, s);
  if (storage == 1)
    return init_typed<__nv_bfloat16>(D, f, plane, nx, ny, nz, rho0, ux, uy, uz, amp, perturb_seed, site_base, s);
  return init_typed<__half>(D, f, plane, nx, ny, nz, rho0, ux, uy, uz, amp, perturb_seed, site_base, s);
}

cudaError_t launch_gather_plane(int D, int storage, int parity, const void *f, long long plane,
                                int nx, int ny, int nz, double rho0, int q, double *out,
                                cudaStream_t s) {
  if (storage == 0) return gather_typed<float>(D, parity, f, plane, nx, ny, nz, rho0, q, out, s);
  if (storage == 1) return gather_typed<__nv_bfloat16>(D, parity, f, plane, nx, ny, nz, rho0, q, out, s);
  return gather_typed<__half>(D, parity, f, plane, nx, ny, nz, rho0, q, out, s);
}

cudaError_t launch_scatter_plane(int D, int storage, int parity, void *f, long long plane, int nx,
                                 int ny, int nz, double rho0, int q, const double *in,
                                 cudaStream_t s) {
  if (storage == 0) return scatter_typed<float>(D, parity, f, plane, nx, ny, nz, rho0, q, in, s);
  if (storage == 1) return scatter_typed<__nv_bfloat16>(D, parity, f, plane, nx, ny, nz, rho0, q, in, s);
  return scatter_typed<__half>(D, parity, f, plane, nx, ny, nz, rho0, q, in, s);
}

cudaError_t launch_gather_sites(int D, int storage, int parity, const void *f, long long plane,
                                int nx, int ny, int nz, double rho0, const long long *sites,
                                long long n, double *out, cudaStream_t s) {
  if (storage == 0) return sites_typed<float>(D, parity, f, plane, nx, ny, nz, rho0, sites, n, out, s);
  if (storage == 1) return sites_typed<__nv_bfloat16>(D, parity, f, plane, nx, ny, nz, rho0, sites, n, out, s);
  return sites_typed<__half>(D, parity, f, plane, nx, ny, nz, rho0, sites, n, out, s);
}

// b_v of the device bases: product of the 1-D norms (1, 1/3, 2/9) over the tensor
// orders of mode v; the rotated D2Q9 pair 3, 4 has norm 2 * (2/9).
double mode_bnorm_lattice(int lattice, int v) {
  if (lattice == 2 && v >= 4 && v <= 6) return v == 4 ? 2.0 / 3.0 : (v == 5 ? 4.0 / 9.0 : 4.0 / 3.0);
  if (lattice == 3) {  // D3Q19, printed in Sec. II-C
    const double b[19] = {1.0,       1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 2.0 / 3.0, 4.0 / 3.0, 4.0 / 9.0,
                          1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 2.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 2.0 / 9.0,
                          2.0 / 9.0, 2.0 / 9.0, 2.0,       4.0 / 3.0, 4.0 / 9.0};
    return b[v];
  }
  return mode_bnorm(lattice == 0 ? 2 : 3, v);
}

float mode_tile_scale(int lattice, int v) {
  if (lattice == 3) return 1.0f;
  if (lattice == 2 && v >= 4 && v <= 6) return 1.0f;  // rotated; halved after the rotation back
  return lattice == 0 ? tile_scale<2>(v) : tile_scale<3>(v);
}

double mode_bnorm(int D, int v) {
  const double b1[3] = {1.0, 1.0 / 3.0, 2.0 / 9.0};
  if (D == 3) {
    const int t = d3q27_mode_tensor(v);
    return b1[t % 3] * b1[(t / 3) % 3] * b1[t / 9];
  }
  if (v == 3 || v == 4) return 2.0 * b1[2];
  const int t = d2q9_mode_tensor(v);
  return b1[t % 3] * b1[t / 3];
}

}  // namespace flbm
