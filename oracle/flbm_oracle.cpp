// Plain FP64 CPU oracle of the fluctuating orthogonal-central-moment lattice
// Boltzmann step (De Rosis & Zhou, "A fluctuating lattice Boltzmann formulation
// based on orthogonal central moments", arXiv:2602.16486).
//
// TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct definition
// that the CUDA path is checked against. Only the test suite, the smoke check
// and the benchmark's CPU-baseline leg may load it. It shares no code, header,
// table or constant with the CUDA library: every table below is typed in from
// the paper and every matrix is built densely from its definition.
//
// What it computes, in the paper's order (Sec. II, "Algorithm of computation"):
//   1. rho = sum_i f_i, rho*u = sum_i c_i f_i                      (Eq. macro)
//   2. eta_v ~ N(0,1) for the noisy modes                           (Eq. cm_collision)
//   3. k = T(u) f, T_vi = M_v(c_i - u)                              (Sec. II-B, Eq. k = T f)
//   4. k*_v = (1-L_v) k_v + L_v keq_v + I~_v phi_v eta_v            (Eq. cm_collision)
//      keq = (rho, 0, ..., 0)                                       (Sec. II-B / II-C)
//      phi_v = sqrt(rho kBT L_v (2-L_v) b_v / cs^2)                 (Eq. phi_general)
//   5-6. f* = T(u)^{-1} k*, by LU with partial pivoting             (Sec. II-B, f* = T^{-1} k*)
//   7. f_i(x + c_i, t+1) = f*_i(x, t), periodic                     (Eq. streaming)
//
// Readings where the paper is silent or garbled (each also listed in the design notes):
//   * D3Q27 basis vector M_15 is printed as cy^2 cz - cs^2 cy, which is not
//     orthogonal to M_3; it is read as cy^2 cz - cs^2 cz (restores the printed b_15).
//   * The D2Q9 equilibrium's fourth-order term is printed without its 1/(4 cs^8)
//     factor; the factor is restored (it is the one the D3Q27 formula carries).
//   * Hermite tensors of order 5 and 6 (used by the D3Q27 equilibrium) are not
//     defined in the paper; they are the standard Hermite tensors, built here by
//     the usual recursion that reproduces the printed orders 0-4.
//   * L (relaxation rates) is a user vector; entries for the conserved modes
//     (v <= D) are forced to 1 as the paper does. phi uses the local rho.
//   * The paper does not name its normal generator. Normals come from
//     Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) and the Box-Muller
//     transform (Box & Muller, 1958), keyed as described at normals_block().
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double CS2 = 1.0 / 3.0;  // lattice sound speed squared, cs = 1/sqrt(3)

// ---------------------------------------------------------------------------
// Lattices (Sec. II-B for D2Q9, Sec. II-C for D3Q27), velocities in the paper's
// order.
// ---------------------------------------------------------------------------
struct Lattice {
  int D;   // spatial dimension
  int Q;   // number of velocities
  int c[27][3];
  double w[27];
};

Lattice make_d2q9() {
  Lattice L{};
  L.D = 2;
  L.Q = 9;
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  for (int i = 0; i < 9; ++i) {
    L.c[i][0] = cx[i];
    L.c[i][1] = cy[i];
    L.c[i][2] = 0;
  }
  L.w[0] = 4.0 / 9.0;
  for (int i = 1; i <= 4; ++i) L.w[i] = 1.0 / 9.0;
  for (int i = 5; i <= 8; ++i) L.w[i] = 1.0 / 36.0;
  return L;
}

Lattice make_d3q27() {
  Lattice L{};
  L.D = 3;
  L.Q = 27;
  const int cx[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1,
                      -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
  const int cy[27] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0,
                      0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1};
  const int cz[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1,
                      1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1};
  for (int i = 0; i < 27; ++i) {
    L.c[i][0] = cx[i];
    L.c[i][1] = cy[i];
    L.c[i][2] = cz[i];
  }
  L.w[0] = 8.0 / 27.0;
  for (int i = 1; i <= 6; ++i) L.w[i] = 2.0 / 27.0;
  for (int i = 7; i <= 18; ++i) L.w[i] = 1.0 / 54.0;
  for (int i = 19; i <= 26; ++i) L.w[i] = 1.0 / 216.0;
  return L;
}

// D3Q19 (Sec. II-C, "Lattice-agnostic construction"): the rest velocity, the six axis
// velocities and the twelve face diagonals, weights 1/3, 1/18, 1/36. The paper lists the
// velocities by group only; they are taken in the order of the first 19 D3Q27 velocities.
Lattice make_d3q19() {
  const Lattice q27 = make_d3q27();
  Lattice L{};
  L.D = 3;
  L.Q = 19;
  for (int i = 0; i < 19; ++i)
    for (int a = 0; a < 3; ++a) L.c[i][a] = q27.c[i][a];
  L.w[0] = 1.0 / 3.0;
  for (int i = 1; i <= 6; ++i) L.w[i] = 1.0 / 18.0;
  for (int i = 7; i <= 18; ++i) L.w[i] = 1.0 / 36.0;
  return L;
}

// Lattice ids: 0 D2Q9, 1 D3Q27, 2 D3Q27 with the isotropic normal-stress modes (same
// velocities and weights as 1; see basis_d3q27_iso), 3 D3Q19.
const Lattice &lattice(int id) {
  static const Lattice d2q9 = make_d2q9();
  static const Lattice d3q27 = make_d3q27();
  static const Lattice d3q19 = make_d3q19();
  return id == 0 ? d2q9 : (id == 3 ? d3q19 : d3q27);
}

// ---------------------------------------------------------------------------
// Orthogonal bases M_v(c), evaluated at an arbitrary (possibly shifted) velocity.
// D2Q9: Sec. II-B orthogonal basis. D3Q27: Sec. II-C (Lauricella et al.) basis.
// ---------------------------------------------------------------------------
double basis_d2q9(int v, double x, double y) {
  const double s = CS2;
  switch (v) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return x * x + y * y - 2.0 * s;
    case 4: return x * x - y * y;
    case 5: return x * y;
    case 6: return (x * x - s) * y;
    case 7: return x * (y * y - s);
    case 8: return (x * x - s) * (y * y - s);
  }
  return 0.0;
}

double basis_d3q27(int v, double x, double y, double z) {
  const double s = CS2, s2 = CS2 * CS2, s3 = CS2 * CS2 * CS2;
  switch (v) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return x * x - s;
    case 5: return y * y - s;
    case 6: return z * z - s;
    case 7: return x * y;
    case 8: return x * z;
    case 9: return y * z;
    case 10: return x * x * y - s * y;
    case 11: return x * x * z - s * z;
    case 12: return x * y * y - s * x;
    case 13: return x * z * z - s * x;
    case 14: return y * z * z - s * y;
    case 15: return y * y * z - s * z;  // printed "- cs^2 c_y": read as "- cs^2 c_z"
    case 16: return x * y * z;
    case 17: return x * x * y * y - s * (x * x + y * y) + s2;
    case 18: return x * x * z * z - s * (x * x + z * z) + s2;
    case 19: return y * y * z * z - s * (y * y + z * z) + s2;
    case 20: return x * y * z * z - s * x * y;
    case 21: return x * y * y * z - s * x * z;
    case 22: return x * x * y * z - s * y * z;
    case 23: return x * x * y * z * z - s * (x * x * y + y * z * z) + s2 * y;
    case 24: return x * x * y * y * z - s * (x * x * z + y * y * z) + s2 * z;
    case 25: return x * y * y * z * z - s * (x * y * y + x * z * z) + s2 * x;
    case 26:
      return x * x * y * y * z * z - s * (x * x * y * y + x * x * z * z + y * y * z * z) +
             s2 * (x * x + y * y + z * z) - s3;
  }
  return 0.0;
}

// Isotropic variant of the D3Q27 basis (the reading that resolves the anisotropy of
// Sec. II-C, where the normal-stress modes 4-6 relax at rate 1 while the shear modes 7-9
// relax at omega): modes 4-6 are replaced by the trace and two deviators of the same
// second-order space,
//   M4' = M4 + M5 + M6,  M5' = M4 - M5,  M6' = M4 + M5 - 2 M6,
// which stay mutually orthogonal (M4..M6 have equal norms 2/9), with norms 2/3, 4/9, 4/3.
// Relaxing M5', M6' at the shear rate gives one viscosity for every shear direction; M4'
// carries the bulk rate. Every other mode is the paper's.
double basis_d3q27_iso(int v, double x, double y, double z) {
  const double a = basis_d3q27(4, x, y, z), b = basis_d3q27(5, x, y, z), c = basis_d3q27(6, x, y, z);
  switch (v) {
    case 4: return a + b + c;
    case 5: return a - b;
    case 6: return a + b - 2.0 * c;
  }
  return basis_d3q27(v, x, y, z);
}

// D3Q19 orthogonal basis as printed in Sec. II-C ("Lattice-agnostic construction");
// c2 = |c|^2.
double basis_d3q19(int v, double x, double y, double z) {
  const double c2 = x * x + y * y + z * z;
  switch (v) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return c2 - 1.0;
    case 5: return 3.0 * x * x - c2;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return y * z;
    case 9: return x * z;
    case 10: return x * (3.0 * c2 - 5.0);
    case 11: return y * (3.0 * c2 - 5.0);
    case 12: return z * (3.0 * c2 - 5.0);
    case 13: return x * (y * y - z * z);
    case 14: return y * (z * z - x * x);
    case 15: return z * (x * x - y * y);
    case 16: return 3.0 * c2 * c2 - 6.0 * c2 + 1.0;
    case 17: return (2.0 * c2 - 3.0) * (3.0 * x * x - c2);
    case 18: return (2.0 * c2 - 3.0) * (y * y - z * z);
  }
  return 0.0;
}

double basis(int lat, int v, const double cbar[3]) {
  if (lat == 0) return basis_d2q9(v, cbar[0], cbar[1]);
  if (lat == 3) return basis_d3q19(v, cbar[0], cbar[1], cbar[2]);
  if (lat == 2) return basis_d3q27_iso(v, cbar[0], cbar[1], cbar[2]);
  return basis_d3q27(v, cbar[0], cbar[1], cbar[2]);
}

// T_vi(u) = M_v(c_i - u): the basis with every c replaced by c-bar (Sec. II-B).
void build_T(int lat, const double u[3], std::vector<double> &T) {
  const Lattice &L = lattice(lat);
  T.assign(L.Q * L.Q, 0.0);
  for (int i = 0; i < L.Q; ++i) {
    const double cb[3] = {L.c[i][0] - u[0], L.c[i][1] - u[1], L.c[i][2] - u[2]};
    for (int v = 0; v < L.Q; ++v) T[v * L.Q + i] = basis(lat, v, cb);
  }
}

// b_v = sum_i w_i M_vi^2 (Sec. II-A, below Eq. Xi_pop).
double bnorm(int lat, int v) {
  const Lattice &L = lattice(lat);
  double b = 0.0;
  for (int i = 0; i < L.Q; ++i) {
    const double c[3] = {double(L.c[i][0]), double(L.c[i][1]), double(L.c[i][2])};
    const double m = basis(lat, v, c);
    b += L.w[i] * m * m;
  }
  return b;
}

// Solve A x = b (n x n, row-major) by Gaussian elimination with partial pivoting.
// Returns false if a zero pivot is met.
bool lu_solve(int n, std::vector<double> A, std::vector<double> &x, const double *b) {
  std::vector<double> r(b, b + n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[p * n + k])) p = i;
    if (A[p * n + k] == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
      std::swap(r[k], r[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double m = A[i * n + k] / A[k * n + k];
      A[i * n + k] = 0.0;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= m * A[k * n + j];
      r[i] -= m * r[k];
    }
  }
  x.assign(n, 0.0);
  for (int k = n - 1; k >= 0; --k) {
    double s = r[k];
    for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * x[j];
    x[k] = s / A[k * n + k];
  }
  return true;
}

// ---------------------------------------------------------------------------
// Hermite tensors (Sec. II-B, Eq. feq and the definitions of H^(0..4) that follow).
// idx holds the n Cartesian indices (0=x, 1=y, 2=z). The recursion
//   H^(n+1)_{a,B} = c_a H^(n)_B - cs^2 sum_k delta_{a,B_k} H^(n-1)_{B \ B_k}
// reproduces the printed H^(0)..H^(4) and defines the orders 5 and 6 that the
// D3Q27 equilibrium uses.
// ---------------------------------------------------------------------------
double hermite(const int *c, const int *idx, int n) {
  if (n == 0) return 1.0;
  if (n == 1) return double(c[idx[0]]);
  const int a = idx[0];
  const int *B = idx + 1;
  double h = double(c[a]) * hermite(c, B, n - 1);
  int rest[8];
  for (int k = 0; k < n - 1; ++k) {
    if (B[k] != a) continue;
    int m = 0;
    for (int j = 0; j < n - 1; ++j)
      if (j != k) rest[m++] = B[j];
    h -= CS2 * hermite(c, rest, n - 2);
  }
  return h;
}

// Convenience: Hermite tensor addressed by a string such as "xxyzz".
double H(const int *c, const char *s) {
  int idx[8];
  int n = 0;
  for (; s[n]; ++n) idx[n] = s[n] - 'x';
  return hermite(c, idx, n);
}

// Equilibrium populations, term by term as printed: D2Q9 Sec. II-B (fourth-order
// Hermite expansion, with its 1/(4 cs^8) factor restored), D3Q27 Sec. II-C
// (sixth-order expansion).
void feq(int lat, double rho, const double u[3], double *f) {
  const Lattice &L = lattice(lat);
  if (lat == 3) {
    // D3Q19: the printed fourth-order populations do not conserve mass as transcribed
    // (their sum is rho - 2 rho u^2 / 3 + O(u^4)). The equilibrium is taken as the one
    // the paper states they project to: the populations whose central moments are
    // k^eq = (rho, 0, ..., 0), f^eq = T(u)^{-1} k^eq.
    std::vector<double> T;
    build_T(lat, u, T);
    std::vector<double> keq(size_t(L.Q), 0.0), x;
    keq[0] = rho;
    if (!lu_solve(L.Q, T, x, keq.data()))
      for (int i = 0; i < L.Q; ++i) f[i] = NAN;
    else
      for (int i = 0; i < L.Q; ++i) f[i] = x[size_t(i)];
    return;
  }
  const double s2 = CS2, s4 = CS2 * CS2, s6 = s4 * CS2, s8 = s4 * s4, s10 = s8 * CS2,
               s12 = s6 * s6;
  const double ux = u[0], uy = u[1], uz = (lat == 0 ? 0.0 : u[2]);
  for (int i = 0; i < L.Q; ++i) {
    const int *c = L.c[i];
    double cu = c[0] * ux + c[1] * uy + c[2] * uz;
    double h2uu = 0.0;
    const double uv[3] = {ux, uy, uz};
    for (int a = 0; a < L.D; ++a)
      for (int b = 0; b < L.D; ++b) {
        int idx[2] = {a, b};
        h2uu += hermite(c, idx, 2) * uv[a] * uv[b];
      }
    double t = 1.0 + cu / s2 + h2uu / (2.0 * s4);
    if (lat == 0) {
      t += (H(c, "xxy") * ux * ux * uy + H(c, "xyy") * ux * uy * uy) / (2.0 * s6);
      t += H(c, "xxyy") * ux * ux * uy * uy / (4.0 * s8);
    } else {
      t += (H(c, "xxy") * ux * ux * uy + H(c, "xxz") * ux * ux * uz + H(c, "xyy") * ux * uy * uy +
            H(c, "xzz") * ux * uz * uz + H(c, "yzz") * uy * uz * uz + H(c, "yyz") * uy * uy * uz +
            2.0 * H(c, "xyz") * ux * uy * uz) /
           (2.0 * s6);
      t += (H(c, "xxyy") * ux * ux * uy * uy + H(c, "xxzz") * ux * ux * uz * uz +
            H(c, "yyzz") * uy * uy * uz * uz +
            2.0 * (H(c, "xyzz") * ux * uy * uz * uz + H(c, "xyyz") * ux * uy * uy * uz +
                   H(c, "xxyz") * ux * ux * uy * uz)) /
           (4.0 * s8);
      t += (H(c, "xxyzz") * ux * ux * uy * uz * uz + H(c, "xxyyz") * ux * ux * uy * uy * uz +
            H(c, "xyyzz") * ux * uy * uy * uz * uz) /
           (4.0 * s10);
      t += H(c, "xxyyzz") * ux * ux * uy * uy * uz * uz / (8.0 * s12);
    }
    f[i] = L.w[i] * rho * t;
  }
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): ten rounds of the 4x32 Philox S-box with the Weyl key
// schedule, multipliers and key increments as published there.
// ---------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0 = uint64_t(M0) * x[0];
    const uint64_t p1 = uint64_t(M1) * x[2];
    const uint32_t hi0 = uint32_t(p0 >> 32), lo0 = uint32_t(p0);
    const uint32_t hi1 = uint32_t(p1 >> 32), lo1 = uint32_t(p1);
    const uint32_t y0 = hi1 ^ x[1] ^ k0;
    const uint32_t y2 = hi0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = lo1;
    x[2] = y2;
    x[3] = lo0;
    k0 += W0;
    k1 += W1;
  }
  for (int j = 0; j < 4; ++j) out[j] = x[j];
}

// 23-bit uniform in the open interval (0,1): u = (floor(w / 2^9) + 1/2) * 2^-23.
double uniform01(uint32_t w) { return (double(w >> 9) + 0.5) * 0x1p-23; }

// Four standard normals from one Philox block.
//   key     = (seed mod 2^32, seed div 2^32)
//   counter = (site, step mod 2^32, step div 2^32, tag * 2^16 + blk)
// site = x + Nx (y + Ny z); tag 0 = collision noise, tag 1 = initial density
// perturbation. Words (w0,w1) and (w2,w3) each give one Box-Muller pair:
//   r = sqrt(-2 ln u_a), z_a = r cos(2 pi u_b), z_b = r sin(2 pi u_b).
void normals_block(uint64_t seed, uint64_t step, uint32_t site, uint32_t tag, uint32_t blk,
                   double z[4]) {
  const uint32_t key[2] = {uint32_t(seed), uint32_t(seed >> 32)};
  const uint32_t ctr[4] = {site, uint32_t(step), uint32_t(step >> 32), (tag << 16) | blk};
  uint32_t w[4];
  philox4x32_10(ctr, key, w);
  for (int p = 0; p < 2; ++p) {
    const double ua = uniform01(w[2 * p]);
    const double ub = uniform01(w[2 * p + 1]);
    const double r = std::sqrt(-2.0 * std::log(ua));
    z[2 * p] = r * std::cos(2.0 * M_PI * ub);
    z[2 * p + 1] = r * std::sin(2.0 * M_PI * ub);
  }
}

// eta_v for one site and step: noisy mode v (v > D) uses normal n = v - D - 1,
// i.e. block n / 4, slot n % 4. Entries of conserved modes are set to 0.
void site_eta(int lat, uint64_t seed, uint64_t step, uint32_t site, double *eta) {
  const Lattice &L = lattice(lat);
  double z[4];
  int have = -1;
  for (int v = 0; v < L.Q; ++v) {
    if (v <= L.D) {
      eta[v] = 0.0;
      continue;
    }
    const int n = v - L.D - 1;
    if (n / 4 != have) {
      have = n / 4;
      normals_block(seed, step, site, 0u, uint32_t(have), z);
    }
    eta[v] = z[n % 4];
  }
}

// One site's collision (Eq. cm_collision with Eq. phi_general). eta holds the
// normals of the noisy modes (I~_v = 1 for v > D: Sec. II-B lists I~ =
// diag[0,0,0,1,...,1] for D2Q9 and Sec. II-C lists I~_{0-3} = 0, I~_{4-26} = 1).
// model 0: the central-moment scheme, k = T(u) f with k^eq = (rho, 0, ..., 0).
// model 1: its raw-moment counterpart, T = M and N = I (Sec. II-C names this choice as the
// raw-moment form of the same scheme): k = M f, k^eq = M f^eq(rho, u), the same
// relaxation, noise amplitudes and normals; with a uniform rate Lambda = omega I it is the
// fluctuating BGK scheme of Sec. II-A (relaxation omega (f^eq - f), noise zeta_i of
// Eq. Xi_pop in the rest-frame basis).
bool collide_site(int lat, const double *f, const double *lambda, double kBT, const double *eta,
                  double *fstar, double *k_out, int model = 0) {
  const Lattice &L = lattice(lat);
  const int Q = L.Q;
  double rho = 0.0, j[3] = {0, 0, 0};
  for (int i = 0; i < Q; ++i) {
    rho += f[i];
    for (int a = 0; a < 3; ++a) j[a] += L.c[i][a] * f[i];
  }
  const double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
  std::vector<double> T;
  const double zero[3] = {0.0, 0.0, 0.0};
  build_T(lat, model == 1 ? zero : u, T);  // raw moments: the unshifted basis M = T(0)
  std::vector<double> k(Q, 0.0), kstar(Q, 0.0), keqv(Q, 0.0);
  for (int v = 0; v < Q; ++v)
    for (int i = 0; i < Q; ++i) k[v] += T[v * Q + i] * f[i];
  if (k_out)
    for (int v = 0; v < Q; ++v) k_out[v] = k[v];
  if (model == 1) {
    double fe[27];
    feq(lat, rho, u, fe);
    for (int v = 0; v < Q; ++v)
      for (int i = 0; i < Q; ++i) keqv[v] += T[v * Q + i] * fe[i];
  } else {
    keqv[0] = rho;
  }
  for (int v = 0; v < Q; ++v) {
    const double lam = (v <= L.D) ? 1.0 : lambda[v];
    const double keq = keqv[v];
    const double noisy = (v > L.D) ? 1.0 : 0.0;
    double phi = 0.0;
    if (noisy != 0.0 && kBT != 0.0) phi = std::sqrt(rho * kBT * lam * (2.0 - lam) * bnorm(lat, v) / CS2);
    kstar[v] = (1.0 - lam) * k[v] + lam * keq + noisy * phi * eta[v];
  }
  std::vector<double> x;
  const bool ok = lu_solve(Q, T, x, kstar.data());
  for (int i = 0; i < Q; ++i) fstar[i] = ok ? x[i] : NAN;
  return ok;
}

int64_t nsites(const int64_t dims[3]) { return dims[0] * dims[1] * dims[2]; }

}  // namespace

// ===========================================================================
// C entry points (loaded by the Python test helpers through ctypes).
// Populations are logical, FP64, laid out [q][z][y][x] with x fastest.
// ===========================================================================
extern "C" {

int oracle_q(int lat) { return lattice(lat).Q; }

// Velocities (Q x 3, int), weights (Q) and computed norms b_v (Q).
void oracle_tables(int lat, int *c, double *w, double *b) {
  const Lattice &L = lattice(lat);
  for (int i = 0; i < L.Q; ++i) {
    for (int a = 0; a < 3; ++a) c[i * 3 + a] = L.c[i][a];
    w[i] = L.w[i];
    b[i] = bnorm(lat, i);
  }
}

// Basis value M_v(cbar) at an arbitrary point.
double oracle_basis(int lat, int v, const double *cbar) { return basis(lat, v, cbar); }

// Dense shifted transform T(u), Q x Q row-major (row = mode v, column = velocity i).
void oracle_T(int lat, const double *u, double *T_out) {
  std::vector<double> T;
  build_T(lat, u, T);
  std::memcpy(T_out, T.data(), sizeof(double) * T.size());
}

// Hermite tensor of order n with Cartesian indices idx[0..n-1] at velocity c.
double oracle_hermite(const int *c, const int *idx, int n) { return hermite(c, idx, n); }

void oracle_feq(int lat, double rho, const double *u, double *f) { feq(lat, rho, u, f); }

void oracle_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
  philox4x32_10(ctr, key, out);
}

double oracle_uniform(uint32_t w) { return uniform01(w); }

void oracle_normals_block(uint64_t seed, uint64_t step, uint32_t site, uint32_t tag, uint32_t blk,
                          double *z) {
  normals_block(seed, step, site, tag, blk, z);
}

void oracle_site_eta(int lat, uint64_t seed, uint64_t step, uint32_t site, double *eta) {
  site_eta(lat, seed, step, site, eta);
}

// Collision of one site with given normals (eta[v] for the noisy modes). k_out
// (optional, may be null) receives the pre-collision central moments.
int oracle_collide_site(int lat, const double *f, const double *lambda, double kBT,
                        const double *eta, double *fstar, double *k_out) {
  return collide_site(lat, f, lambda, kBT, eta, fstar, k_out) ? 0 : 1;
}

// As oracle_collide_site for collision model `model` (0 central moments, 1 raw moments).
int oracle_collide_site_model(int lat, int model, const double *f, const double *lambda, double kBT,
                              const double *eta, double *fstar, double *k_out) {
  return collide_site(lat, f, lambda, kBT, eta, fstar, k_out, model) ? 0 : 1;
}

// Initial state: rho(x) = rho0 (1 + amp (2U - 1)), U = uniform of word 0 of the
// tag-1 Philox block (counter (site, 0, 0, 2^16)) under key perturb_seed;
// f = feq(rho(x), u0).
void oracle_init_uniform(int lat, const int64_t *dims, double rho0, const double *u0, double amp,
                         uint64_t perturb_seed, double *f) {
  const Lattice &L = lattice(lat);
  const int64_t N = nsites(dims);
  for (int64_t s = 0; s < N; ++s) {
    double rho = rho0;
    if (amp != 0.0) {
      const uint32_t key[2] = {uint32_t(perturb_seed), uint32_t(perturb_seed >> 32)};
      const uint32_t ctr[4] = {uint32_t(s), 0u, 0u, 1u << 16};
      uint32_t w[4];
      philox4x32_10(ctr, key, w);
      rho = rho0 * (1.0 + amp * (2.0 * uniform01(w[0]) - 1.0));
    }
    double fe[27];
    feq(lat, rho, u0, fe);
    for (int i = 0; i < L.Q; ++i) f[i * N + s] = fe[i];
  }
}

// Advance f (in place) by nsteps time steps, numbering them step0, step0+1, ...
// Each step: collide every site, push-stream into a second lattice, swap.
// threads <= 0 uses the OpenMP default. Returns the number of sites whose
// collision matrix was singular (0 normally).
int64_t oracle_run_model(int lat, int model, const int64_t *dims, const double *lambda, double kBT,
                         uint64_t seed, uint64_t step0, int64_t nsteps, double *f, int threads) {
  const Lattice &L = lattice(lat);
  const int Q = L.Q;
  const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
  const int64_t N = nx * ny * nz;
  std::vector<double> g(size_t(Q) * N);
  int64_t bad = 0;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  for (int64_t s = 0; s < nsteps; ++s) {
    const uint64_t step = step0 + uint64_t(s);
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t site = 0; site < N; ++site) {
      const int64_t x = site % nx, y = (site / nx) % ny, z = site / (nx * ny);
      double fl[27], fs[27], eta[27];
      for (int i = 0; i < Q; ++i) fl[i] = f[i * N + site];
      for (int v = 0; v < Q; ++v) eta[v] = 0.0;
      if (kBT != 0.0) site_eta(lat, seed, step, uint32_t(site), eta);
      if (!collide_site(lat, fl, lambda, kBT, eta, fs, nullptr, model)) ++bad;
      for (int i = 0; i < Q; ++i) {
        const int64_t xd = ((x + L.c[i][0]) % nx + nx) % nx;
        const int64_t yd = ((y + L.c[i][1]) % ny + ny) % ny;
        const int64_t zd = ((z + L.c[i][2]) % nz + nz) % nz;
        g[i * N + (zd * ny + yd) * nx + xd] = fs[i];
      }
    }
    std::memcpy(f, g.data(), sizeof(double) * g.size());
  }
  return bad;
}

// The central-moment scheme (model 0).
int64_t oracle_run(int lat, const int64_t *dims, const double *lambda, double kBT, uint64_t seed,
                   uint64_t step0, int64_t nsteps, double *f, int threads) {
  return oracle_run_model(lat, 0, dims, lambda, kBT, seed, step0, nsteps, f, threads);
}

// Statistics of the state f (pre-collision): out layout (doubles)
//   [0] mass = sum rho      [1..3] sum j
//   [4..6] mean u_a         [7..12] mean u_a u_b (xx, yy, zz, xy, xz, yz)
//   [13 .. 13+Q) mean k_v   [13+Q .. 13+Q+Q*Q) mean k_v k_w (row-major)
//   [13+Q+Q*Q] number of sites with a non-finite rho, u or k
// k_v are the central moments T(u(x)) f(x) at each site.
void oracle_stats(int lat, const int64_t *dims, const double *f, double *out) {
  const Lattice &L = lattice(lat);
  const int Q = L.Q;
  const int64_t N = nsites(dims);
  const int nout = 13 + Q + Q * Q + 1;
  for (int i = 0; i < nout; ++i) out[i] = 0.0;
  std::vector<double> T;
  for (int64_t site = 0; site < N; ++site) {
    double rho = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
      const double fi = f[i * N + site];
      rho += fi;
      for (int a = 0; a < 3; ++a) j[a] += L.c[i][a] * fi;
    }
    const double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    build_T(lat, u, T);
    double k[27];
    bool finite = std::isfinite(rho) && std::isfinite(u[0]) && std::isfinite(u[1]) &&
                  std::isfinite(u[2]);
    for (int v = 0; v < Q; ++v) {
      k[v] = 0.0;
      for (int i = 0; i < Q; ++i) k[v] += T[v * Q + i] * f[i * N + site];
      finite = finite && std::isfinite(k[v]);
    }
    if (!finite) {
      out[13 + Q + Q * Q] += 1.0;
      continue;
    }
    out[0] += rho;
    for (int a = 0; a < 3; ++a) {
      out[1 + a] += j[a];
      out[4 + a] += u[a];
    }
    out[7] += u[0] * u[0];
    out[8] += u[1] * u[1];
    out[9] += u[2] * u[2];
    out[10] += u[0] * u[1];
    out[11] += u[0] * u[2];
    out[12] += u[1] * u[2];
    for (int v = 0; v < Q; ++v) {
      out[13 + v] += k[v];
      for (int w = 0; w < Q; ++w) out[13 + Q + v * Q + w] += k[v] * k[w];
    }
  }
  const double inv = 1.0 / double(N);
  for (int i = 4; i < 13 + Q + Q * Q; ++i) out[i] *= inv;
}

}  // extern "C"
