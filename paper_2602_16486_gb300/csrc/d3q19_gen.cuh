// GENERATED by gen_d3q19.py from the D3Q19 basis of Sec. II-C ("Lattice-agnostic
// construction and the D3Q19 example"); do not edit. See the generator for the algebra.
#pragma once

#include "vec.cuh"

namespace flbm {

// r_v = sum_i M_vi d_i (r_0 = rho - rho0; r_1..3 = j).
template <typename T>
__device__ __forceinline__ void d3q19_raw(const T (&f)[19], T (&r)[19]) {
  const T f0 = f[0];
  const T f1 = f[1];
  const T f2 = f[2];
  const T f3 = f[3];
  const T f4 = f[4];
  const T f5 = f[5];
  const T f6 = f[6];
  const T f7 = f[7];
  const T f8 = f[8];
  const T f9 = f[9];
  const T f10 = f[10];
  const T f11 = f[11];
  const T f12 = f[12];
  const T f13 = f[13];
  const T f14 = f[14];
  const T f15 = f[15];
  const T f16 = f[16];
  const T f17 = f[17];
  const T f18 = f[18];
  const T a0 = vadd(f15, f16);
  const T a1 = vadd(a0, f5);
  const T a2 = vadd(f6, f7);
  const T a3 = vadd(f10, f9);
  const T a4 = vadd(a3, f17);
  const T a5 = vadd(f11, f12);
  const T a6 = vadd(a5, f18);
  const T a7 = vadd(f13, f14);
  const T a8 = vadd(a7, f8);
  const T a9 = vadd(vadd(a4, a6), a8);
  const T a10 = vmul(rat<T>(-1.0), f14);
  const T a11 = vmul(rat<T>(-1.0), f8);
  const T a12 = vadd(a11, f7);
  const T a13 = vmul(rat<T>(-1.0), f12);
  const T a14 = vadd(a13, f11);
  const T a15 = vadd(a14, f13);
  const T a16 = vmul(rat<T>(-1.0), f3);
  const T a17 = vadd(a3, f4);
  const T a18 = vmul(rat<T>(-1.0), f15);
  const T a19 = vmul(rat<T>(-1.0), f17);
  const T a20 = vadd(a19, f18);
  const T a21 = vmul(rat<T>(-1.0), f7);
  const T a22 = vadd(a11, a21);
  const T a23 = vadd(vadd(vadd(a18, a20), a22), f16);
  const T a24 = vmul(rat<T>(-1.0), f6);
  const T a25 = vadd(a24, a5);
  const T a26 = vmul(rat<T>(-1.0), f18);
  const T a27 = vmul(rat<T>(-1.0), f13);
  const T a28 = vadd(a10, a27);
  const T a29 = vadd(vadd(a19, a26), a28);
  const T a30 = vadd(a9, f7);
  const T a31 = vmul(rat<T>(2.0), f2);
  const T a32 = vmul(rat<T>(2.0), f1);
  const T a33 = vadd(a32, f8);
  const T a34 = vsub(f7, f5);
  const T a35 = vsub(vadd(a16, a3), f4);
  const T a36 = vfma(rat<T>(-2.0), f18, vfma(rat<T>(-2.0), f17, vfma(rat<T>(-2.0), f16, vmul(rat<T>(-2.0), f15))));
  const T a37 = vadd(a17, f3);
  const T a38 = vmul(rat<T>(-1.0), f11);
  const T a39 = vadd(a10, f8);
  const T a40 = vadd(vadd(vadd(a13, a27), a38), a39);
  const T a41 = vsub(f10, f9);
  const T a42 = vmul(rat<T>(-1.0), f16);
  const T a43 = vadd(a42, f15);
  const T a44 = vadd(a27, f14);
  const T a45 = vmul(rat<T>(-1.0), a31);
  const T a46 = vadd(a21, a41);
  const T a47 = vmul(rat<T>(-2.0), f4);
  const T a48 = vmul(rat<T>(2.0), f3);
  const T a49 = vmul(rat<T>(2.0), f6);
  const T a50 = vfma(rat<T>(-2.0), f5, a0);
  const T a51 = vsub(a45, a32);
  const T a52 = vadd(a2, f5);
  r[0] = vadd(vadd(vadd(vadd(vadd(vadd(vadd(a1, a2), a9), f0), f1), f2), f3), f4);
  r[1] = vsub(vsub(vadd(vadd(vadd(vadd(a10, a12), a15), f1), f9), f10), f2);
  r[2] = vsub(vsub(vmul(rat<T>(-1.0), a16), a17), a23);
  r[3] = vadd(vadd(a1, a25), a29);
  r[4] = vsub(vadd(a0, a30), f0);
  r[5] = vadd(vadd(vadd(vadd(vadd(vadd(a25, a31), a33), a34), a35), a36), a7);
  r[6] = vadd(vadd(vadd(a24, a34), a37), a40);
  r[7] = vadd(a12, a41);
  r[8] = vadd(a20, a43);
  r[9] = vadd(a14, a44);
  r[10] = vsub(vsub(vsub(vsub(vsub(vmul(rat<T>(-1.0), a33), a38), a44), a45), a46), f12);
  r[11] = vsub(vsub(vsub(vmul(rat<T>(-1.0), a23), a3), a47), a48);
  r[12] = vadd(vadd(vadd(a29, a49), a5), a50);
  r[13] = vsub(vsub(vmul(rat<T>(-1.0), a15), a39), a46);
  r[14] = vadd(vadd(vadd(a22, a26), a4), a43);
  r[15] = vadd(vadd(vadd(vadd(a18, a28), a42), a6), f17);
  r[16] = vsub(vsub(vadd(vadd(vadd(vadd(a30, a47), a50), a51), f0), a48), a49);
  r[17] = vadd(vadd(vadd(vadd(vadd(a36, a37), a5), a51), a52), a8);
  r[18] = vadd(vadd(a35, a40), a52);
}

// Central moments k_v, v = 4..18, in place over the raw moments r (r_0..3 are not read:
// the shift uses r_0 = rho and r_a = rho u_a).
template <typename T>
__device__ __forceinline__ void d3q19_central(T (&r)[19], T rho, T ux, T uy, T uz) {
  const T x4 = r[4]; const T x5 = r[5]; const T x6 = r[6]; const T x7 = r[7]; const T x8 = r[8]; const T x9 = r[9]; const T x10 = r[10]; const T x11 = r[11]; const T x12 = r[12]; const T x13 = r[13]; const T x14 = r[14]; const T x15 = r[15]; const T x16 = r[16]; const T x17 = r[17]; const T x18 = r[18];
  const T b0 = vmul(ux, ux);
  const T b1 = vmul(uy, uy);
  const T b2 = vmul(uz, uz);
  const T b3 = vadd(b1, b2);
  const T b4 = vmul(rat<T>(2.0), b0);
  const T b5 = vmul(ux, uy);
  const T b6 = vmul(uy, uz);
  const T b7 = vmul(ux, uz);
  const T b8 = vmul(rat<T>(6.0), ux);
  const T b9 = vmul(rat<T>(2.0), ux);
  const T b10 = vmul(rat<T>(-1.0), b9);
  const T b11 = vmul(rat<T>(6.0), uy);
  const T b12 = vmul(rat<T>(-1.0), b11);
  const T b13 = vmul(rat<T>(6.0), uz);
  const T b14 = vmul(rat<T>(-1.0), b13);
  const T b15 = vmul(rat<T>(-1.0), b8);
  const T b16 = vmul(rat<T>(2.0), uy);
  const T b17 = vmul(rat<T>(2.0), uz);
  const T b18 = vmul(rat<T>(0.5), uy);
  const T b19 = vmul(rat<T>(0.5), uz);
  const T b20 = vmul(rat<T>(4.0), b0);
  const T b21 = vmul(vmul(vmul(ux, ux), ux), ux);
  const T b22 = vmul(rat<T>(4.0), b1);
  const T b23 = vmul(vmul(vmul(uy, uy), uy), uy);
  const T b24 = vmul(rat<T>(4.0), b2);
  const T b25 = vmul(vmul(vmul(uz, uz), uz), uz);
  const T b26 = vmul(rat<T>(18.0), b0);
  const T b27 = vmul(b1, b2);
  const T b28 = vmul(rat<T>(6.0), b1);
  const T b29 = vmul(rat<T>(6.0), b2);
  const T b30 = vmul(rat<T>(-4.0), ux);
  const T b31 = vmul(b0, b28);
  const T b32 = vsub(vfma(rat<T>(6.0), b23, vmul(rat<T>(1.6666666666666667), b1)), vmul(b0, b29));
  const T b33 = vmul(rat<T>(4.666666666666667), b1);
  const T b34 = vmul(rat<T>(4.666666666666667), b2);
  const T b35 = vmul(rat<T>(8.0), b5);
  const T b36 = vmul(rat<T>(8.0), b7);
  const T b37 = vmul(rat<T>(0.6666666666666666), uy);
  const T b38 = vmul(rat<T>(0.6666666666666666), uz);
  const T bp0 = vsub(vmul(rat<T>(-1.0), b0), b3);
  const T bp1 = vsub(b3, b4);
  const T bp2 = vsub(b2, b1);
  const T bp3 = vmul(rat<T>(-1.0), b5);
  const T bp4 = vmul(rat<T>(-1.0), b6);
  const T bp5 = vmul(rat<T>(-1.0), b7);
  const T bp6 = vadd(vadd(vmul(rat<T>(6.0), vmul(vmul(ux, ux), ux)), vmul(b1, b8)), vmul(b2, b8));
  const T bp7 = vmul(rat<T>(-5.0), ux);
  const T bp11 = vadd(vadd(vmul(rat<T>(6.0), vmul(vmul(uy, uy), uy)), vmul(b0, b11)), vmul(b11, b2));
  const T bp12 = vmul(rat<T>(-5.0), uy);
  const T bp14 = vmul(rat<T>(-3.0), uy);
  const T bp17 = vadd(vadd(vmul(rat<T>(6.0), vmul(vmul(uz, uz), uz)), vmul(b0, b13)), vmul(b1, b13));
  const T bp18 = vmul(rat<T>(-5.0), uz);
  const T bp20 = vmul(rat<T>(3.0), uz);
  const T bp23 = vsub(vmul(b1, b9), vmul(b2, b9));
  const T bp24 = vmul(rat<T>(-1.0), ux);
  const T bp25 = vmul(rat<T>(-1.0), b16);
  const T bp27 = vsub(vmul(rat<T>(2.0), vmul(b2, uy)), vmul(b4, uy));
  const T bp31 = vmul(rat<T>(-1.0), b17);
  const T bp32 = vsub(vmul(b4, uz), vmul(b1, b17));
  const T bp33 = vmul(rat<T>(-1.0), b19);
  const T bp37 = vsub(vsub(vsub(vsub(vsub(vfma(rat<T>(-9.0), b25, vfma(rat<T>(-9.0), b23, vfma(rat<T>(-9.0), b21, vmul(rat<T>(-18.0), b27)))), vmul(b1, b26)), vmul(b2, b26)), b20), b22), b24);
  const T bp38 = vfma(rat<T>(10.0), b2, vfma(rat<T>(10.0), b1, vmul(rat<T>(10.0), b0)));
  const T bp39 = vfma(rat<T>(-2.0), b2, vfma(rat<T>(-2.0), b1, b20));
  const T bp40 = vsub(b28, b29);
  const T bp41 = vmul(rat<T>(24.0), b5);
  const T bp42 = vmul(rat<T>(24.0), b6);
  const T bp43 = vmul(rat<T>(24.0), b7);
  const T bp45 = vmul(rat<T>(-4.0), uy);
  const T bp46 = vmul(rat<T>(-4.0), uz);
  const T bp47 = vsub(vfma(rat<T>(-12.0), b21, vfma(rat<T>(-3.3333333333333335), b0, vadd(vfma(rat<T>(6.0), b25, vfma(rat<T>(1.6666666666666667), b2, vmul(rat<T>(12.0), b27))), b32))), b31);
  const T bp48 = vsub(vsub(vmul(rat<T>(9.333333333333334), b0), b33), b34);
  const T bp49 = vfma(rat<T>(7.333333333333333), b0, vfma(rat<T>(3.3333333333333335), b2, vmul(rat<T>(3.3333333333333335), b1)));
  const T bp50 = vsub(b24, b22);
  const T bp52 = vmul(rat<T>(-16.0), b6);
  const T bp54 = vmul(rat<T>(-1.3333333333333333), ux);
  const T bp59 = vsub(vsub(vfma(rat<T>(6.0), b25, vmul(rat<T>(1.6666666666666667), b2)), b31), b32);
  const T bp60 = vsub(b33, b34);
  const T bp61 = vfma(rat<T>(-1.3333333333333333), b1, vmul(rat<T>(1.3333333333333333), b2));
  const T bp62 = vadd(vadd(b28, b29), b4);
  const T bp64 = vmul(rat<T>(-1.0), b36);
  const T bp65 = vmul(rat<T>(-1.0), b37);
  r[4] = vfma(rho, bp0, x4);
  r[5] = vfma(rho, bp1, x5);
  r[6] = vfma(rho, bp2, x6);
  r[7] = vfma(rho, bp3, x7);
  r[8] = vfma(rho, bp4, x8);
  r[9] = vfma(rho, bp5, x9);
  r[10] = vfma(b14, x9, vfma(b12, x7, vfma(b10, x5, vfma(bp7, x4, vfma(rho, bp6, x10)))));
  r[11] = vfma(b14, x8, vfma(b15, x7, vfma(bp14, x6, vfma(uy, x5, vfma(bp12, x4, vfma(rho, bp11, x11))))));
  r[12] = vfma(b15, x9, vfma(b12, x8, vfma(bp20, x6, vfma(uz, x5, vfma(bp18, x4, vfma(rho, bp17, x12))))));
  r[13] = vfma(b17, x9, vfma(bp25, x7, vfma(bp24, x6, vfma(rho, bp23, x13))));
  r[14] = vfma(bp31, x8, vfma(b9, x7, vfma(b18, x6, vfma(b18, x5, vfma(rho, bp27, x14)))));
  r[15] = vfma(b10, x9, vfma(b16, x8, vfma(b19, x6, vfma(bp33, x5, vfma(rho, bp32, x15)))));
  r[16] = vfma(bp46, x12, vfma(bp45, x11, vfma(b30, x10, vfma(bp43, x9, vfma(bp42, x8, vfma(bp41, x7, vfma(bp40, x6, vfma(bp39, x5, vfma(bp38, x4, vfma(rho, bp37, x16))))))))));
  r[17] = vfma(b14, x15, vfma(b11, x14, vfma(b38, x12, vfma(b37, x11, vfma(bp54, x10, vfma(b36, x9, vfma(bp52, x8, vfma(b35, x7, vfma(bp50, x6, vfma(bp49, x5, vfma(bp48, x4, vfma(rho, bp47, x17))))))))))));
  r[18] = vfma(b17, x15, vfma(b16, x14, vfma(b30, x13, vfma(b38, x12, vfma(bp65, x11, vfma(bp64, x9, vfma(b35, x7, vfma(bp62, x6, vfma(bp61, x5, vfma(bp60, x4, vfma(rho, bp59, x18)))))))))));
}

// Only the shear central moments k_7 (xy), k_8 (yz), k_9 (xz).
template <typename T>
__device__ __forceinline__ void d3q19_shear_central(const T (&r)[19], T rho, T ux, T uy, T uz, T &k7, T &k8, T &k9) {
  const T r7 = r[7], r8 = r[8], r9 = r[9];
  const T c0 = vmul(rho, uy);
  k7 = vsub(r7, vmul(c0, ux));
  k8 = vsub(r8, vmul(c0, uz));
  k9 = vsub(r9, vmul(vmul(rho, ux), uz));
}

// Raw moments r*_v, v = 4..18, from the post-collision central moments k* (in place,
// ascending: row v uses the raw values of the rows below it; r*_0 = rho, r*_a = rho u_a).
template <typename T>
__device__ __forceinline__ void d3q19_raw_from_central(T (&k)[19], T rho, T ux, T uy, T uz) {
  const T k4 = k[4]; const T k5 = k[5]; const T k6 = k[6]; const T k7 = k[7]; const T k8 = k[8]; const T k9 = k[9]; const T k10 = k[10]; const T k11 = k[11]; const T k12 = k[12]; const T k13 = k[13]; const T k14 = k[14]; const T k15 = k[15]; const T k16 = k[16]; const T k17 = k[17]; const T k18 = k[18];
  const T d0 = vmul(ux, ux);
  const T d1 = vmul(uy, uy);
  const T d2 = vmul(uz, uz);
  const T d3 = vadd(d1, d2);
  const T d4 = vmul(rat<T>(2.0), d0);
  const T d5 = vmul(ux, uy);
  const T d6 = vmul(uy, uz);
  const T d7 = vmul(ux, uz);
  const T d8 = vmul(rat<T>(6.0), ux);
  const T d9 = vmul(rat<T>(2.0), ux);
  const T d10 = vmul(rat<T>(6.0), uy);
  const T d11 = vmul(rat<T>(6.0), uz);
  const T d12 = vmul(rat<T>(2.0), uy);
  const T d13 = vmul(rat<T>(2.0), uz);
  const T d14 = vmul(rat<T>(-1.0), d13);
  const T d15 = vmul(rat<T>(-0.5), uy);
  const T d16 = vmul(rat<T>(0.5), uz);
  const T d17 = vmul(rat<T>(-1.0), d12);
  const T d18 = vmul(rat<T>(4.0), d0);
  const T d19 = vmul(vmul(vmul(ux, ux), ux), ux);
  const T d20 = vmul(rat<T>(4.0), d1);
  const T d21 = vmul(vmul(vmul(uy, uy), uy), uy);
  const T d22 = vmul(rat<T>(4.0), d2);
  const T d23 = vmul(vmul(vmul(uz, uz), uz), uz);
  const T d24 = vmul(rat<T>(18.0), d0);
  const T d25 = vmul(d1, d2);
  const T d26 = vmul(rat<T>(6.0), d1);
  const T d27 = vmul(rat<T>(6.0), d2);
  const T d28 = vmul(rat<T>(4.0), ux);
  const T d29 = vmul(rat<T>(6.0), d23);
  const T d30 = vmul(rat<T>(1.6666666666666667), d2);
  const T d31 = vsub(vfma(rat<T>(6.0), d21, vmul(rat<T>(1.6666666666666667), d1)), vmul(d0, d27));
  const T d32 = vmul(rat<T>(4.666666666666667), d1);
  const T d33 = vmul(rat<T>(-8.0), d5);
  const T d34 = vmul(rat<T>(8.0), d7);
  const T d35 = vmul(rat<T>(0.6666666666666666), uy);
  const T d36 = vmul(rat<T>(-0.6666666666666666), uz);
  const T dp0 = vadd(d0, d3);
  const T dp1 = vsub(d4, d3);
  const T dp2 = vsub(d1, d2);
  const T dp6 = vsub(vsub(vmul(rat<T>(-6.0), vmul(vmul(ux, ux), ux)), vmul(d1, d8)), vmul(d2, d8));
  const T dp7 = vmul(rat<T>(5.0), ux);
  const T dp11 = vsub(vsub(vmul(rat<T>(-6.0), vmul(vmul(uy, uy), uy)), vmul(d0, d10)), vmul(d10, d2));
  const T dp12 = vmul(rat<T>(5.0), uy);
  const T dp13 = vmul(rat<T>(-1.0), uy);
  const T dp14 = vmul(rat<T>(3.0), uy);
  const T dp17 = vsub(vsub(vmul(rat<T>(-6.0), vmul(vmul(uz, uz), uz)), vmul(d0, d11)), vmul(d1, d11));
  const T dp18 = vmul(rat<T>(5.0), uz);
  const T dp19 = vmul(rat<T>(-1.0), uz);
  const T dp20 = vmul(rat<T>(-3.0), uz);
  const T dp23 = vsub(vmul(rat<T>(2.0), vmul(d2, ux)), vmul(d1, d9));
  const T dp27 = vsub(vmul(d4, uy), vmul(d12, d2));
  const T dp30 = vmul(rat<T>(-1.0), d9);
  const T dp32 = vsub(vmul(rat<T>(2.0), vmul(d1, uz)), vmul(d4, uz));
  const T dp34 = vmul(rat<T>(-1.0), d16);
  const T dp37 = vadd(vadd(vadd(vadd(vadd(vfma(rat<T>(9.0), d23, vfma(rat<T>(9.0), d21, vfma(rat<T>(9.0), d19, vmul(rat<T>(18.0), d25)))), vmul(d1, d24)), d18), vmul(d2, d24)), d20), d22);
  const T dp38 = vfma(rat<T>(-10.0), d2, vfma(rat<T>(-10.0), d1, vmul(rat<T>(-10.0), d0)));
  const T dp39 = vsub(vfma(rat<T>(2.0), d2, vmul(rat<T>(2.0), d1)), d18);
  const T dp40 = vsub(d27, d26);
  const T dp41 = vmul(rat<T>(-24.0), d5);
  const T dp42 = vmul(rat<T>(-24.0), d6);
  const T dp43 = vmul(rat<T>(-24.0), d7);
  const T dp45 = vmul(rat<T>(4.0), uy);
  const T dp46 = vmul(rat<T>(4.0), uz);
  const T dp47 = vsub(vsub(vsub(vfma(rat<T>(-12.0), d25, vfma(rat<T>(6.0), vmul(d0, d1), vfma(rat<T>(12.0), d19, vmul(rat<T>(3.3333333333333335), d0)))), d29), d30), d31);
  const T dp48 = vfma(rat<T>(-9.333333333333334), d0, vadd(vmul(rat<T>(4.666666666666667), d2), d32));
  const T dp49 = vfma(rat<T>(-7.333333333333333), d0, vfma(rat<T>(-3.3333333333333335), d2, vmul(rat<T>(-3.3333333333333335), d1)));
  const T dp50 = vsub(d20, d22);
  const T dp52 = vmul(rat<T>(16.0), d6);
  const T dp53 = vmul(rat<T>(-1.0), d34);
  const T dp54 = vmul(rat<T>(1.3333333333333333), ux);
  const T dp55 = vmul(rat<T>(-1.0), d35);
  const T dp57 = vmul(rat<T>(-1.0), d10);
  const T dp59 = vsub(vsub(vadd(vmul(d0, d26), d31), d29), d30);
  const T dp60 = vsub(vmul(rat<T>(4.666666666666667), d2), d32);
  const T dp61 = vfma(rat<T>(-1.3333333333333333), d2, vmul(rat<T>(1.3333333333333333), d1));
  const T dp62 = vsub(vsub(vmul(rat<T>(-1.0), d26), d27), d4);
  const T x4 = vfma(rho, dp0, k4);
  k[4] = x4;
  const T x5 = vfma(rho, dp1, k5);
  k[5] = x5;
  const T x6 = vfma(rho, dp2, k6);
  k[6] = x6;
  const T x7 = vfma(rho, d5, k7);
  k[7] = x7;
  const T x8 = vfma(rho, d6, k8);
  k[8] = x8;
  const T x9 = vfma(rho, d7, k9);
  k[9] = x9;
  const T x10 = vfma(d11, x9, vfma(d10, x7, vfma(d9, x5, vfma(dp7, x4, vfma(rho, dp6, k10)))));
  k[10] = x10;
  const T x11 = vfma(d11, x8, vfma(d8, x7, vfma(dp14, x6, vfma(dp13, x5, vfma(dp12, x4, vfma(rho, dp11, k11))))));
  k[11] = x11;
  const T x12 = vfma(d8, x9, vfma(d10, x8, vfma(dp20, x6, vfma(dp19, x5, vfma(dp18, x4, vfma(rho, dp17, k12))))));
  k[12] = x12;
  const T x13 = vfma(d14, x9, vfma(d12, x7, vfma(ux, x6, vfma(rho, dp23, k13))));
  k[13] = x13;
  const T x14 = vfma(d13, x8, vfma(dp30, x7, vfma(d15, x6, vfma(d15, x5, vfma(rho, dp27, k14)))));
  k[14] = x14;
  const T x15 = vfma(d9, x9, vfma(d17, x8, vfma(dp34, x6, vfma(d16, x5, vfma(rho, dp32, k15)))));
  k[15] = x15;
  const T x16 = vfma(dp46, x12, vfma(dp45, x11, vfma(d28, x10, vfma(dp43, x9, vfma(dp42, x8, vfma(dp41, x7, vfma(dp40, x6, vfma(dp39, x5, vfma(dp38, x4, vfma(rho, dp37, k16))))))))));
  k[16] = x16;
  const T x17 = vfma(d11, x15, vfma(dp57, x14, vfma(d36, x12, vfma(dp55, x11, vfma(dp54, x10, vfma(dp53, x9, vfma(dp52, x8, vfma(d33, x7, vfma(dp50, x6, vfma(dp49, x5, vfma(dp48, x4, vfma(rho, dp47, k17))))))))))));
  k[17] = x17;
  const T x18 = vfma(d14, x15, vfma(d17, x14, vfma(d28, x13, vfma(d36, x12, vfma(d35, x11, vfma(d34, x9, vfma(d33, x7, vfma(dp62, x6, vfma(dp61, x5, vfma(dp60, x4, vfma(rho, dp59, k18)))))))))));
  k[18] = x18;
}

// As d3q19_central, each row evaluating its own u-polynomials (fewer live registers).
template <typename T>
__device__ __forceinline__ void d3q19_central_lr(T (&r)[19], T rho, T ux, T uy, T uz) {
  const T x4 = r[4]; const T x5 = r[5]; const T x6 = r[6]; const T x7 = r[7]; const T x8 = r[8]; const T x9 = r[9]; const T x10 = r[10]; const T x11 = r[11]; const T x12 = r[12]; const T x13 = r[13]; const T x14 = r[14]; const T x15 = r[15]; const T x16 = r[16]; const T x17 = r[17]; const T x18 = r[18];
  {
  r[4] = vfma(rho, vsub(vsub(vmul(rat<T>(-1.0), vmul(ux, ux)), vmul(uy, uy)), vmul(uz, uz)), x4);
  }
  {
  r[5] = vfma(rho, vfma(rat<T>(-2.0), vmul(ux, ux), vadd(vmul(uy, uy), vmul(uz, uz))), x5);
  }
  {
  r[6] = vfma(rho, vsub(vmul(uz, uz), vmul(uy, uy)), x6);
  }
  {
  r[7] = vfma(rho, vmul(rat<T>(-1.0), vmul(ux, uy)), x7);
  }
  {
  r[8] = vfma(rho, vmul(rat<T>(-1.0), vmul(uy, uz)), x8);
  }
  {
  r[9] = vfma(rho, vmul(rat<T>(-1.0), vmul(ux, uz)), x9);
  }
  {
    const T g10_0 = vmul(rat<T>(6.0), ux);
  r[10] = vfma(vmul(rat<T>(-6.0), uz), x9, vfma(vmul(rat<T>(-6.0), uy), x7, vfma(vmul(rat<T>(-2.0), ux), x5, vfma(vmul(rat<T>(-5.0), ux), x4, vfma(rho, vadd(vadd(vmul(rat<T>(6.0), vmul(vmul(ux, ux), ux)), vmul(vmul(g10_0, uy), uy)), vmul(vmul(g10_0, uz), uz)), x10)))));
  }
  {
    const T g11_0 = vmul(rat<T>(6.0), uy);
  r[11] = vfma(vmul(rat<T>(-6.0), uz), x8, vfma(vmul(rat<T>(-6.0), ux), x7, vfma(vmul(rat<T>(-3.0), uy), x6, vfma(uy, x5, vfma(vmul(rat<T>(-5.0), uy), x4, vfma(rho, vadd(vadd(vmul(rat<T>(6.0), vmul(vmul(uy, uy), uy)), vmul(vmul(g11_0, ux), ux)), vmul(vmul(g11_0, uz), uz)), x11))))));
  }
  {
    const T g12_0 = vmul(rat<T>(6.0), uz);
  r[12] = vfma(vmul(rat<T>(-6.0), ux), x9, vfma(vmul(rat<T>(-6.0), uy), x8, vfma(vmul(rat<T>(3.0), uz), x6, vfma(uz, x5, vfma(vmul(rat<T>(-5.0), uz), x4, vfma(rho, vadd(vadd(vmul(rat<T>(6.0), vmul(vmul(uz, uz), uz)), vmul(vmul(g12_0, ux), ux)), vmul(vmul(g12_0, uy), uy)), x12))))));
  }
  {
    const T g13_0 = vmul(rat<T>(2.0), ux);
  r[13] = vfma(vmul(rat<T>(2.0), uz), x9, vfma(vmul(rat<T>(-2.0), uy), x7, vfma(vmul(rat<T>(-1.0), ux), x6, vfma(rho, vsub(vmul(vmul(g13_0, uy), uy), vmul(vmul(g13_0, uz), uz)), x13))));
  }
  {
    const T g14_0 = vmul(rat<T>(0.5), uy);
  r[14] = vfma(vmul(rat<T>(-2.0), uz), x8, vfma(vmul(rat<T>(2.0), ux), x7, vfma(g14_0, x6, vfma(g14_0, x5, vfma(rho, vfma(rat<T>(-2.0), vmul(vmul(uy, ux), ux), vmul(rat<T>(2.0), vmul(vmul(uy, uz), uz))), x14)))));
  }
  {
    const T g15_0 = vmul(rat<T>(2.0), uz);
    const T g15_1 = vmul(rat<T>(0.5), uz);
  r[15] = vfma(vmul(rat<T>(-2.0), ux), x9, vfma(vmul(rat<T>(2.0), uy), x8, vfma(g15_1, x6, vfma(vmul(rat<T>(-1.0), g15_1), x5, vfma(rho, vsub(vmul(vmul(g15_0, ux), ux), vmul(vmul(g15_0, uy), uy)), x15)))));
  }
  {
    const T g16_0 = vmul(ux, ux);
    const T g16_1 = vmul(rat<T>(4.0), g16_0);
    const T g16_2 = vmul(uy, uy);
    const T g16_3 = vmul(uz, uz);
    const T g16_4 = vmul(rat<T>(18.0), g16_0);
    const T g16_5 = vmul(rat<T>(24.0), uy);
  r[16] = vfma(vmul(rat<T>(-4.0), uz), x12, vfma(vmul(rat<T>(-4.0), uy), x11, vfma(vmul(rat<T>(-4.0), ux), x10, vfma(vmul(rat<T>(24.0), vmul(ux, uz)), x9, vfma(vmul(g16_5, uz), x8, vfma(vmul(g16_5, ux), x7, vfma(vfma(rat<T>(-6.0), g16_3, vmul(rat<T>(6.0), g16_2)), x6, vfma(vfma(rat<T>(-2.0), g16_3, vfma(rat<T>(-2.0), g16_2, g16_1)), x5, vfma(vfma(rat<T>(10.0), g16_3, vfma(rat<T>(10.0), g16_2, vmul(rat<T>(10.0), g16_0))), x4, vfma(rho, vsub(vsub(vsub(vfma(rat<T>(-9.0), vmul(vmul(vmul(uz, uz), uz), uz), vfma(rat<T>(-9.0), vmul(vmul(vmul(uy, uy), uy), uy), vfma(rat<T>(-9.0), vmul(vmul(vmul(ux, ux), ux), ux), vfma(rat<T>(-4.0), g16_3, vfma(rat<T>(-4.0), g16_2, vmul(rat<T>(-18.0), vmul(g16_2, g16_3))))))), g16_1), vmul(g16_2, g16_4)), vmul(g16_3, g16_4)), x16))))))))));
  }
  {
    const T g17_0 = vmul(ux, ux);
    const T g17_1 = vmul(uy, uy);
    const T g17_2 = vmul(uz, uz);
    const T g17_3 = vmul(rat<T>(6.0), g17_0);
    const T g17_4 = vmul(rat<T>(8.0), ux);
  r[17] = vfma(vmul(rat<T>(-6.0), uz), x15, vfma(vmul(rat<T>(6.0), uy), x14, vfma(vmul(rat<T>(0.6666666666666666), uz), x12, vfma(vmul(rat<T>(0.6666666666666666), uy), x11, vfma(vmul(rat<T>(-1.3333333333333333), ux), x10, vfma(vmul(g17_4, uz), x9, vfma(vmul(rat<T>(-16.0), vmul(uy, uz)), x8, vfma(vmul(g17_4, uy), x7, vfma(vfma(rat<T>(-4.0), g17_1, vmul(rat<T>(4.0), g17_2)), x6, vfma(vfma(rat<T>(7.333333333333333), g17_0, vfma(rat<T>(3.3333333333333335), g17_2, vmul(rat<T>(3.3333333333333335), g17_1))), x5, vfma(vfma(rat<T>(-4.666666666666667), g17_2, vfma(rat<T>(-4.666666666666667), g17_1, vmul(rat<T>(9.333333333333334), g17_0))), x4, vfma(rho, vsub(vsub(vfma(rat<T>(-12.0), vmul(vmul(vmul(ux, ux), ux), ux), vfma(rat<T>(-3.3333333333333335), g17_0, vfma(rat<T>(6.0), vmul(vmul(vmul(uz, uz), uz), uz), vfma(rat<T>(6.0), vmul(vmul(vmul(uy, uy), uy), uy), vfma(rat<T>(1.6666666666666667), g17_2, vfma(rat<T>(1.6666666666666667), g17_1, vmul(rat<T>(12.0), vmul(g17_1, g17_2)))))))), vmul(g17_1, g17_3)), vmul(g17_2, g17_3)), x17))))))))))));
  }
  {
    const T g18_0 = vmul(uy, uy);
    const T g18_1 = vmul(uz, uz);
    const T g18_2 = vmul(ux, ux);
    const T g18_3 = vmul(rat<T>(6.0), g18_0);
    const T g18_4 = vmul(rat<T>(8.0), ux);
  r[18] = vfma(vmul(rat<T>(2.0), uz), x15, vfma(vmul(rat<T>(2.0), uy), x14, vfma(vmul(rat<T>(-4.0), ux), x13, vfma(vmul(rat<T>(0.6666666666666666), uz), x12, vfma(vmul(rat<T>(-0.6666666666666666), uy), x11, vfma(vmul(rat<T>(-1.0), vmul(g18_4, uz)), x9, vfma(vmul(g18_4, uy), x7, vfma(vadd(vfma(rat<T>(6.0), g18_1, vmul(rat<T>(2.0), g18_2)), g18_3), x6, vfma(vfma(rat<T>(-1.3333333333333333), g18_0, vmul(rat<T>(1.3333333333333333), g18_1)), x5, vfma(vfma(rat<T>(-4.666666666666667), g18_1, vmul(rat<T>(4.666666666666667), g18_0)), x4, vfma(rho, vsub(vfma(rat<T>(-6.0), vmul(vmul(vmul(uy, uy), uy), uy), vfma(rat<T>(-1.6666666666666667), g18_0, vfma(rat<T>(6.0), vmul(vmul(vmul(uz, uz), uz), uz), vfma(rat<T>(6.0), vmul(g18_1, g18_2), vmul(rat<T>(1.6666666666666667), g18_1))))), vmul(g18_2, g18_3)), x18)))))))))));
  }
}

// As d3q19_raw_from_central, each row evaluating its own u-polynomials.
template <typename T>
__device__ __forceinline__ void d3q19_raw_from_central_lr(T (&k)[19], T rho, T ux, T uy, T uz) {
  T x4; T x5; T x6; T x7; T x8; T x9; T x10; T x11; T x12; T x13; T x14; T x15; T x16; T x17; T x18;
  const T k4 = k[4]; const T k5 = k[5]; const T k6 = k[6]; const T k7 = k[7]; const T k8 = k[8]; const T k9 = k[9]; const T k10 = k[10]; const T k11 = k[11]; const T k12 = k[12]; const T k13 = k[13]; const T k14 = k[14]; const T k15 = k[15]; const T k16 = k[16]; const T k17 = k[17]; const T k18 = k[18];
  {
  x4 = vfma(rho, vadd(vadd(vmul(ux, ux), vmul(uy, uy)), vmul(uz, uz)), k4);
    k[4] = x4;
  }
  {
  x5 = vfma(rho, vsub(vsub(vmul(rat<T>(2.0), vmul(ux, ux)), vmul(uy, uy)), vmul(uz, uz)), k5);
    k[5] = x5;
  }
  {
  x6 = vfma(rho, vsub(vmul(uy, uy), vmul(uz, uz)), k6);
    k[6] = x6;
  }
  {
  x7 = vfma(rho, vmul(ux, uy), k7);
    k[7] = x7;
  }
  {
  x8 = vfma(rho, vmul(uy, uz), k8);
    k[8] = x8;
  }
  {
  x9 = vfma(rho, vmul(ux, uz), k9);
    k[9] = x9;
  }
  {
    const T h10_0 = vmul(rat<T>(6.0), ux);
  x10 = vfma(vmul(rat<T>(6.0), uz), x9, vfma(vmul(rat<T>(6.0), uy), x7, vfma(vmul(rat<T>(2.0), ux), x5, vfma(vmul(rat<T>(5.0), ux), x4, vfma(rho, vsub(vsub(vmul(rat<T>(-6.0), vmul(vmul(ux, ux), ux)), vmul(vmul(h10_0, uy), uy)), vmul(vmul(h10_0, uz), uz)), k10)))));
    k[10] = x10;
  }
  {
    const T h11_0 = vmul(rat<T>(6.0), uy);
  x11 = vfma(vmul(rat<T>(6.0), uz), x8, vfma(vmul(rat<T>(6.0), ux), x7, vfma(vmul(rat<T>(3.0), uy), x6, vfma(vmul(rat<T>(-1.0), uy), x5, vfma(vmul(rat<T>(5.0), uy), x4, vfma(rho, vsub(vsub(vmul(rat<T>(-6.0), vmul(vmul(uy, uy), uy)), vmul(vmul(h11_0, ux), ux)), vmul(vmul(h11_0, uz), uz)), k11))))));
    k[11] = x11;
  }
  {
    const T h12_0 = vmul(rat<T>(6.0), uz);
  x12 = vfma(vmul(rat<T>(6.0), ux), x9, vfma(vmul(rat<T>(6.0), uy), x8, vfma(vmul(rat<T>(-3.0), uz), x6, vfma(vmul(rat<T>(-1.0), uz), x5, vfma(vmul(rat<T>(5.0), uz), x4, vfma(rho, vsub(vsub(vmul(rat<T>(-6.0), vmul(vmul(uz, uz), uz)), vmul(vmul(h12_0, ux), ux)), vmul(vmul(h12_0, uy), uy)), k12))))));
    k[12] = x12;
  }
  {
  x13 = vfma(vmul(rat<T>(-2.0), uz), x9, vfma(vmul(rat<T>(2.0), uy), x7, vfma(ux, x6, vfma(rho, vfma(rat<T>(-2.0), vmul(vmul(ux, uy), uy), vmul(rat<T>(2.0), vmul(vmul(ux, uz), uz))), k13))));
    k[13] = x13;
  }
  {
    const T h14_0 = vmul(rat<T>(2.0), uy);
    const T h14_1 = vmul(rat<T>(-0.5), uy);
  x14 = vfma(vmul(rat<T>(2.0), uz), x8, vfma(vmul(rat<T>(-2.0), ux), x7, vfma(h14_1, x6, vfma(h14_1, x5, vfma(rho, vsub(vmul(vmul(h14_0, ux), ux), vmul(vmul(h14_0, uz), uz)), k14)))));
    k[14] = x14;
  }
  {
    const T h15_0 = vmul(rat<T>(0.5), uz);
  x15 = vfma(vmul(rat<T>(2.0), ux), x9, vfma(vmul(rat<T>(-2.0), uy), x8, vfma(vmul(rat<T>(-1.0), h15_0), x6, vfma(h15_0, x5, vfma(rho, vfma(rat<T>(-2.0), vmul(vmul(uz, ux), ux), vmul(rat<T>(2.0), vmul(vmul(uz, uy), uy))), k15)))));
    k[15] = x15;
  }
  {
    const T h16_0 = vmul(ux, ux);
    const T h16_1 = vmul(rat<T>(4.0), h16_0);
    const T h16_2 = vmul(uy, uy);
    const T h16_3 = vmul(uz, uz);
    const T h16_4 = vmul(rat<T>(18.0), h16_0);
    const T h16_5 = vmul(rat<T>(24.0), uy);
  x16 = vfma(vmul(rat<T>(4.0), uz), x12, vfma(vmul(rat<T>(4.0), uy), x11, vfma(vmul(rat<T>(4.0), ux), x10, vfma(vmul(rat<T>(-24.0), vmul(ux, uz)), x9, vfma(vmul(rat<T>(-1.0), vmul(h16_5, uz)), x8, vfma(vmul(rat<T>(-1.0), vmul(h16_5, ux)), x7, vfma(vfma(rat<T>(-6.0), h16_2, vmul(rat<T>(6.0), h16_3)), x6, vfma(vsub(vfma(rat<T>(2.0), h16_3, vmul(rat<T>(2.0), h16_2)), h16_1), x5, vfma(vfma(rat<T>(-10.0), h16_3, vfma(rat<T>(-10.0), h16_2, vmul(rat<T>(-10.0), h16_0))), x4, vfma(rho, vadd(vadd(vadd(vfma(rat<T>(9.0), vmul(vmul(vmul(uz, uz), uz), uz), vfma(rat<T>(9.0), vmul(vmul(vmul(uy, uy), uy), uy), vfma(rat<T>(9.0), vmul(vmul(vmul(ux, ux), ux), ux), vfma(rat<T>(4.0), h16_3, vfma(rat<T>(4.0), h16_2, vmul(rat<T>(18.0), vmul(h16_2, h16_3))))))), h16_1), vmul(h16_2, h16_4)), vmul(h16_3, h16_4)), k16))))))))));
    k[16] = x16;
  }
  {
    const T h17_0 = vmul(ux, ux);
    const T h17_1 = vmul(uy, uy);
    const T h17_2 = vmul(uz, uz);
    const T h17_3 = vmul(rat<T>(8.0), ux);
  x17 = vfma(vmul(rat<T>(6.0), uz), x15, vfma(vmul(rat<T>(-6.0), uy), x14, vfma(vmul(rat<T>(-0.6666666666666666), uz), x12, vfma(vmul(rat<T>(-0.6666666666666666), uy), x11, vfma(vmul(rat<T>(1.3333333333333333), ux), x10, vfma(vmul(rat<T>(-1.0), vmul(h17_3, uz)), x9, vfma(vmul(rat<T>(16.0), vmul(uy, uz)), x8, vfma(vmul(rat<T>(-1.0), vmul(h17_3, uy)), x7, vfma(vfma(rat<T>(-4.0), h17_2, vmul(rat<T>(4.0), h17_1)), x6, vfma(vfma(rat<T>(-7.333333333333333), h17_0, vfma(rat<T>(-3.3333333333333335), h17_2, vmul(rat<T>(-3.3333333333333335), h17_1))), x5, vfma(vfma(rat<T>(-9.333333333333334), h17_0, vfma(rat<T>(4.666666666666667), h17_2, vmul(rat<T>(4.666666666666667), h17_1))), x4, vfma(rho, vfma(rat<T>(-6.0), vmul(vmul(vmul(uz, uz), uz), uz), vfma(rat<T>(-6.0), vmul(vmul(vmul(uy, uy), uy), uy), vfma(rat<T>(-1.6666666666666667), h17_2, vfma(rat<T>(-1.6666666666666667), h17_1, vfma(rat<T>(-12.0), vmul(h17_1, h17_2), vfma(rat<T>(6.0), vmul(h17_0, h17_2), vfma(rat<T>(6.0), vmul(h17_0, h17_1), vfma(rat<T>(12.0), vmul(vmul(vmul(ux, ux), ux), ux), vmul(rat<T>(3.3333333333333335), h17_0))))))))), k17))))))))))));
    k[17] = x17;
  }
  {
    const T h18_0 = vmul(uy, uy);
    const T h18_1 = vmul(uz, uz);
    const T h18_2 = vmul(ux, ux);
    const T h18_3 = vmul(rat<T>(6.0), h18_0);
    const T h18_4 = vmul(rat<T>(6.0), h18_1);
    const T h18_5 = vmul(rat<T>(8.0), ux);
  x18 = vfma(vmul(rat<T>(-2.0), uz), x15, vfma(vmul(rat<T>(-2.0), uy), x14, vfma(vmul(rat<T>(4.0), ux), x13, vfma(vmul(rat<T>(-0.6666666666666666), uz), x12, vfma(vmul(rat<T>(0.6666666666666666), uy), x11, vfma(vmul(h18_5, uz), x9, vfma(vmul(rat<T>(-1.0), vmul(h18_5, uy)), x7, vfma(vsub(vsub(vmul(rat<T>(-2.0), h18_2), h18_3), h18_4), x6, vfma(vfma(rat<T>(-1.3333333333333333), h18_1, vmul(rat<T>(1.3333333333333333), h18_0)), x5, vfma(vfma(rat<T>(-4.666666666666667), h18_0, vmul(rat<T>(4.666666666666667), h18_1)), x4, vfma(rho, vsub(vfma(rat<T>(-6.0), vmul(vmul(vmul(uz, uz), uz), uz), vfma(rat<T>(-1.6666666666666667), h18_1, vadd(vfma(rat<T>(6.0), vmul(vmul(vmul(uy, uy), uy), uy), vmul(rat<T>(1.6666666666666667), h18_0)), vmul(h18_2, h18_3)))), vmul(h18_2, h18_4)), k18)))))))))));
    k[18] = x18;
  }
}

// Deviations d*_i = sum_v w_i M_vi r*_v / b_v (M^{-1} = W M^T B^{-1}); r*_0 = rho - rho0.
template <typename T>
__device__ __forceinline__ void d3q19_pop(const T (&r)[19], T (&f)[19]) {
  const T r0 = r[0];
  const T r1 = r[1];
  const T r2 = r[2];
  const T r3 = r[3];
  const T r4 = r[4];
  const T r5 = r[5];
  const T r6 = r[6];
  const T r7 = r[7];
  const T r8 = r[8];
  const T r9 = r[9];
  const T r10 = r[10];
  const T r11 = r[11];
  const T r12 = r[12];
  const T r13 = r[13];
  const T r14 = r[14];
  const T r15 = r[15];
  const T r16 = r[16];
  const T r17 = r[17];
  const T r18 = r[18];
  const T e0 = vmul(rat<T>(0.16666666666666666), r10);
  const T e1 = vmul(rat<T>(0.16666666666666666), r1);
  const T e2 = vfma(rat<T>(-0.05555555555555555), r16, vmul(rat<T>(0.05555555555555555), r0));
  const T e3 = vfma(rat<T>(-0.08333333333333333), r17, vfma(rat<T>(0.08333333333333333), r5, e2));
  const T e4 = vmul(rat<T>(0.16666666666666666), r11);
  const T e5 = vmul(rat<T>(0.16666666666666666), r2);
  const T e6 = vmul(rat<T>(0.125), r18);
  const T e7 = vmul(rat<T>(0.125), r6);
  const T e8 = vmul(rat<T>(0.041666666666666664), r5);
  const T e9 = vmul(rat<T>(-1.0), e8);
  const T e10 = vmul(rat<T>(0.041666666666666664), r17);
  const T e11 = vadd(vadd(e10, e2), e9);
  const T e12 = vsub(vadd(e11, e7), e6);
  const T e13 = vmul(rat<T>(0.16666666666666666), r12);
  const T e14 = vmul(rat<T>(0.16666666666666666), r3);
  const T e15 = vsub(vadd(e11, e6), e7);
  const T e16 = vfma(rat<T>(0.041666666666666664), r4, vfma(rat<T>(0.013888888888888888), r16, vmul(rat<T>(0.027777777777777776), r0)));
  const T e17 = vmul(rat<T>(0.125), r13);
  const T e18 = vmul(rat<T>(0.020833333333333332), r17);
  const T e19 = vmul(rat<T>(0.020833333333333332), r5);
  const T e20 = vadd(vadd(e17, e18), e19);
  const T e21 = vadd(e16, e20);
  const T e22 = vmul(rat<T>(0.08333333333333333), r1);
  const T e23 = vmul(rat<T>(0.041666666666666664), r10);
  const T e24 = vadd(e22, e23);
  const T e25 = vmul(rat<T>(0.25), r7);
  const T e26 = vmul(rat<T>(0.0625), r18);
  const T e27 = vmul(rat<T>(0.0625), r6);
  const T e28 = vadd(vadd(e25, e26), e27);
  const T e29 = vmul(rat<T>(0.125), r14);
  const T e30 = vmul(rat<T>(0.08333333333333333), r2);
  const T e31 = vmul(rat<T>(0.041666666666666664), r11);
  const T e32 = vadd(e30, e31);
  const T e33 = vsub(e32, e29);
  const T e34 = vsub(vmul(rat<T>(-1.0), e22), e23);
  const T e35 = vsub(vadd(e26, e27), e25);
  const T e36 = vsub(vadd(e18, e19), e17);
  const T e37 = vadd(e16, e36);
  const T e38 = vadd(e16, e29);
  const T e39 = vsub(vsub(e38, e30), e31);
  const T e40 = vmul(rat<T>(0.25), r9);
  const T e41 = vmul(rat<T>(-1.0), e26);
  const T e42 = vmul(rat<T>(-1.0), e27);
  const T e43 = vadd(vadd(e24, e41), e42);
  const T e44 = vmul(rat<T>(0.125), r15);
  const T e45 = vmul(rat<T>(0.08333333333333333), r3);
  const T e46 = vmul(rat<T>(0.041666666666666664), r12);
  const T e47 = vadd(e45, e46);
  const T e48 = vadd(e44, e47);
  const T e49 = vmul(rat<T>(-1.0), e40);
  const T e50 = vadd(vadd(e34, e41), e42);
  const T e51 = vmul(rat<T>(-1.0), e44);
  const T e52 = vadd(e16, e51);
  const T e53 = vsub(vmul(rat<T>(-1.0), e45), e46);
  const T e54 = vadd(e52, e53);
  const T e55 = vmul(rat<T>(0.25), r8);
  const T e56 = vadd(vadd(vadd(e29, e30), e31), e55);
  const T e57 = vsub(e9, e10);
  const T e58 = vadd(e44, e53);
  const T e59 = vfma(rat<T>(-0.041666666666666664), r4, vfma(rat<T>(-0.013888888888888888), r16, vfma(rat<T>(-0.027777777777777776), r0, vadd(e10, e8))));
  const T e60 = vsub(e32, e55);
  f[0] = vfma(rat<T>(-0.5), r4, vfma(rat<T>(0.16666666666666666), r16, vmul(rat<T>(0.3333333333333333), r0)));
  f[1] = vsub(vadd(e1, e3), e0);
  f[2] = vsub(vadd(e0, e3), e1);
  f[3] = vsub(vadd(e12, e5), e4);
  f[4] = vsub(vadd(e12, e4), e5);
  f[5] = vsub(vadd(e14, e15), e13);
  f[6] = vsub(vadd(e13, e15), e14);
  f[7] = vadd(vadd(vadd(e21, e24), e28), e33);
  f[8] = vadd(vadd(vadd(e33, e34), e35), e37);
  f[9] = vadd(vadd(vadd(e20, e24), e35), e39);
  f[10] = vadd(vadd(vadd(e28, e34), e36), e39);
  f[11] = vadd(vadd(vadd(e37, e40), e43), e48);
  f[12] = vadd(vadd(vadd(e21, e48), e49), e50);
  f[13] = vadd(vadd(vadd(e36, e43), e49), e54);
  f[14] = vadd(vadd(vadd(e20, e40), e50), e54);
  f[15] = vadd(vadd(vadd(e47, e52), e56), e57);
  f[16] = vsub(vsub(vmul(rat<T>(-1.0), e56), e58), e59);
  f[17] = vadd(vadd(vadd(e38, e57), e58), e60);
  f[18] = vsub(vsub(vsub(vsub(vmul(rat<T>(-1.0), e29), e47), e51), e59), e60);
}

}  // namespace flbm
