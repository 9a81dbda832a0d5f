"""Writes d3q19_gen.cuh: the D3Q19 moment transforms of the fused step, as straight-line
code generated from the basis printed in Sec. II-C ("Lattice-agnostic construction and the
D3Q19 example").

    python paper_2602_16486_gb300/csrc/gen_d3q19.py      (needs sympy; run after editing)

The D3Q19 basis is not a tensor product, so the factorised per-axis transforms of the
D2Q9/D3Q27 kernels do not apply. What does hold (checked here, exactly): with
M the raw-moment matrix of the printed polynomials and T(u) = [M_v(c_i - u)] the
central-moment matrix, N(u) = T(u) M^{-1} is unit lower triangular with entries that are
polynomials of degree <= 4 in u. The kernels therefore compute
    r = M d (raw moments of the stored deviations),
    k_v = r_v + rho P_v(u) + sum_{4 <= w < v} N_vw(u) r_w      (v >= 4),
with P_v(u) = N_v0 + N_v1 u_x + N_v2 u_y + N_v3 u_z (r_0 = rho and r_a = rho u_a), and
invert the collision result by forward substitution with the same N(u):
    r*_v = k*_v - rho P_v(u) - sum_{4 <= w < v} N_vw(u) r*_w,
    d* = M^{-1} r* with r*_0 = rho - rho0 and r*_a = rho u_a,
where M^{-1} = W M^T B^{-1} (the printed orthogonality, B = diag(b_v)). All functions are
templated on the value type (float: one site, float2: two sites) and use the helpers of
vec.cuh.
"""
import os

import sympy as sp

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "d3q19_gen.cuh")

# Velocities: the first 19 of the paper's D3Q27 order (rest, +-x, +-y, +-z, then the
# xy, xz, yz face diagonals).
CX = [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0]
CY = [0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1]
CZ = [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1]
W = [sp.Rational(1, 3)] + [sp.Rational(1, 18)] * 6 + [sp.Rational(1, 36)] * 12


def basis(x, y, z):
    c2 = x * x + y * y + z * z
    return [1, x, y, z, c2 - 1, 3 * x * x - c2, y * y - z * z, x * y, y * z, x * z, x * (3 * c2 - 5),
            y * (3 * c2 - 5), z * (3 * c2 - 5), x * (y * y - z * z), y * (z * z - x * x), z * (x * x - y * y),
            3 * c2 * c2 - 6 * c2 + 1, (2 * c2 - 3) * (3 * x * x - c2), (2 * c2 - 3) * (y * y - z * z)]


ux, uy, uz, rho = sp.symbols("ux uy uz rho")
M = sp.Matrix([[sp.Integer(basis(CX[i], CY[i], CZ[i])[v]) for i in range(19)] for v in range(19)])
B = [sum(W[i] * M[v, i] ** 2 for i in range(19)) for v in range(19)]
T = sp.Matrix([[sp.expand(basis(CX[i] - ux, CY[i] - uy, CZ[i] - uz)[v]) for i in range(19)] for v in range(19)])
N = (T * M.inv()).applyfunc(sp.expand)
for v in range(19):
    assert N[v, v] == 1
    for w in range(v + 1, 19):
        assert N[v, w] == 0
# orthogonality (the printed norms): M W M^T = diag(b)
G = M * sp.diag(*W) * M.T
assert all(G[a, b] == 0 for a in range(19) for b in range(19) if a != b)
P = [sp.expand(N[v, 0] + N[v, 1] * ux + N[v, 2] * uy + N[v, 3] * uz) for v in range(19)]


def lit(c):
    t = repr(float(c))
    if "." not in t and "e" not in t:
        t += ".0"
    return f"rat<T>({t})"


def emit(e):
    """Code for a polynomial expression e with rational coefficients (vec.cuh helpers)."""
    e = sp.expand(e) if not isinstance(e, sp.Symbol) else e
    if e.is_Number:
        return lit(e)
    if isinstance(e, sp.Symbol):
        return str(e)
    if e.is_Add:
        terms = list(e.args)
        # a term with a positive coefficient first, constants last
        terms.sort(key=lambda t: (bool(t.is_Number), float(t.as_coeff_Mul()[0]) < 0, str(t)))
        acc = None
        for t in terms:
            c, rest = t.as_coeff_Mul()
            if acc is None:
                acc = emit(t)
            elif rest == 1:
                acc = f"vadd({acc}, {lit(c)})"
            elif c == 1:
                acc = f"vadd({acc}, {emit(rest)})"
            elif c == -1:
                acc = f"vsub({acc}, {emit(rest)})"
            else:
                acc = f"vfma({lit(c)}, {emit(rest)}, {acc})"
        return acc
    if e.is_Mul:
        c, rest = e.as_coeff_Mul()
        factors = []
        for f in sp.Mul.make_args(rest):
            if f.is_Pow:
                base, ex = f.as_base_exp()
                factors += [base] * int(ex)
            else:
                factors.append(f)
        code = emit(factors[0])
        for f in factors[1:]:
            code = f"vmul({code}, {emit(f)})"
        if c != 1:
            code = f"vmul({lit(c)}, {code})"
        return code
    if e.is_Pow:
        base, ex = e.as_base_exp()
        code = emit(base)
        for _ in range(int(ex) - 1):
            code = f"vmul({code}, {emit(base)})"
        return code
    raise ValueError(e)


def body(assignments, prefix):
    """assignments: list of (target code, expression). Common subexpressions become
    temporaries named prefix0, prefix1, ..."""
    exprs = [e for _, e in assignments]
    reps, red = sp.cse(exprs, symbols=sp.numbered_symbols(prefix), optimizations=None)
    lines = [f"  const T {s} = {emit(v)};" for s, v in reps]
    lines += [f"  {t} = {emit(e)};" for (t, _), e in zip(assignments, red)]
    return "\n".join(lines)


fs = sp.symbols("f0:19")
rs = sp.symbols("r0:19")
out = []
out.append('''// GENERATED by gen_d3q19.py from the D3Q19 basis of Sec. II-C ("Lattice-agnostic
// construction and the D3Q19 example"); do not edit. See the generator for the algebra.
#pragma once

#include "vec.cuh"

namespace flbm {
''')
# raw moments of the deviations
out.append("// r_v = sum_i M_vi d_i (r_0 = rho - rho0; r_1..3 = j).")
out.append("template <typename T>\n__device__ __forceinline__ void d3q19_raw(const T (&f)[19], T (&r)[19]) {")
for i in range(19):
    out.append(f"  const T f{i} = f[{i}];")
out.append(body([(f"r[{v}]", sum(M[v, i] * fs[i] for i in range(19))) for v in range(19)], "a"))
out.append("}\n")

def shift_rows(sign, prefix, src, dst_fmt):
    """Rows v = 4..18 of  dst_v = src_v + sign (rho P_v(u) + sum_{4<=w<v} N_vw(u) x_w),
    where x_w is the raw value of row w (src for the forward shift, the already computed
    rows for the inverse). The u-polynomials are shared through CSE; the rows are emitted
    in order, as FMA chains."""
    keys, polys = [], []
    for v in range(4, 19):
        if P[v] != 0:
            keys.append(("P", v, None))
            polys.append(sign * P[v])
        for w in range(4, v):
            if N[v, w] != 0:
                keys.append(("N", v, w))
                polys.append(sign * N[v, w])
    reps, red = sp.cse(polys, symbols=sp.numbered_symbols(prefix), optimizations=None)
    lines = [f"  const T {t} = {emit(e)};" for t, e in reps]
    names = {}
    for n, (key, e) in enumerate(zip(keys, red)):
        if isinstance(e, sp.Symbol):
            names[key] = str(e)
        else:
            nm = f"{prefix}p{n}"
            lines.append(f"  const T {nm} = {emit(e)};")
            names[key] = nm
    for v in range(4, 19):
        acc = f"{src}{v}"
        if ("P", v, None) in names:
            acc = f"vfma(rho, {names[('P', v, None)]}, {acc})"
        for w in range(4, v):
            if ("N", v, w) in names:
                acc = f"vfma({names[('N', v, w)]}, x{w}, {acc})"
        lines.append(dst_fmt.format(v=v, code=acc))
    return "\n".join(lines)


def shift_rows_local(sign, prefix, src, dst_fmt):
    """As shift_rows, but each row evaluates its own u-polynomials inside a block, so that
    no polynomial stays live across rows (fewer registers, some repeated products)."""
    lines = []
    for v in range(4, 19):
        keys, polys = [], []
        if P[v] != 0:
            keys.append(("P", v, None))
            polys.append(sign * P[v])
        for w in range(4, v):
            if N[v, w] != 0:
                keys.append(("N", v, w))
                polys.append(sign * N[v, w])
        reps, red = sp.cse(polys, symbols=sp.numbered_symbols(f"{prefix}{v}_"), optimizations=None)
        lines.append("  {")
        lines += [f"    const T {t} = {emit(e)};" for t, e in reps]
        acc = f"{src}{v}"
        for key, e in zip(keys, red):
            term = emit(e)
            if key[0] == "P":
                acc = f"vfma(rho, {term}, {acc})"
            else:
                acc = f"vfma({term}, x{key[2]}, {acc})"
        lines.append("  " + dst_fmt.format(v=v, code=acc).replace("\n", "\n  "))
        lines.append("  }")
    return "\n".join(lines)


# forward central transform, in place, rows 4..18 (every row reads raw values)
out.append("// Central moments k_v, v = 4..18, in place over the raw moments r (r_0..3 are not read:\n"
           "// the shift uses r_0 = rho and r_a = rho u_a).")
out.append("template <typename T>\n__device__ __forceinline__ void d3q19_central(T (&r)[19], T rho, T ux, T uy, T uz) {")
out.append("  " + " ".join(f"const T x{w} = r[{w}];" for w in range(4, 19)))
out.append(shift_rows(1, "b", "x", "  r[{v}] = {code};"))
out.append("}\n")
# shear central moments only
out.append("// Only the shear central moments k_7 (xy), k_8 (yz), k_9 (xz).")
out.append("template <typename T>\n__device__ __forceinline__ void d3q19_shear_central(const T (&r)[19], T rho, T ux, "
           "T uy, T uz, T &k7, T &k8, T &k9) {")
out.append("  const T r7 = r[7], r8 = r[8], r9 = r[9];")
for v in (7, 8, 9):
    assert all(N[v, w] == 0 for w in range(4, v))
out.append(body([("k7", rs[7] + rho * P[7]), ("k8", rs[8] + rho * P[8]), ("k9", rs[9] + rho * P[9])], "c"))
out.append("}\n")
# inverse: forward substitution, in place, ascending
out.append("// Raw moments r*_v, v = 4..18, from the post-collision central moments k* (in place,\n"
           "// ascending: row v uses the raw values of the rows below it; r*_0 = rho, r*_a = rho u_a).")
out.append("template <typename T>\n__device__ __forceinline__ void d3q19_raw_from_central(T (&k)[19], T rho, T ux, "
           "T uy, T uz) {")
out.append("  " + " ".join(f"const T k{v} = k[{v}];" for v in range(4, 19)))
out.append(shift_rows(-1, "d", "k", "  const T x{v} = {code};\n  k[{v}] = x{v};"))
out.append("}\n")
# the same two shifts with per-row polynomials (register-lean forms)
out.append("// As d3q19_central, each row evaluating its own u-polynomials (fewer live registers).")
out.append("template <typename T>\n__device__ __forceinline__ void d3q19_central_lr(T (&r)[19], T rho, T ux, T uy, "
           "T uz) {")
out.append("  " + " ".join(f"const T x{w} = r[{w}];" for w in range(4, 19)))
out.append(shift_rows_local(1, "g", "x", "r[{v}] = {code};"))
out.append("}\n")
out.append("// As d3q19_raw_from_central, each row evaluating its own u-polynomials.")
out.append("template <typename T>\n__device__ __forceinline__ void d3q19_raw_from_central_lr(T (&k)[19], T rho, T ux, "
           "T uy, T uz) {")
out.append("  " + " ".join(f"T x{v};" for v in range(4, 19)))
out.append("  " + " ".join(f"const T k{v} = k[{v}];" for v in range(4, 19)))
out.append(shift_rows_local(-1, "h", "k", "x{v} = {code};\n  k[{v}] = x{v};"))
out.append("}\n")
# populations from raw moments: f = W M^T B^{-1} r
out.append("// Deviations d*_i = sum_v w_i M_vi r*_v / b_v (M^{-1} = W M^T B^{-1}); r*_0 = rho - rho0.")
out.append("template <typename T>\n__device__ __forceinline__ void d3q19_pop(const T (&r)[19], T (&f)[19]) {")
for v in range(19):
    out.append(f"  const T r{v} = r[{v}];")
out.append(body([(f"f[{i}]", sum(W[i] * M[v, i] / B[v] * rs[v] for v in range(19))) for i in range(19)], "e"))
out.append("}\n")
out.append("}  // namespace flbm\n")
with open(OUT, "w") as fh:
    fh.write("\n".join(out))
print("wrote", OUT, "b =", B)
