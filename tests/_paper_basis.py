"""The paper's orthogonal bases typed in as polynomials in (c_x, c_y, c_z), for the oracle's
pins: {(l, m, n): coefficient} per mode, evaluated at any point. Test helper only.
D2Q9: Sec. II-B; D3Q27: Sec. II-C (M15 read as c_y^2 c_z - c_s^2 c_z); the isotropic
reading of D3Q27 (modes 4-6 as trace and deviators); D3Q19: Sec. II-C example."""
import numpy as np

CS2 = 1.0 / 3.0


def _mono(l, m, n, c=1.0):
    return {(l, m, n): c}


def _add(*ps):
    out = {}
    for p in ps:
        for k, v in p.items():
            out[k] = out.get(k, 0.0) + v
    return out


def _scale(p, s):
    return {k: v * s for k, v in p.items()}


def _mul(p, q):
    out = {}
    for (a, b, c), u in p.items():
        for (d, e, f), v in q.items():
            k = (a + d, b + e, c + f)
            out[k] = out.get(k, 0.0) + u * v
    return out


X, Y, Z, ONE = _mono(1, 0, 0), _mono(0, 1, 0), _mono(0, 0, 1), _mono(0, 0, 0)
X2, Y2, Z2 = _mono(2, 0, 0), _mono(0, 2, 0), _mono(0, 0, 2)


def _basis_d2q9():
    # Sec. II-B, the orthogonal D2Q9 basis.
    return [
        ONE, X, Y,
        _add(X2, Y2, _scale(ONE, -2 * CS2)),
        _add(X2, _scale(Y2, -1)),
        _mul(X, Y),
        _mul(_add(X2, _scale(ONE, -CS2)), Y),
        _mul(X, _add(Y2, _scale(ONE, -CS2))),
        _mul(_add(X2, _scale(ONE, -CS2)), _add(Y2, _scale(ONE, -CS2))),
    ]


def _basis_d3q27():
    # Sec. II-C, the orthogonal D3Q27 basis (M15 read as cy^2 cz - cs^2 cz, the printed
    # cs^2 cy being a typo: test_oracle_basis.test_printed_m15_is_a_typo).
    s, s2, s3 = CS2, CS2 ** 2, CS2 ** 3
    xy, xz, yz, xyz = _mul(X, Y), _mul(X, Z), _mul(Y, Z), _mul(_mul(X, Y), Z)
    return [
        ONE, X, Y, Z,
        _add(X2, _scale(ONE, -s)), _add(Y2, _scale(ONE, -s)), _add(Z2, _scale(ONE, -s)),
        xy, xz, yz,
        _add(_mul(X2, Y), _scale(Y, -s)),
        _add(_mul(X2, Z), _scale(Z, -s)),
        _add(_mul(X, Y2), _scale(X, -s)),
        _add(_mul(X, Z2), _scale(X, -s)),
        _add(_mul(Y, Z2), _scale(Y, -s)),
        _add(_mul(Y2, Z), _scale(Z, -s)),
        xyz,
        _add(_mul(X2, Y2), _scale(_add(X2, Y2), -s), _scale(ONE, s2)),
        _add(_mul(X2, Z2), _scale(_add(X2, Z2), -s), _scale(ONE, s2)),
        _add(_mul(Y2, Z2), _scale(_add(Y2, Z2), -s), _scale(ONE, s2)),
        _add(_mul(xy, Z2), _scale(xy, -s)),
        _add(_mul(xz, Y2), _scale(xz, -s)),
        _add(_mul(yz, X2), _scale(yz, -s)),
        _add(_mul(_mul(X2, Y), Z2), _scale(_add(_mul(X2, Y), _mul(Y, Z2)), -s), _scale(Y, s2)),
        _add(_mul(_mul(X2, Y2), Z), _scale(_add(_mul(X2, Z), _mul(Y2, Z)), -s), _scale(Z, s2)),
        _add(_mul(_mul(X, Y2), Z2), _scale(_add(_mul(X, Y2), _mul(X, Z2)), -s), _scale(X, s2)),
        _add(_mul(_mul(X2, Y2), Z2), _scale(_add(_mul(X2, Y2), _mul(X2, Z2), _mul(Y2, Z2)), -s),
             _scale(_add(X2, Y2, Z2), s2), _scale(ONE, -s3)),
    ]


def _basis_d3q27_iso():
    # The isotropic reading of the D3Q27 basis: modes 4-6 replaced by the trace and two
    # deviators of the normal stresses, M4' = M4 + M5 + M6, M5' = M4 - M5,
    # M6' = M4 + M5 - 2 M6.
    b = _basis_d3q27()
    m4, m5, m6 = b[4], b[5], b[6]
    b[4] = _add(m4, m5, m6)
    b[5] = _add(m4, _scale(m5, -1))
    b[6] = _add(m4, m5, _scale(m6, -2))
    return b


def _basis_d3q19():
    # Sec. II-C, "Lattice-agnostic construction and the D3Q19 example".
    c2 = _add(X2, Y2, Z2)
    c2m = lambda a, b: _add(_scale(c2, a), _scale(ONE, b))  # a c^2 + b  # noqa: E731
    x3c = _add(_scale(X2, 3), _scale(c2, -1))
    yz2 = _add(Y2, _scale(Z2, -1))
    return [
        ONE, X, Y, Z,
        c2m(1, -1), x3c, yz2,
        _mul(X, Y), _mul(Y, Z), _mul(X, Z),
        _mul(X, c2m(3, -5)), _mul(Y, c2m(3, -5)), _mul(Z, c2m(3, -5)),
        _mul(X, yz2), _mul(Y, _add(Z2, _scale(X2, -1))), _mul(Z, _add(X2, _scale(Y2, -1))),
        _add(_scale(_mul(c2, c2), 3), _scale(c2, -6), ONE),
        _mul(c2m(2, -3), x3c),
        _mul(c2m(2, -3), yz2),
    ]


BASES = {0: _basis_d2q9, 1: _basis_d3q27, 2: _basis_d3q27_iso, 3: _basis_d3q19}




def evaluate(poly, c):
    """Value of the polynomial at points c[..., 3]."""
    c = np.asarray(c, dtype=float)
    out = np.zeros(c.shape[:-1])
    for (l, m, n), coef in poly.items():
        out = out + coef * c[..., 0] ** l * c[..., 1] ** m * c[..., 2] ** n
    return out


def matrix(lat, c):
    """M[v, i] = M_v(c_i) of the lattice's basis at the velocities c[Q, 3]."""
    return np.array([evaluate(p, c) for p in BASES[lat]()])
