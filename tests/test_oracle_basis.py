"""Pins of the oracle's lattices, bases and transform T(u) against what the paper prints.

Every expected value here comes from the paper (golden files or formulas printed in
the paper's text) or from mathematics (lattice isotropy, orthogonality), never from
the oracle itself.
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CS2 = 1.0 / 3.0


def _read_fracs(name):
    vals = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                vals.append(float(Fraction(line)))
    return np.array(vals)


@pytest.mark.parametrize("lat,Q,D", [(0, 9, 2), (1, 27, 3)])
def test_velocity_set_and_weights(oracle_mod, lat, Q, D):
    c, w, _ = oracle_mod.tables(lat)
    # Q distinct vectors spanning {-1,0,1}^D (Sec. II-B / II-C velocity lists).
    vecs = {tuple(v[:D]) for v in c}
    assert len(vecs) == Q
    assert vecs == set(itertools.product((-1, 0, 1), repeat=D))
    assert np.all(c[:, D:] == 0)
    # Weights are the tensor product of the 1-D weights (2/3, 1/6, 1/6).
    w1 = {0: 2 / 3, 1: 1 / 6, -1: 1 / 6}
    for i in range(Q):
        assert w[i] == pytest.approx(np.prod([w1[int(x)] for x in c[i, :D]]), abs=1e-15)
    # Lattice isotropy up to fourth order (textbook quadrature properties, cs^2 = 1/3).
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    for a in range(D):
        assert (w * c[:, a]).sum() == pytest.approx(0.0, abs=1e-15)
        for b in range(D):
            assert (w * c[:, a] * c[:, b]).sum() == pytest.approx(CS2 * (a == b), abs=1e-15)
    for a, b, g, d in itertools.product(range(D), repeat=4):
        expect = CS2 ** 2 * ((a == b) * (g == d) + (a == g) * (b == d) + (a == d) * (b == g))
        got = (w * c[:, a] * c[:, b] * c[:, g] * c[:, d]).sum()
        assert got == pytest.approx(expect, abs=1e-15)


def test_paper_velocity_groups_d3q27(oracle_mod):
    # Sec. II-C: w0 = 8/27, w1-6 = 2/27, w7-18 = 1/54, w19-26 = 1/216 by index.
    c, w, _ = oracle_mod.tables(1)
    expect = [8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8
    np.testing.assert_allclose(w, expect, rtol=0, atol=1e-16)
    speed2 = (c ** 2).sum(1)
    assert list(speed2) == [0] + [1] * 6 + [2] * 12 + [3] * 8


def test_paper_velocity_groups_d2q9(oracle_mod):
    # Sec. II-B: w0 = 4/9, w1-4 = 1/9, w5-8 = 1/36.
    c, w, _ = oracle_mod.tables(0)
    np.testing.assert_allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, rtol=0, atol=1e-16)


@pytest.mark.parametrize("lat,golden", [(0, "bnorm_d2q9.txt"), (1, "bnorm_d3q27.txt")])
def test_bnorm_matches_printed(oracle_mod, lat, golden):
    _, _, b = oracle_mod.tables(lat)
    np.testing.assert_allclose(b, _read_fracs(golden), rtol=1e-14, atol=0)


@pytest.mark.parametrize("lat", [0, 1])
def test_weighted_orthogonality_at_rest(oracle_mod, lat):
    # sum_i w_i T_vi T_li = b_v delta_vl in the local rest frame (Sec. II-B).
    c, w, b = oracle_mod.tables(lat)
    T = oracle_mod.T(lat, [0.0, 0.0, 0.0])
    G = T @ np.diag(w) @ T.T
    np.testing.assert_allclose(G, np.diag(b), atol=1e-15)


@pytest.mark.parametrize("lat", [0, 1])
def test_T_is_M_of_shifted_velocity(oracle_mod, lat):
    # T = N M with M = T(0) and N = M^{-1} T ... check T(u) f = sum f M(c - u) directly.
    rng = np.random.default_rng(1)
    c, w, _ = oracle_mod.tables(lat)
    Q = len(w)
    u = rng.uniform(-0.1, 0.1, 3)
    if lat == 0:
        u[2] = 0.0
    T = oracle_mod.T(lat, u)
    for i in range(Q):
        for v in range(Q):
            assert T[v, i] == oracle_mod.basis(lat, v, c[i] - u)
    # k_{lm} = sum f cbar_x^l cbar_y^m for the pure powers in the basis.
    f = rng.uniform(0.0, 0.2, Q)
    cb = c - u
    assert (T @ f)[0] == pytest.approx(f.sum(), rel=1e-14)
    assert (T @ f)[1] == pytest.approx((f * cb[:, 0]).sum(), abs=1e-14)
    assert (T @ f)[2] == pytest.approx((f * cb[:, 1]).sum(), abs=1e-14)


def test_printed_m15_is_a_typo():
    # Sec. II-C prints M_15 = cy^2 cz - cs^2 cy; with that form <M_15, M_3>_w != 0,
    # contradicting the printed orthogonality. The reading cy^2 cz - cs^2 cz restores it
    # and gives the printed b_15 = 2/27.
    c = np.array(list(itertools.product((-1, 0, 1), repeat=3)), dtype=float)
    w = np.prod(np.where(c == 0, 2 / 3, 1 / 6), axis=1)
    cx, cy, cz = c.T
    printed = cy ** 2 * cz - CS2 * cy
    reading = cy ** 2 * cz - CS2 * cz
    assert abs((w * printed * cz).sum()) > 1e-3
    assert abs((w * reading * cz).sum()) < 1e-15
    assert (w * reading ** 2).sum() == pytest.approx(2 / 27, rel=1e-14)


def test_d2q9_printed_precollision_moments(oracle_mod):
    # Sec. II-B: k4 = r4 - rho (ux^2 - uy^2), r4 = f1 - f2 + f3 - f4;
    #            k5 = r5 - rho ux uy,        r5 = f5 - f6 + f7 - f8.
    rng = np.random.default_rng(2)
    c, w, _ = oracle_mod.tables(0)
    for _ in range(20):
        f = w * (1.0 + rng.uniform(-0.2, 0.2, 9))
        rho = f.sum()
        ux, uy = (f[:, None] * c[:, :2]).sum(0) / rho
        k = oracle_mod.T(0, [ux, uy, 0.0]) @ f
        r4 = f[1] - f[2] + f[3] - f[4]
        r5 = f[5] - f[6] + f[7] - f[8]
        assert k[4] == pytest.approx(r4 - rho * (ux * ux - uy * uy), abs=1e-15)
        assert k[5] == pytest.approx(r5 - rho * ux * uy, abs=1e-15)
        assert abs(k[1]) < 1e-15 and abs(k[2]) < 1e-15


def test_d3q27_printed_shear_moments(oracle_mod):
    # Sec. II-C prints k7, k8, k9 as signed population sums minus rho u_a u_b.
    rng = np.random.default_rng(3)
    c, w, _ = oracle_mod.tables(1)
    s7 = {7: 1, 8: -1, 9: -1, 10: 1, 19: 1, 20: -1, 21: -1, 22: 1, 23: 1, 24: -1, 25: -1, 26: 1}
    s8 = {11: 1, 12: -1, 13: -1, 14: 1, 19: 1, 20: -1, 21: 1, 22: -1, 23: -1, 24: 1, 25: -1, 26: 1}
    s9 = {15: 1, 16: -1, 17: -1, 18: 1, 19: 1, 20: 1, 21: -1, 22: -1, 23: -1, 24: -1, 25: 1, 26: 1}
    for _ in range(20):
        f = w * (1.0 + rng.uniform(-0.2, 0.2, 27))
        rho = f.sum()
        u = (f[:, None] * c).sum(0) / rho
        k = oracle_mod.T(1, u) @ f
        for v, s, (a, b) in ((7, s7, (0, 1)), (8, s8, (0, 2)), (9, s9, (1, 2))):
            printed = sum(sg * f[i] for i, sg in s.items()) - rho * u[a] * u[b]
            assert k[v] == pytest.approx(printed, abs=1e-15)


def test_second_order_equilibrium_offsets(oracle_mod):
    # Sec. II-B prints k^eq for a second-order truncated equilibrium: only the ghost
    # modes 6, 7, 8 carry velocity-dependent offsets. This pins rows 6-8 of T(u).
    rows = np.loadtxt(os.path.join(GOLDEN, "k2nd_order_d2q9.txt"))
    c, w, _ = oracle_mod.tables(0)
    rng = np.random.default_rng(4)
    for _ in range(10):
        rho = rng.uniform(0.5, 2.0)
        u = np.array([*rng.uniform(-0.15, 0.15, 2), 0.0])
        cu = c @ u
        f2 = w * rho * (1 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - (u @ u) / (2 * CS2))
        k = oracle_mod.T(0, u) @ f2
        for v, coef, px, py in rows:
            expect = coef * rho * u[0] ** px * u[1] ** py
            assert k[int(v)] == pytest.approx(expect, rel=1e-12, abs=1e-15)


def test_hermite_recursion_reproduces_printed_orders(oracle_mod):
    # H^(2), H^(3), H^(4) as printed in Sec. II-B after Eq. feq.
    d = lambda a, b: 1.0 if a == b else 0.0  # noqa: E731
    for cv in itertools.product((-1, 0, 1), repeat=3):
        c = np.array(cv, dtype=float)
        for a, b in itertools.product(range(3), repeat=2):
            assert oracle_mod.hermite(cv, [a, b]) == pytest.approx(c[a] * c[b] - CS2 * d(a, b), abs=1e-15)
        for a, b, g in itertools.product(range(3), repeat=3):
            e = c[a] * c[b] * c[g] - CS2 * (c[a] * d(b, g) + c[b] * d(a, g) + c[g] * d(a, b))
            assert oracle_mod.hermite(cv, [a, b, g]) == pytest.approx(e, abs=1e-15)
        for a, b, g, dd in itertools.product(range(3), repeat=4):
            e = (c[a] * c[b] * c[g] * c[dd]
                 - CS2 * (c[a] * c[b] * d(g, dd) + c[a] * c[g] * d(b, dd) + c[a] * c[dd] * d(b, g)
                          + c[b] * c[g] * d(a, dd) + c[b] * c[dd] * d(a, g) + c[g] * c[dd] * d(a, b))
                 + CS2 ** 2 * (d(a, b) * d(g, dd) + d(a, g) * d(b, dd) + d(a, dd) * d(b, g)))
            assert oracle_mod.hermite(cv, [a, b, g, dd]) == pytest.approx(e, abs=1e-15)
