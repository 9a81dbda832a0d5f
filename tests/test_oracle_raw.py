"""Pins of the oracle's raw-moment collision (model RAW: T = M, N = I), the comparison
scheme of the paper. Sec. II-C (end of the D3Q27 construction) identifies the choice T = M,
N = I as the raw-moment form of the scheme and a single rate Lambda = omega I as BGK; with
that rate the update must be the fluctuating BGK operator of Sec. II-A (relaxation
omega (f^eq - f) plus the noise zeta_i of Eq. Xi_pop).

Expected values come from the paper's formulas written out here with the printed basis
polynomials (tests/_paper_basis.py), the printed norms (golden files) and the closed product
form of the equilibrium, not from the oracle's transform matrices."""
import os
from fractions import Fraction

import numpy as np
import pytest

from _paper_basis import CS2, matrix

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RAW = 1


def _printed_b(lat):
    name = {0: "bnorm_d2q9.txt", 1: "bnorm_d3q27.txt"}[lat]
    vals = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            vals.append(float(Fraction(line)))
    return np.array(vals)


def _feq_product(c, rho, u, D):
    def g(ci, ua):
        return np.where(ci == 0, 2.0 / 3.0 - ua * ua, 1.0 / 6.0 + ci * ua / 2.0 + ua * ua / 2.0)

    out = rho * np.ones(len(c))
    for a in range(D):
        out = out * g(c[:, a], u[a])
    return out


def _state(oracle_mod, lat, seed, drift=(0.06, -0.04, 0.03)):
    c, w, _ = oracle_mod.tables(lat)
    rng = np.random.default_rng(seed)
    D = 2 if lat == 0 else 3
    u = np.array(drift[:D] + (0.0,) * (3 - D))
    f = _feq_product(c, 1.07, u, D) * (1.0 + 0.05 * rng.uniform(-1, 1, len(w)))
    return c, w, D, f


@pytest.mark.parametrize("lat", [0, 1])
def test_bgk_closed_form_without_noise(oracle_mod, lat):
    # Sec. II-A: f* = f + omega (f^eq - f) with f^eq at the site's rho and u.
    c, w, D, f = _state(oracle_mod, lat, 3)
    Q = len(w)
    for omega in (0.7, 1.0, 1.6, 1.95):
        lam = np.full(Q, omega)
        fs, _ = oracle_mod.collide_site(lat, f, lam, 0.0, np.zeros(Q), model=RAW)
        rho = f.sum()
        u = (c.T @ f) / rho
        expect = f + omega * (_feq_product(c, rho, u, D) - f)
        np.testing.assert_allclose(fs, expect, rtol=0, atol=1e-14)


@pytest.mark.parametrize("lat", [0, 1])
def test_bgk_noise_is_eq_xi_pop(oracle_mod, lat):
    # The stochastic part of the fluctuating BGK step is zeta_i = w_i sum_v b_v^-1 e_vi phi_v eta_v
    # over the non-conserved modes (Eq. Xi_pop), e_v the rest-frame basis vectors and
    # phi_v = sqrt(rho kBT omega (2 - omega) b_v / cs^2) (Eq. phi_general).
    c, w, D, f = _state(oracle_mod, lat, 4)
    Q = len(w)
    b = _printed_b(lat)
    M = matrix(lat, c)
    rng = np.random.default_rng(9)
    eta = rng.standard_normal(Q)
    omega, kBT = 1.45, 3e-4
    lam = np.full(Q, omega)
    fs, _ = oracle_mod.collide_site(lat, f, lam, kBT, eta, model=RAW)
    det, _ = oracle_mod.collide_site(lat, f, lam, 0.0, np.zeros(Q), model=RAW)
    rho = f.sum()
    phi = np.sqrt(rho * kBT * omega * (2.0 - omega) * b / CS2)
    zeta = w * sum(M[v] * phi[v] * eta[v] / b[v] for v in range(D + 1, Q))
    np.testing.assert_allclose(fs - det, zeta, rtol=0, atol=1e-15)
    # zeta carries no mass and no momentum
    assert abs(zeta.sum()) < 1e-16 and np.abs(c.T @ zeta).max() < 1e-16


@pytest.mark.parametrize("lat", [0, 1])
def test_raw_mrt_relaxes_raw_moments(oracle_mod, lat):
    # Mode-dependent rates on the raw moments r = M f: r*_v = (1 - L_v) r_v + L_v r^eq_v,
    # r^eq = M f^eq; conserved rows (v <= D) unchanged.
    c, w, D, f = _state(oracle_mod, lat, 5)
    Q = len(w)
    rng = np.random.default_rng(2)
    lam = rng.uniform(0.3, 1.9, Q)
    fs, r_pre = oracle_mod.collide_site(lat, f, lam, 0.0, np.zeros(Q), model=RAW)
    M = matrix(lat, c)
    rho = f.sum()
    u = (c.T @ f) / rho
    r = M @ f
    req = M @ _feq_product(c, rho, u, D)
    np.testing.assert_allclose(r_pre, r, rtol=0, atol=1e-14)
    L = np.where(np.arange(Q) <= D, 1.0, lam)
    np.testing.assert_allclose(M @ fs, (1 - L) * r + L * req, rtol=0, atol=1e-14)
    np.testing.assert_allclose((M @ fs)[: D + 1], r[: D + 1], rtol=0, atol=1e-14)


@pytest.mark.parametrize("lat", [0, 1])
def test_raw_equals_central_at_rest(oracle_mod, lat):
    # At u = 0 the shifted basis is the raw one (T(0) = M), so both models coincide.
    c, w, D, f = _state(oracle_mod, lat, 6, drift=(0.0, 0.0, 0.0))
    Q = len(w)
    # remove the momentum exactly: f_i -> f_i - w_i (c_i . j) / cs^2 has zero momentum
    j = c.T @ f
    f = f - w * (c @ j) / CS2
    assert np.abs(c.T @ f).max() < 1e-15
    rng = np.random.default_rng(1)
    lam = rng.uniform(0.3, 1.9, Q)
    eta = rng.standard_normal(Q)
    a, _ = oracle_mod.collide_site(lat, f, lam, 2e-4, eta, model=0)
    b, _ = oracle_mod.collide_site(lat, f, lam, 2e-4, eta, model=RAW)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


@pytest.mark.parametrize("lat,dims", [(0, (9, 7, 1)), (1, (5, 4, 3))])
def test_raw_run_conserves_mass_and_momentum(oracle_mod, lat, dims):
    c, w, _ = oracle_mod.tables(lat)
    Q = len(w)
    f0 = oracle_mod.init_uniform(lat, dims, 1.0, (0.04, -0.02, 0.01), 1e-2, 9)
    lam = np.full(Q, 1.5)
    f = oracle_mod.run(lat, dims, lam, 1e-3, 3, f0, 0, 10, model=RAW)
    assert f.sum() == pytest.approx(f0.sum(), rel=1e-13)
    j0 = c.T.astype(float) @ f0.reshape(Q, -1).sum(1)
    j1 = c.T.astype(float) @ f.reshape(Q, -1).sum(1)
    np.testing.assert_allclose(j1, j0, atol=1e-12)
    assert np.abs(f - f0).max() > 1e-4
