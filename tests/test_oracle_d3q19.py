"""Pins of the oracle's D3Q19 lattice (id 3; Sec. II-C, "Lattice-agnostic construction
and the D3Q19 example"): the printed basis and norms, the equilibrium read as
T(u)^{-1} (rho, 0, ..., 0) (the printed populations do not conserve mass as transcribed)
checked against the moments a second-order Hermite-consistent equilibrium must have,
the printed post-collision noise prefactors, conservation and the shear viscosity."""
import os
from fractions import Fraction

import numpy as np
import pytest

D3Q19 = 3
CS2 = 1.0 / 3.0
HERE = os.path.dirname(os.path.abspath(__file__))


def _golden(name):
    rows = []
    with open(os.path.join(HERE, "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_velocities_weights_and_printed_norms(oracle_mod):
    c, w, b = oracle_mod.tables(D3Q19)
    assert len(w) == 19
    speed2 = (c ** 2).sum(1)
    assert sorted(speed2) == [0] + [1] * 6 + [2] * 12
    assert len({tuple(v) for v in c}) == 19
    np.testing.assert_allclose(w, np.where(speed2 == 0, 1 / 3, np.where(speed2 == 1, 1 / 18, 1 / 36)), atol=1e-16)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    printed = [float(Fraction(r[0])) for r in _golden("bnorm_d3q19.txt")]
    np.testing.assert_allclose(b, printed, rtol=1e-14)
    T = oracle_mod.T(D3Q19, [0.0, 0.0, 0.0])
    np.testing.assert_allclose((T * w) @ T.T, np.diag(b), atol=1e-15)


@pytest.mark.parametrize("u", [(0.0, 0.0, 0.0), (0.08, -0.05, 0.03), (-0.02, 0.1, 0.0)])
def test_equilibrium_moments(oracle_mod, u):
    rho = 1.3
    c, w, _ = oracle_mod.tables(D3Q19)
    f = oracle_mod.feq(D3Q19, rho, u)
    u = np.array(u)
    cf = c.astype(float)
    assert f.sum() == pytest.approx(rho, rel=1e-14)
    np.testing.assert_allclose(cf.T @ f, rho * u, atol=1e-15)
    # second moments of a Hermite-consistent equilibrium: rho (cs^2 delta + u u)
    P = np.einsum("ia,ib,i->ab", cf, cf, f)
    np.testing.assert_allclose(P, rho * (CS2 * np.eye(3) + np.outer(u, u)), atol=1e-14)
    k = oracle_mod.T(D3Q19, u) @ f
    assert k[0] == pytest.approx(rho, rel=1e-14)
    assert np.abs(k[1:]).max() < 1e-14
    if not u.any():
        np.testing.assert_allclose(f, rho * w, rtol=1e-14)


def test_printed_noise_prefactors(oracle_mod):
    # With Lambda = 1 except Lambda_7-9 = omega, k*_v - (1 - Lambda_v) k_v = A_v eta_v with
    # the printed A_v (the paper's Eq. phi_general with the D3Q19 norms).
    omega, rho, kbt = 1.6, 1.1, 3e-4
    lam = np.ones(19)
    lam[7:10] = omega
    rng = np.random.default_rng(4)
    eta = rng.standard_normal(19)
    u = (0.03, -0.02, 0.01)
    f = oracle_mod.feq(D3Q19, rho, u) * (1.0 + 0.01 * rng.standard_normal(19))
    f *= rho / f.sum()
    fs, k = oracle_mod.collide_site(D3Q19, f, lam, kbt, eta)
    c, _, _ = oracle_mod.tables(D3Q19)
    rho_s = f.sum()
    ustar = (c.T.astype(float) @ fs) / fs.sum()
    np.testing.assert_allclose(ustar, (c.T.astype(float) @ f) / rho_s, atol=1e-14)
    kstar = oracle_mod.T(D3Q19, ustar) @ fs
    wfac = omega * (2.0 - omega)
    for v, a2 in _golden("d3q19_kstar_prefactors.txt"):
        v = int(v)
        A2 = wfac / float(Fraction(a2[2:])) if a2.startswith("w/") else float(Fraction(a2))
        expect = (1.0 - lam[v]) * k[v] + np.sqrt(A2 * rho_s * kbt) * eta[v]
        assert kstar[v] == pytest.approx(expect, rel=1e-10, abs=1e-15), v


def test_run_conserves_mass_and_momentum(oracle_mod):
    c, _, _ = oracle_mod.tables(D3Q19)
    lam = np.ones(19)
    lam[4:] = np.random.default_rng(2).uniform(0.5, 1.9, 15)
    f0 = oracle_mod.init_uniform(D3Q19, (6, 5, 4), 1.0, (0.04, -0.02, 0.01), 1e-2, 9)
    f = oracle_mod.run(D3Q19, (6, 5, 4), lam, 1e-3, 3, f0, 0, 15)
    assert f.sum() == pytest.approx(f0.sum(), rel=1e-13)
    cf = c.astype(float)
    np.testing.assert_allclose(cf.T @ f.reshape(19, -1).sum(1), cf.T @ f0.reshape(19, -1).sum(1), atol=1e-12)
    assert np.abs(f - f0).max() > 1e-4


def test_shear_wave_decays_at_the_shear_viscosity(oracle_mod):
    # u_x = U sin(2 pi y / n) relaxes through the xy shear mode (Lambda_7 = omega):
    # u(t) = u(0) exp(-nu k^2 t), nu = cs^2 (1/omega - 1/2).
    n, U, omega = 32, 1e-3, 1.4
    dims = (2, n, 2)
    lam = np.ones(19)
    lam[7:10] = omega
    c, _, _ = oracle_mod.tables(D3Q19)
    k = 2.0 * np.pi / n
    f = np.zeros((19, 2, n, 2))
    for y in range(n):
        fe = oracle_mod.feq(D3Q19, 1.0, (U * np.sin(k * y), 0.0, 0.0))
        f[:, :, y, :] = fe[:, None, None]

    def amp(f):
        ux = np.einsum("i,i...->...", c[:, 0].astype(float), f) / f.sum(0)
        return 2.0 * np.mean(ux[0, :, 0] * np.sin(k * np.arange(n)))

    # rate between steps 50 and 250 (after the start-up transient of an equilibrium start)
    f = oracle_mod.run(D3Q19, dims, lam, 0.0, 0, f, 0, 50)
    a0 = amp(f)
    f = oracle_mod.run(D3Q19, dims, lam, 0.0, 0, f, 50, 200)
    rate = np.log(a0 / amp(f)) / 200
    nu = CS2 * (1.0 / omega - 0.5)
    # the lattice's O(k^2) dispersion at 32 points per wavelength stays below 1 %
    assert rate == pytest.approx(nu * k * k, rel=1e-2)
