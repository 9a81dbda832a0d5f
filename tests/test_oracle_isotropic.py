"""Pins of the oracle's isotropic D3Q27 variant (lattice id 2): the paper relaxes the
D3Q27 normal-stress modes 4-6 at rate 1 and only the shear modes 7-9 at omega
(Sec. II-C), so the deterministic viscosity differs between shear and extensional
flow. The variant replaces modes 4-6 by their trace and two deviators; these pins fix
it by the mathematics (orthogonality with closed-form norms, equilibrium, agreement
with the paper's variant where their rates coincide) and by the physics it is for
(3-D Taylor-Green decay at one viscosity)."""
import numpy as np
import pytest

CS2 = 1.0 / 3.0
ISO, D3Q27 = 2, 1


def test_iso_basis_orthogonal_with_closed_form_norms(oracle_mod):
    c, w, b = oracle_mod.tables(ISO)
    _, w1, b1 = oracle_mod.tables(D3Q27)
    assert np.array_equal(w, w1)
    M = np.array([[oracle_mod.basis(ISO, v, c[i]) for i in range(27)] for v in range(27)])
    G = (M * w) @ M.T
    np.testing.assert_allclose(G, np.diag(np.diag(G)), atol=1e-15)
    # trace: 3 x 2/9; deviators (1,-1,0): 2 x 2/9 and (1,1,-2): 6 x 2/9; the rest unchanged
    np.testing.assert_allclose(b[4:7], [2.0 / 3.0, 4.0 / 9.0, 4.0 / 3.0], rtol=1e-15)
    np.testing.assert_allclose(np.delete(b, [4, 5, 6]), np.delete(b1, [4, 5, 6]), rtol=1e-15)


@pytest.mark.parametrize("u", [(0.0, 0.0, 0.0), (0.05, -0.03, 0.02)])
def test_iso_equilibrium_central_moments(oracle_mod, u):
    f = oracle_mod.feq(ISO, 1.2, u)
    k = oracle_mod.T(ISO, u) @ f
    assert k[0] == pytest.approx(1.2, rel=1e-14)
    assert np.abs(k[1:]).max() < 1e-14


def test_iso_equals_paper_variant_when_normal_rates_are_one(oracle_mod):
    # With Lambda_4..6 = 1 both variants restart the whole normal-stress space from its
    # equilibrium, so the deterministic collisions coincide.
    rng = np.random.default_rng(3)
    lam = np.ones(27)
    lam[7:10] = 1.7
    lam[10:] = rng.uniform(0.5, 1.9, 17)
    for _ in range(5):
        f = oracle_mod.feq(1, 1.0 + 0.01 * rng.standard_normal(), 0.05 * rng.standard_normal(3))
        f = f * (1.0 + 0.02 * rng.standard_normal(27))
        a, _ = oracle_mod.collide_site(D3Q27, f, lam, 0.0, np.zeros(27))
        b, _ = oracle_mod.collide_site(ISO, f, lam, 0.0, np.zeros(27))
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-15)


def _tg_energy_rate(oracle_mod, lat, lam, n=16, steps=(20, 80), U=0.01):
    # 3-D Taylor-Green vortex u = U (sin x cos y cos z, -cos x sin y cos z, 0), k = 2 pi / n.
    # Incompressible decay of the kinetic energy: exp(-2 nu 3 k^2 t).
    c, w, _ = oracle_mod.tables(lat)
    k = 2.0 * np.pi / n
    x = np.arange(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    ux = U * np.sin(k * X) * np.cos(k * Y) * np.cos(k * Z)
    uy = -U * np.cos(k * X) * np.sin(k * Y) * np.cos(k * Z)
    f = np.zeros((27, n, n, n))
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                f[:, iz, iy, ix] = oracle_mod.feq(lat, 1.0, (ux[iz, iy, ix], uy[iz, iy, ix], 0.0))

    def energy(f):
        rho = f.sum(0)
        j = np.einsum("ia,i...->a...", c.astype(float), f)
        return 0.5 * float((j ** 2 / rho).sum())

    f1 = oracle_mod.run(lat, (n, n, n), lam, 0.0, 0, f, 0, steps[0])
    f2 = oracle_mod.run(lat, (n, n, n), lam, 0.0, 0, f1, steps[0], steps[1] - steps[0])
    return np.log(energy(f1) / energy(f2)) / (steps[1] - steps[0]), k


@pytest.mark.slow
def test_taylor_green_3d_one_viscosity_only_in_the_iso_variant(oracle_mod):
    omega = 1.8
    nu = CS2 * (1.0 / omega - 0.5)
    # Isotropic variant: deviators at the shear rate, trace (bulk) at 1.
    lam_iso = np.ones(27)
    lam_iso[[5, 6, 7, 8, 9]] = omega
    rate_iso, k = _tg_energy_rate(oracle_mod, ISO, lam_iso)
    expected = 2.0 * nu * 3.0 * k * k
    assert rate_iso == pytest.approx(expected, rel=0.03)
    # The paper's variant (normal stresses at rate 1, extensional viscosity cs^2/2)
    # dissipates this vortex measurably faster.
    lam_paper = np.ones(27)
    lam_paper[[7, 8, 9]] = omega
    rate_paper, _ = _tg_energy_rate(oracle_mod, D3Q27, lam_paper)
    assert rate_paper > 1.15 * expected
