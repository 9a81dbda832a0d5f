"""Pins of the oracle's equilibrium and collision against the paper's printed algebra,
closed forms and the Ornstein-Uhlenbeck statistics each mode must follow."""
import numpy as np
import pytest

CS2 = 1.0 / 3.0


def _product_feq(c, rho, u):
    # f^eq = rho prod_a g(c_a, u_a), g(0,u) = 2/3 - u^2, g(+-1,u) = 1/6 (1 +- 3u + 3u^2):
    # the tensor-product form of the full Hermite equilibrium (textbook closed form).
    g = np.where(c == 0, 2 / 3 - u ** 2, (1 + 3 * c * u + 3 * u ** 2) / 6)
    return rho * np.prod(g, axis=1)


@pytest.mark.parametrize("lat", [0, 1])
def test_feq_equals_product_form(oracle_mod, lat):
    c, w, _ = oracle_mod.tables(lat)
    D = 2 if lat == 0 else 3
    rng = np.random.default_rng(10)
    for _ in range(50):
        rho = rng.uniform(0.3, 3.0)
        u = np.zeros(3)
        u[:D] = rng.uniform(-0.3, 0.3, D)
        np.testing.assert_allclose(oracle_mod.feq(lat, rho, u), _product_feq(c[:, :D], rho, u[:D]),
                                   rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("lat", [0, 1])
def test_feq_central_moments_and_hydro_moments(oracle_mod, lat):
    # k^eq = T f^eq = (rho, 0, ..., 0) (Sec. II-B, II-C) and the Euler-level moments.
    c, w, _ = oracle_mod.tables(lat)
    D = 2 if lat == 0 else 3
    Q = len(w)
    rng = np.random.default_rng(11)
    for _ in range(30):
        rho = rng.uniform(0.3, 3.0)
        u = np.zeros(3)
        u[:D] = rng.uniform(-0.2, 0.2, D)
        f = oracle_mod.feq(lat, rho, u)
        k = oracle_mod.T(lat, u) @ f
        assert k[0] == pytest.approx(rho, rel=1e-14)
        np.testing.assert_allclose(k[1:], np.zeros(Q - 1), atol=1e-14 * rho)
        assert f.sum() == pytest.approx(rho, rel=1e-14)
        np.testing.assert_allclose((f[:, None] * c).sum(0), rho * u, atol=1e-15)
        P = np.einsum("i,ia,ib->ab", f, c[:, :D], c[:, :D])
        np.testing.assert_allclose(P, rho * (CS2 * np.eye(D) + np.outer(u[:D], u[:D])), atol=1e-15)


def _printed_prefactors(lat, rho, kBT, omega):
    """phi_v as printed next to each k*_v (Sec. II-B for D2Q9, Sec. II-C for D3Q27),
    with the paper's relaxation: D2Q9 L4 = L5 = omega, D3Q27 L7-9 = omega, others 1."""
    cs = np.sqrt(CS2)
    s = rho * kBT
    om = omega * (2 - omega)
    if lat == 0:
        return {3: 2 * np.sqrt(s * CS2), 4: 2 * np.sqrt(s * CS2 * om), 5: np.sqrt(s * CS2 * om),
                6: np.sqrt(2 * s) * CS2, 7: np.sqrt(2 * s) * CS2, 8: 2 * np.sqrt(s) * cs ** 3}
    p = {}
    for v in (4, 5, 6):
        p[v] = np.sqrt(2 * s * CS2)
    for v in (7, 8, 9):
        p[v] = np.sqrt(s * CS2 * om)
    for v in range(10, 16):
        p[v] = np.sqrt(2 * s) * CS2
    p[16] = np.sqrt(s) * CS2
    for v in (17, 18, 19):
        p[v] = 2 * np.sqrt(s) * cs ** 3
    for v in (20, 21, 22):
        p[v] = np.sqrt(2 * s) * cs ** 3
    for v in (23, 24, 25):
        p[v] = 2 * np.sqrt(s) * cs ** 4
    p[26] = np.sqrt(8 * s) * cs ** 5
    return p


def _paper_lambda(lat, omega):
    if lat == 0:
        lam = np.ones(9)
        lam[[4, 5]] = omega
    else:
        lam = np.ones(27)
        lam[[7, 8, 9]] = omega
    return lam


@pytest.mark.parametrize("lat", [0, 1])
def test_collision_matches_printed_kstar(oracle_mod, lat):
    # Post-collision central moments printed in Sec. II-B (D2Q9) and Sec. II-C (D3Q27).
    c, w, _ = oracle_mod.tables(lat)
    Q = len(w)
    D = 2 if lat == 0 else 3
    rng = np.random.default_rng(12)
    for _ in range(20):
        omega = rng.uniform(0.2, 1.95)
        kBT = rng.uniform(1e-5, 1e-2)
        f = w * (1.0 + rng.uniform(-0.1, 0.1, Q))
        rho = f.sum()
        eta = rng.standard_normal(Q)
        lam = _paper_lambda(lat, omega)
        fs, k = oracle_mod.collide_site(lat, f, lam, kBT, eta)
        u = (f[:, None] * c).sum(0) / rho
        ks = oracle_mod.T(lat, u) @ fs
        pref = _printed_prefactors(lat, rho, kBT, omega)
        assert ks[0] == pytest.approx(rho, rel=1e-13)
        np.testing.assert_allclose(ks[1:D + 1], 0.0, atol=1e-14)
        for v in range(D + 1, Q):
            expect = (1 - lam[v]) * k[v] + pref[v] * eta[v]
            assert ks[v] == pytest.approx(expect, rel=1e-10, abs=1e-15)


def test_d2q9_inverse_transform_matches_printed(oracle_mod):
    # r* = N^{-1} k* and f* = M^{-1} r* printed explicitly in Sec. II-B.
    c, w, b = oracle_mod.tables(0)
    rng = np.random.default_rng(13)
    for _ in range(30):
        rho = rng.uniform(0.5, 2.0)
        ux, uy = rng.uniform(-0.2, 0.2, 2)
        kBT = 1e-3
        kst = np.zeros(9)
        kst[3:] = rng.uniform(-0.05, 0.05, 6)
        # Reach an arbitrary k* with L = 1 on every noisy mode: k*_v = phi_v eta_v.
        lam = np.ones(9)
        phi = np.sqrt(rho * kBT * b / CS2)
        eta = np.zeros(9)
        eta[3:] = kst[3:] / phi[3:]
        f_in = oracle_mod.feq(0, rho, [ux, uy, 0.0])
        fs, _ = oracle_mod.collide_site(0, f_in, lam, kBT, eta)
        k0, k3, k4, k5, k6, k7, k8 = rho, *kst[3:]
        r = np.zeros(9)
        r[0] = k0
        r[1] = rho * ux
        r[2] = rho * uy
        r[3] = k3 + rho * (ux ** 2 + uy ** 2)
        r[4] = k4 + rho * (ux ** 2 - uy ** 2)
        r[5] = k5 + rho * ux * uy
        r[6] = k6 + 2 * ux * k5 + 0.5 * uy * (k3 + k4) + rho * ux ** 2 * uy
        r[7] = k7 + 2 * uy * k5 + 0.5 * ux * (k3 - k4) + rho * ux * uy ** 2
        r[8] = (k8 + 2 * (ux * k7 + uy * k6) + 4 * ux * uy * k5 - 0.5 * (ux ** 2 - uy ** 2) * k4
                + 0.5 * (ux ** 2 + uy ** 2) * k3 + rho * ux ** 2 * uy ** 2)
        fp = np.array([
            4 * r[0] / 9 - 2 * r[3] / 3 + r[8],
            r[0] / 9 + r[1] / 3 + r[3] / 12 + r[4] / 4 - (r[7] + r[8]) / 2,
            r[0] / 9 + r[2] / 3 + r[3] / 12 - r[4] / 4 - (r[6] + r[8]) / 2,
            r[0] / 9 - r[1] / 3 + r[3] / 12 + r[4] / 4 + (r[7] - r[8]) / 2,
            r[0] / 9 - r[2] / 3 + r[3] / 12 - r[4] / 4 + (r[6] - r[8]) / 2,
            r[0] / 36 + (r[1] + r[2] + r[3]) / 12 + (r[5] + r[6] + r[7] + r[8]) / 4,
            r[0] / 36 + (-r[1] + r[2] + r[3]) / 12 + (-r[5] + r[6] - r[7] + r[8]) / 4,
            r[0] / 36 + (-r[1] - r[2] + r[3]) / 12 + (r[5] - r[6] - r[7] + r[8]) / 4,
            r[0] / 36 + (r[1] - r[2] + r[3]) / 12 + (-r[5] - r[6] + r[7] + r[8]) / 4,
        ])
        np.testing.assert_allclose(fs, fp, rtol=1e-12, atol=1e-15)


def test_d2q9_closed_form_rest_population(oracle_mod):
    # Deterministic f0* printed in Sec. III (Test 2 discussion), paper relaxation rates.
    c, w, _ = oracle_mod.tables(0)
    rng = np.random.default_rng(14)
    for _ in range(30):
        omega = rng.uniform(0.3, 1.9)
        f = w * (1.0 + rng.uniform(-0.2, 0.2, 9))
        rho = f.sum()
        ux, uy = (f[:, None] * c[:, :2]).sum(0) / rho
        fs, _ = oracle_mod.collide_site(0, f, _paper_lambda(0, omega), 0.0, np.zeros(9))
        k4 = f[1] - f[2] + f[3] - f[4] - rho * (ux ** 2 - uy ** 2)
        k5 = f[5] - f[6] + f[7] - f[8] - rho * ux * uy
        f0 = (rho * (ux ** 2 * uy ** 2 - 2 * CS2 * (ux ** 2 + uy ** 2) + 4 * CS2 ** 2)
              + (uy ** 2 - ux ** 2) / 2 * (1 - omega) * k4 + 4 * ux * uy * (1 - omega) * k5)
        assert fs[0] == pytest.approx(f0, rel=1e-12)


@pytest.mark.parametrize("lat", [0, 1])
def test_uniform_rate_is_bgk(oracle_mod, lat):
    # L = omega I and kBT = 0 reduce the scheme to BGK (Sec. II-C, last paragraph).
    c, w, _ = oracle_mod.tables(lat)
    Q = len(w)
    D = 2 if lat == 0 else 3
    rng = np.random.default_rng(15)
    for _ in range(20):
        omega = rng.uniform(0.2, 1.95)
        f = w * (1.0 + rng.uniform(-0.2, 0.2, Q))
        rho = f.sum()
        u = (f[:, None] * c).sum(0) / rho
        fs, _ = oracle_mod.collide_site(lat, f, np.full(Q, omega), 0.0, np.zeros(Q))
        fe = _product_feq(c[:, :D], rho, u[:D])
        np.testing.assert_allclose(fs, f + omega * (fe - f), rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("lat", [0, 1])
def test_collision_conserves_mass_and_momentum(oracle_mod, lat):
    c, w, _ = oracle_mod.tables(lat)
    Q = len(w)
    rng = np.random.default_rng(16)
    for _ in range(30):
        f = w * (1.0 + rng.uniform(-0.3, 0.3, Q))
        lam = rng.uniform(0.05, 1.99, Q)
        fs, _ = oracle_mod.collide_site(lat, f, lam, 1e-3, rng.standard_normal(Q))
        assert fs.sum() == pytest.approx(f.sum(), rel=1e-14)
        np.testing.assert_allclose((fs[:, None] * c).sum(0), (f[:, None] * c).sum(0), atol=1e-15)


@pytest.mark.parametrize("lat,iters", [(0, 40000), (1, 12000)])
def test_single_site_ornstein_uhlenbeck(oracle_mod, lat, iters):
    # Collision only at one site (no streaming): every noisy mode is a discrete OU
    # process k' = (1-L) k + phi eta, whose stationary variance is the equilibrium
    # variance rho kBT b_v / cs^2 (Sec. II-B, C^eq diagonal) and whose lag-1
    # autocorrelation is 1 - L. Off-diagonal covariances vanish.
    c, w, b = oracle_mod.tables(lat)
    Q = len(w)
    D = 2 if lat == 0 else 3
    rng = np.random.default_rng(17)
    lam = np.ones(Q)
    lam[D + 1:] = rng.uniform(0.4, 1.9, Q - D - 1)
    kBT, rho = 2e-4, 1.3
    f = oracle_mod.feq(lat, rho, [0, 0, 0])
    ks = np.empty((iters, Q))
    for t in range(iters):
        f, k = oracle_mod.collide_site(lat, f, lam, kBT, rng.standard_normal(Q))
        ks[t] = k
    ks = ks[200:]
    var_target = rho * kBT * b / CS2
    for v in range(D + 1, Q):
        x = ks[:, v]
        a = 1 - lam[v]
        n_eff = len(x) * (1 - a * a) / (1 + a * a)
        rel_sigma = np.sqrt(2.0 / n_eff)
        assert x.var() / var_target[v] == pytest.approx(1.0, abs=5 * rel_sigma), v
        ac = np.corrcoef(x[:-1], x[1:])[0, 1]
        assert ac == pytest.approx(a, abs=5 / np.sqrt(len(x)) + 0.01), v
    z = ks[:, D + 1:] / np.sqrt(var_target[D + 1:])
    C = np.corrcoef(z.T)
    off = C[~np.eye(len(C), dtype=bool)]
    assert np.abs(off).max() < 6 / np.sqrt(len(z) * 0.3)
