"""Pins of the oracle's statistics (``oracle.stats``): the sums and means of the density,
momentum and velocity and the means and raw second moments of the central moments k_v,
which the GPU statistics reduction is compared with.

Every expected value comes from the paper or from mathematics, by routes the oracle
does not take:
  * a uniform equilibrium state, whose central moments are (rho, 0, ..., 0) (Sec. II-B and
    II-C: all equilibrium central moments vanish except k_0 = rho), built here from the
    closed product form of the equilibrium;
  * a random state, whose central moments are formed here from the raw moments
    sum_i f_i c^l by the binomial theorem (the definition of k_{a^l b^m g^n} in Sec. II-B /
    II-C with cbar = c - u) and combined into modes by the printed basis polynomials, not
    through a shifted transform matrix;
  * the stationary state of the collision alone (a one-site periodic box, where streaming
    is the identity), whose mode covariance is diagonal with entries
    rho kBT b_v / cs^2 (Sec. II-B, C^eq and Eq. phi_general);
  * a state with one non-finite site, which is counted and left out of every sum.
"""
import itertools
import numpy as np
import pytest

from _paper_basis import BASES, CS2  # noqa: E402


def _central_modes(lat, c, f):
    """k[v, site] from raw moments: kappa_lmn = sum_abc C(l,a) C(m,b) C(n,g) (-ux)^(l-a)
    (-uy)^(m-b) (-uz)^(n-g) r_abg, r_abg = sum_i f_i cx^a cy^b cz^g; then the modes by the
    basis polynomials. Returns k, rho, j, u (per site, flattened)."""
    import math

    Q = f.shape[0]
    ff = f.reshape(Q, -1)
    cf = c.astype(float)
    rho = ff.sum(0)
    j = cf.T @ ff
    u = j / rho
    basis = BASES[lat]()
    need = set()
    for p in basis:
        need.update(p.keys())
    raw = {}
    for a, b, g in itertools.product(range(5), repeat=3):
        raw[(a, b, g)] = (cf[:, 0] ** a * cf[:, 1] ** b * cf[:, 2] ** g) @ ff
    kappa = {}
    for (l, m, n) in need:
        acc = np.zeros_like(rho)
        for a in range(l + 1):
            for b in range(m + 1):
                for g in range(n + 1):
                    coef = math.comb(l, a) * math.comb(m, b) * math.comb(n, g)
                    acc = acc + coef * (-u[0]) ** (l - a) * (-u[1]) ** (m - b) * (-u[2]) ** (n - g) * raw[(a, b, g)]
        kappa[(l, m, n)] = acc
    k = np.array([sum(coef * kappa[mono] for mono, coef in p.items()) for p in basis])
    return k, rho, j, u


def _equilibrium_product(c, rho, u, D):
    # f_i^eq = rho prod_a g(c_ia, u_a), g(0, u) = 2/3 - u^2, g(+-1, u) = 1/6 +- u/2 + u^2/2,
    # over the D axes: the complete Hermite equilibrium of Sec. II-B / II-C on
    # tensor-product lattices.
    def g(ci, ua):
        return np.where(ci == 0, 2.0 / 3.0 - ua * ua, 1.0 / 6.0 + ci * ua / 2.0 + ua * ua / 2.0)

    out = rho * np.ones(len(c))
    for a in range(D):
        out = out * g(c[:, a], u[a])
    return out


@pytest.mark.parametrize("lat,dims,u", [(0, (5, 4, 1), (0.07, -0.03, 0.0)),
                                        (1, (3, 4, 2), (0.05, 0.02, -0.04))])
def test_uniform_equilibrium_statistics(oracle_mod, lat, dims, u):
    c, w, _ = oracle_mod.tables(lat)
    Q = len(w)
    rho = 1.3
    u = np.array(u, dtype=float)
    feq = _equilibrium_product(c, rho, u, 2 if lat == 0 else 3)
    N = int(np.prod(dims))
    f = np.repeat(feq[:, None], N, axis=1).reshape(Q, dims[2], dims[1], dims[0])
    st = oracle_mod.stats(lat, dims, f)
    assert st["nonfinite"] == 0 and st["sites"] == N
    assert st["mass"] == pytest.approx(N * rho, rel=1e-14)
    np.testing.assert_allclose(st["mom"], N * rho * u, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(st["u_mean"], u, rtol=1e-13, atol=1e-16)
    uu = [u[0] * u[0], u[1] * u[1], u[2] * u[2], u[0] * u[1], u[0] * u[2], u[1] * u[2]]
    np.testing.assert_allclose(st["uu"], uu, rtol=1e-12, atol=1e-17)
    k_eq = np.zeros(Q)
    k_eq[0] = rho
    np.testing.assert_allclose(st["k_mean"], k_eq, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(st["k_cov"], np.outer(k_eq, k_eq), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("lat,dims", [(0, (6, 5, 1)), (1, (4, 3, 3)), (2, (3, 3, 4)), (3, (4, 3, 2))])
def test_random_state_statistics_from_raw_moments(oracle_mod, lat, dims):
    c, w, _ = oracle_mod.tables(lat)
    Q = len(w)
    rng = np.random.default_rng(11 + lat)
    N = int(np.prod(dims))
    # Populations about w_i with +-30 % fluctuations and a drift: u of order 0.1.
    f = w[:, None] * (1.0 + 0.3 * rng.uniform(-1, 1, (Q, N)))
    f += 0.02 * w[:, None] * c[:, 0:1] * rng.uniform(0.5, 1.5, (1, N))
    f = f.reshape(Q, dims[2], dims[1], dims[0])
    st = oracle_mod.stats(lat, dims, f)
    k, rho, j, u = _central_modes(lat, c, f)
    assert st["nonfinite"] == 0
    assert st["mass"] == pytest.approx(rho.sum(), rel=1e-14)
    np.testing.assert_allclose(st["mom"], j.sum(1), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(st["u_mean"], u.mean(1), rtol=1e-11, atol=1e-15)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    np.testing.assert_allclose(st["uu"], [np.mean(u[a] * u[b]) for a, b in pairs], rtol=1e-11, atol=1e-17)
    # Raw second moments <k_v k_w>, not covariances about the mean: <k_0 k_0> = <rho^2>.
    np.testing.assert_allclose(st["k_mean"], k.mean(1), rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(st["k_cov"], (k @ k.T) / N, rtol=1e-10, atol=1e-15)
    assert st["k_cov"][0, 0] == pytest.approx(np.mean(rho ** 2), rel=1e-13)
    # The conserved central moments k_1..k_D vanish at every site.
    D = 2 if lat == 0 else 3
    np.testing.assert_allclose(st["k_mean"][1:D + 1], 0.0, atol=1e-15)


@pytest.mark.parametrize("lat", [0, 1])
def test_collision_stationary_covariance_is_diagonal_ceq(oracle_mod, lat):
    # One site in a periodic 1x1x1 box: streaming maps the site onto itself, so every
    # step is the collision alone, a discrete Ornstein-Uhlenbeck process per mode whose
    # stationary variance is rho kBT b_v / cs^2 (Eq. phi_general), with zero covariance
    # between modes (C^eq diagonal, Sec. II-B).
    c, w, b = oracle_mod.tables(lat)
    Q = len(w)
    D = 2 if lat == 0 else 3
    lam = np.ones(Q)
    lam[D + 1:] = 1.45
    lam[[4, 5] if lat == 0 else [7, 8, 9]] = 1.7
    kBT, rho0, seed = 2e-4, 1.1, 5
    dims1 = (1, 1, 1)
    f = oracle_mod.init_uniform(lat, dims1, rho0)
    f = oracle_mod.run(lat, dims1, lam, kBT, seed, f, 0, 60)  # forget the start
    n, gap = 3000, 3
    states = np.empty((Q, n))
    step = 60
    for s in range(n):
        f = oracle_mod.run(lat, dims1, lam, kBT, seed, f, step, gap)
        step += gap
        states[:, s] = f.reshape(Q)
    st = oracle_mod.stats(lat, (n, 1, 1), states.reshape(Q, 1, 1, n))
    assert st["nonfinite"] == 0
    # Conserved quantities never move at a single site.
    assert st["mass"] == pytest.approx(n * rho0, rel=1e-13)
    np.testing.assert_allclose(st["u_mean"], 0.0, atol=1e-12)
    target = rho0 * kBT * b / CS2
    cov = st["k_cov"][D + 1:, D + 1:] - np.outer(st["k_mean"][D + 1:], st["k_mean"][D + 1:])
    var = np.diag(cov)
    # Sampling error of a variance from ~n independent draws: sqrt(2/n) = 2.6 %; 5 sigma.
    np.testing.assert_allclose(var / target[D + 1:], 1.0, atol=5 * np.sqrt(2.0 / n))
    corr = cov / np.sqrt(np.outer(var, var))
    off = corr[~np.eye(Q - D - 1, dtype=bool)]
    assert np.abs(off).max() < 5.0 / np.sqrt(n)
    # The means of the non-conserved modes vanish (k^eq_v = 0 for v > 0).
    assert np.all(np.abs(st["k_mean"][D + 1:]) < 5 * np.sqrt(target[D + 1:] / n))


@pytest.mark.parametrize("lat,dims", [(0, (6, 4, 1)), (1, (3, 3, 3))])
def test_non_finite_site_is_counted_and_left_out(oracle_mod, lat, dims):
    c, w, _ = oracle_mod.tables(lat)
    Q = len(w)
    rng = np.random.default_rng(3)
    N = int(np.prod(dims))
    f = (w[:, None] * (1.0 + 0.2 * rng.uniform(-1, 1, (Q, N))))
    bad = 5
    clean = np.delete(f, bad, axis=1)
    ref = oracle_mod.stats(lat, (N - 1, 1, 1), clean.reshape(Q, 1, 1, N - 1))
    for poison in (np.nan, np.inf):
        g = f.copy()
        g[Q // 2, bad] = poison
        st = oracle_mod.stats(lat, dims, g.reshape(Q, dims[2], dims[1], dims[0]))
        assert st["nonfinite"] == 1 and st["sites"] == N
        # Sums leave the site out; means divide by all N sites (the record's convention).
        assert st["mass"] == pytest.approx(ref["mass"], rel=1e-14)
        np.testing.assert_allclose(st["mom"], ref["mom"], rtol=1e-13, atol=1e-16)
        scale = (N - 1) / N
        for key in ("u_mean", "uu", "k_mean", "k_cov"):
            np.testing.assert_allclose(st[key], ref[key] * scale, rtol=1e-12, atol=1e-18, err_msg=key)
