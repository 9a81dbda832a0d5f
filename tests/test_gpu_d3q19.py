"""GPU parity and statistics of the D3Q19 lattice (FLBM_D3Q19; Sec. II-C, "Lattice-agnostic
construction and the D3Q19 example") against the oracle's lattice 3.
Tolerance as everywhere: max |f_gpu - f_oracle| / (w_i rho0) <= 1e-5."""
import numpy as np
import pytest

from _gram_tol import uu_tol

pytestmark = pytest.mark.gpu

TOL = 1e-5
Q19 = 3
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12).reshape(-1, 1, 1, 1)


@pytest.fixture(scope="module")
def fl():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_16486_gb300 as fl

    return fl


def _paper_rates(omega):
    lam = np.ones(19)
    lam[7:10] = omega
    return lam


def _general_rates():
    rng = np.random.default_rng(31)
    lam = np.ones(19)
    lam[4:] = rng.uniform(0.4, 1.95, 15)
    return lam


def _run(fl, oracle_mod, dims, lam, kbt, seed, steps, variant, storage=0):
    with fl.Lattice(Q19, dims, lam, kbt, 1.0, seed, storage) as lat:
        lat.variant = variant
        lat.init_uniform((0.04, -0.02, 0.01), 1e-3, 5)
        f0 = lat.populations()
        lat.step(steps)
        assert lat.step_count == steps
        fg = lat.populations()
    fo = oracle_mod.run(Q19, dims, lam, kbt, seed, f0, 0, steps)
    return float((np.abs(fg - fo) / W).max())


def test_d3q19_init_matches_oracle_equilibrium(fl, oracle_mod):
    dims = (10, 6, 5)
    with fl.Lattice(Q19, dims, _paper_rates(1.5), 1e-4, 1.0, 1) as lat:
        lat.init_uniform((0.05, 0.02, -0.01), 1e-3, 7)
        fg = lat.populations()
    fo = oracle_mod.init_uniform(Q19, dims, 1.0, (0.05, 0.02, -0.01), 1e-3, 7)
    assert float((np.abs(fg - fo) / W).max()) <= 1e-6  # FP32 storage of FP64 deviations


@pytest.mark.parametrize("variant,dims", [(1, (33, 8, 6)), (1, (64, 9, 7)), (2, (64, 9, 7)), (3, (64, 9, 7)),
                                          (5, (64, 9, 7)), (7, (64, 9, 7)), (8, (40, 6, 5))])
def test_d3q19_paper_rates_match_oracle(fl, oracle_mod, variant, dims):
    assert _run(fl, oracle_mod, dims, _paper_rates(1.6), 3e-4, 41, 100, variant) <= TOL


@pytest.mark.parametrize("variant,dims", [(1, (33, 8, 6)), (2, (64, 9, 7)), (5, (64, 9, 7)), (7, (64, 9, 7))])
def test_d3q19_general_rates_match_oracle(fl, oracle_mod, variant, dims):
    assert _run(fl, oracle_mod, dims, _general_rates(), 1e-4, 42, 100, variant) <= TOL


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 1), (5, 1, 4)])
def test_d3q19_degenerate_boxes(fl, oracle_mod, dims):
    assert _run(fl, oracle_mod, dims, _general_rates(), 1e-4, 43, 20, 0) <= TOL


def test_d3q19_stats_match_oracle(fl, oracle_mod):
    dims = (20, 16, 12)
    with fl.Lattice(Q19, dims, _general_rates(), 1e-3, 1.0, 23) as lat:
        lat.init_uniform((0.05, 0.02, 0.0), 1e-3, 3)
        lat.step(13)
        st = lat.stats()
        f = lat.populations()
    ref = oracle_mod.stats(Q19, dims, f)
    assert st["q"] == 19
    assert st["mass"] == pytest.approx(ref["mass"], rel=1e-7)
    n = int(np.prod(dims))  # near-zero entries: the reduction's own error (tests/_gram_tol.py)
    assert np.all(np.abs(np.asarray(st["uu"]) - ref["uu"]) <= 1e-5 * np.abs(ref["uu"]) + uu_tol(ref["uu"], n))
    scale = np.sqrt(np.abs(np.diag(ref["k_cov"])))
    np.testing.assert_allclose(st["k_mean"][:19], ref["k_mean"], atol=1e-5 * scale.max() + 1e-9)
    np.testing.assert_allclose(st["k_cov"], ref["k_cov"], rtol=1e-4, atol=1e-5 * np.outer(scale, scale).max())


def test_d3q19_equipartition_and_mode_variances(fl, oracle_mod):
    kbt = 1e-4
    _, _, b = oracle_mod.tables(Q19)
    with fl.Lattice(Q19, (64, 64, 64), _paper_rates(1.7), kbt, 1.0, 4) as lat:
        lat.step(1000)
        uu, kk = [], []
        for _ in range(50):
            s = lat.stats()
            uu.append(np.array(s["uu"][:3]) - np.array(s["u_mean"][:3]) ** 2)
            kk.append(np.diag(s["k_cov"]))
            lat.step(100)
    ratio = np.mean(uu, axis=0) / (kbt * (1 + 9 * kbt))
    assert np.abs(ratio - 1.0).max() <= 1e-2, ratio
    modes = np.mean(kk, axis=0)[4:] / (3.0 * kbt * b[4:])
    assert np.abs(modes - 1.0).max() <= 2e-2, np.round(modes, 4)


def test_d3q19_checkpoint_roundtrip(fl):
    with fl.Lattice(Q19, (16, 6, 5), _paper_rates(1.3), 1e-4, 1.0, 9) as a:
        a.init_uniform((0.01, 0.0, 0.02), 1e-3, 1)
        a.step(5)
        blob = a.save()
        a.step(4)
        fa = a.populations()
    with fl.Lattice(Q19, (16, 6, 5), _paper_rates(1.3), 1e-4, 1.0, 9) as b:
        b.load(blob)
        b.step(4)
        assert np.array_equal(b.populations(), fa)


def test_d3q19_rejected_in_batches(fl):
    with pytest.raises(fl.FlbmError) as e:
        fl.Batch([dict(lattice=Q19, dims=(8, 8, 8), lam=np.ones(19), kBT=1e-4, rho0=1.0, seed=0)])
    assert e.value.status == fl.FLBM_EINVAL


@pytest.mark.parametrize("storage,bits", [(1, 8), (2, 11)])
@pytest.mark.parametrize("dims", [(20, 7, 6), (13, 6, 5)])
def test_d3q19_reduced_precision_one_step_bound(fl, oracle_mod, storage, bits, dims):
    # One update from the stored state: the only error beyond FP32 arithmetic is the
    # rounding of each stored deviation d* to the format (relative 2^-bits).
    lam = _paper_rates(1.6)
    with fl.Lattice(Q19, dims, lam, 1e-4, 1.0, 5, storage) as lat:
        lat.init_uniform((0.02, -0.01, 0.01), 1e-3, 2)
        lat.step(3)
        f0 = lat.populations()
        lat.step(1)
        fg = lat.populations()
    fo = oracle_mod.run(Q19, dims, lam, 1e-4, 5, f0, 3, 1)
    w = oracle_mod.tables(Q19)[1].reshape((19, 1, 1, 1))
    dev = np.abs(fo - w)
    # 3e-8 covers the absolute spacing of FP16 subnormals (2^-24) below 6.1e-5.
    assert np.all(np.abs(fg - fo) <= dev * 2.0 ** -bits * 1.01 + 2e-6 * np.abs(fo) + 3e-8), \
        float((np.abs(fg - fo) / (dev * 2.0 ** -bits + 1e-30)).max())
