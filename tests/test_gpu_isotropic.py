"""GPU parity and statistics of the isotropic D3Q27 variant (FLBM_D3Q27_ISO: modes 4-6
are the trace and two deviators of the normal stresses) against the oracle's lattice 2.
Tolerance as everywhere: max |f_gpu - f_oracle| / (w_i rho0) <= 1e-5."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-5
ISO = 2


@pytest.fixture(scope="module")
def fl():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_16486_gb300 as fl

    return fl


def _w():
    return np.array([8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8).reshape(-1, 1, 1, 1)


def _run(fl, oracle_mod, dims, lam, kbt, seed, steps, variant, storage=0):
    with fl.Lattice(ISO, dims, lam, kbt, 1.0, seed, storage) as lat:
        lat.variant = variant
        lat.init_uniform((0.04, -0.02, 0.01), 1e-3, 5)
        f0 = lat.populations()
        lat.step(steps)
        fg = lat.populations()
    fo = oracle_mod.run(ISO, dims, lam, kbt, seed, f0, 0, steps)
    return float((np.abs(fg - fo) / _w()).max())


def _general_rates():
    rng = np.random.default_rng(11)
    lam = np.ones(27)
    lam[4] = 1.2                # bulk (trace)
    lam[5:10] = 1.6             # deviators and shear: one viscosity
    lam[10:] = rng.uniform(0.5, 1.9, 17)
    return lam


@pytest.mark.parametrize("variant", [1, 2, 3, 5, 7, 8])
def test_iso_general_rates_match_oracle(fl, oracle_mod, variant):
    assert _run(fl, oracle_mod, (64, 9, 7), _general_rates(), 1e-4, 21, 100, variant) <= TOL


@pytest.mark.parametrize("variant,dims", [(1, (33, 8, 6)), (2, (64, 9, 7)), (5, (64, 9, 7))])
def test_iso_paper_structure_path_matches_oracle(fl, oracle_mod, variant, dims):
    # Rate 1 above mode 9: the specialised path forms the six second-order central
    # moments from raw moments and rotates 4-6.
    lam = np.ones(27)
    lam[5:10] = 1.7
    assert _run(fl, oracle_mod, dims, lam, 3e-4, 22, 100, variant) <= TOL


def test_iso_stats_match_oracle(fl, oracle_mod):
    with fl.Lattice(ISO, (20, 16, 12), _general_rates(), 1e-3, 1.0, 23) as lat:
        lat.init_uniform((0.05, 0.02, 0.0), 1e-3, 3)
        lat.step(13)
        st = lat.stats()
        f = lat.populations()
    ref = oracle_mod.stats(ISO, (20, 16, 12), f)
    scale = np.sqrt(np.abs(np.diag(ref["k_cov"])))
    np.testing.assert_allclose(st["k_mean"], ref["k_mean"], atol=1e-5 * scale.max() + 1e-9)
    np.testing.assert_allclose(st["k_cov"], ref["k_cov"], rtol=1e-4, atol=1e-5 * np.outer(scale, scale).max())


def test_iso_equipartition_and_mode_variances(fl, oracle_mod):
    # The variant keeps the fluctuation-dissipation balance of every mode: <u^2> =
    # kBT/rho0 (bias-corrected as in test_gpu_statistics) and <k_v^2> = rho0 kBT b_v/cs^2
    # with the rotated norms b_4..6 = 2/3, 4/9, 4/3.
    kbt = 1e-4
    _, _, b = oracle_mod.tables(ISO)
    with fl.Lattice(ISO, (64, 64, 64), _general_rates(), kbt, 1.0, 4) as lat:
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


def test_iso_rejected_in_batches(fl):
    lam = np.ones(27)
    with pytest.raises(fl.FlbmError) as e:
        fl.Batch([dict(lattice=ISO, dims=(8, 8, 8), lam=lam, kBT=1e-4, rho0=1.0, seed=0)])
    assert e.value.status == fl.FLBM_EINVAL


@pytest.mark.parametrize("storage,bits", [(1, 8), (2, 11)])
@pytest.mark.parametrize("dims", [(20, 7, 6), (13, 6, 5)])
def test_iso_reduced_precision_one_step_bound(fl, oracle_mod, storage, bits, dims):
    # One update from the stored state: the only error beyond FP32 arithmetic is the
    # rounding of each stored deviation d* to the format (relative 2^-bits).
    lam = np.ones(27)
    lam[5:10] = 1.6
    with fl.Lattice(ISO, dims, lam, 1e-4, 1.0, 5, storage) as lat:
        lat.init_uniform((0.02, -0.01, 0.01), 1e-3, 2)
        lat.step(3)
        f0 = lat.populations()
        lat.step(1)
        fg = lat.populations()
    fo = oracle_mod.run(ISO, dims, lam, 1e-4, 5, f0, 3, 1)
    dev = np.abs(fo - _w())
    # 3e-8 covers the absolute spacing of FP16 subnormals (2^-24) below 6.1e-5.
    assert np.all(np.abs(fg - fo) <= dev * 2.0 ** -bits * 1.01 + 2e-6 * np.abs(fo) + 3e-8), \
        float((np.abs(fg - fo) / (dev * 2.0 ** -bits + 1e-30)).max())
