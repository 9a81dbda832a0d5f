"""Statistical checks of the GPU path against what the paper fixes (Sec. III):

* equipartition <u_a^2> = kBT / rho0 per component (Eq. for <u^2>, Tests 2-5), corrected
  for the bias of the estimator u = j / rho: E[u_a^2] = (kBT/rho0)(1 + 9 kBT/rho0) to
  first order, from Var(rho) = rho0 kBT / cs^2 and j independent of rho at equilibrium;
* proportional to kBT (Test 3), to 1/rho0 (Test 4), independent of the relaxation time up
  to the over-relaxation limit (Test 6), isotropic on anisotropic boxes (Test 7);
* Gaussian velocity fluctuations (Test 8);
* every non-conserved central moment with variance rho0 kBT b_v / cs^2 (the diagonal
  equilibrium covariance, Sec. II-B), b_v from the oracle's basis norms (pinned to the
  paper's printed values in test_oracle_basis.py);
* equipartition in the co-moving frame under a uniform drift (Galilean invariance; the
  paper runs no drift, so this is the reading that the same statistics hold for u - <u>).

Pass criterion ("1 % at 3 sigma"): the time- and seed-averaged ratio lies within 1 % of 1
and its 3-sigma statistical error (spread of independent samples) is below 0.5 %.

The C2 ensemble (96 runs: D2Q9 512^2 and D3Q27 64^3, kBT 1e-5..1e-3, shear rate 1.0..1.98,
seeds 0..3, 10,000 steps of which the first 1000 are discarded) runs as one batch
(flbm_batch_*), sampled with flbm_sample every 100 steps.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def fl():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_16486_gb300 as fl

    return fl


def _lam(lattice, shear):
    q = 27 if lattice else 9
    lam = np.ones(q)
    lam[[7, 8, 9] if lattice else [4, 5]] = shear
    return lam


def _target(kbt, rho0=1.0):
    return kbt / rho0 * (1.0 + 9.0 * kbt / rho0)


def _run_batch(fl, specs, warm, total, every, u0=None, amp=0.0):
    b = fl.Batch(specs)
    for i in range(len(specs)):
        b.lattice(i).init_uniform(u0[i] if u0 else (0.0, 0.0, 0.0), amp, 50 + i)
    b.step(warm)
    n = warm
    while True:
        for i in range(len(specs)):
            b.lattice(i).sample()
        if n >= total:
            break
        b.step(every)
        n += every
    b.sync()
    out = [b.lattice(i).fetch_samples() for i in range(len(specs))]
    b.close()
    return out


def _velocity_ratio(samples, D, kbt, rho0=1.0):
    """Per sample and component: (<u_a^2> - <u_a>^2) / target."""
    uu = np.array([s["uu"][:D] for s in samples])
    um = np.array([s["u_mean"][:D] for s in samples])
    return (uu - um ** 2) / _target(kbt, rho0)


@pytest.fixture(scope="module")
def c2(fl):
    specs = []
    for lat, dims in ((0, (512, 512, 1)), (1, (64, 64, 64))):
        for kbt in (1e-5, 1e-4, 1e-3):
            for om in (1.0, 1.5, 1.9, 1.98):
                for seed in range(4):
                    specs.append(dict(lattice=lat, dims=dims, lam=_lam(lat, om), kBT=kbt, rho0=1.0,
                                      seed=seed, om=om))
    samples = _run_batch(fl, specs, warm=1000, total=10000, every=100)  # 10,000 steps
    return specs, samples


def _groups(specs):
    keys = sorted({(d["lattice"], d["kBT"], d["om"]) for d in specs})
    return {k: [i for i, d in enumerate(specs) if (d["lattice"], d["kBT"], d["om"]) == k] for k in keys}


def test_c2_equipartition_every_rate_and_temperature(c2):
    specs, samples = c2
    for (lat, kbt, om), idx in _groups(specs).items():
        D = 3 if lat else 2
        r = np.concatenate([_velocity_ratio(samples[i], D, kbt) for i in idx])  # samples x D
        per = r.mean(axis=1)
        mean = per.mean()
        sig3 = 3.0 * per.std(ddof=1) / np.sqrt(per.size)
        print(f"C2 {'D3Q27' if lat else 'D2Q9'} kBT={kbt:g} rate={om}: <u^2>/target = {mean:.5f} "
              f"(3 sigma {sig3:.1e})")
        assert sig3 <= 5e-3, (lat, kbt, om, sig3)
        assert abs(mean - 1.0) <= 1e-2, (lat, kbt, om, mean)
        # isotropy: every component within 1 % of the others
        comp = r.mean(axis=0)
        assert comp.max() / comp.min() - 1.0 <= 1e-2, (lat, kbt, om, comp)


def test_c2_independent_of_relaxation_rate(c2):
    # Test 6: <u^2> does not depend on tau, up to the over-relaxation limit (rate 1.98).
    specs, samples = c2
    g = _groups(specs)
    for lat in (0, 1):
        D = 3 if lat else 2
        for kbt in (1e-5, 1e-4, 1e-3):
            means = [np.concatenate([_velocity_ratio(samples[i], D, kbt) for i in g[(lat, kbt, om)]]).mean()
                     for om in (1.0, 1.5, 1.9, 1.98)]
            assert max(means) / min(means) - 1.0 <= 1e-2, (lat, kbt, means)


def test_c2_mode_variances(c2, oracle_mod):
    # <k_v^2> = rho0 kBT b_v / cs^2 for every non-conserved mode v (central moments about
    # the local velocity, rest-frame norms b_v).
    specs, samples = c2
    for (lat, kbt, om), idx in _groups(specs).items():
        if kbt > 1e-4:
            continue  # at 1e-3 the O(kBT) corrections of the estimator reach the percent level
        D = 3 if lat else 2
        _, _, b = oracle_mod.tables(lat)
        q = b.size
        kk = np.mean([[np.diag(s["k_cov"])[:q] for s in samples[i]] for i in idx], axis=(0, 1))
        ratio = kk[D + 1:] / (3.0 * kbt * b[D + 1:])
        print(f"C2 {'D3Q27' if lat else 'D2Q9'} kBT={kbt:g} rate={om}: mode variance / (rho0 kBT b_v/cs^2) "
              f"in [{ratio.min():.4f}, {ratio.max():.4f}]")
        assert np.abs(ratio - 1.0).max() <= 2e-2, (lat, kbt, om, np.round(ratio, 4))


def test_density_scaling(fl):
    # Test 4: <u^2> proportional to 1 / rho0.
    specs = [dict(lattice=0, dims=(256, 256, 1), lam=_lam(0, 1.5), kBT=1e-4, rho0=rho0, seed=s)
             for rho0 in (0.5, 2.0) for s in range(2)]
    samples = _run_batch(fl, specs, warm=1000, total=6000, every=100)
    for rho0 in (0.5, 2.0):
        idx = [i for i, d in enumerate(specs) if d["rho0"] == rho0]
        per = np.concatenate([_velocity_ratio(samples[i], 2, 1e-4, rho0) for i in idx]).mean(axis=1)
        assert abs(per.mean() - 1.0) <= 1e-2, (rho0, per.mean())
        assert 3.0 * per.std(ddof=1) / np.sqrt(per.size) <= 5e-3


def test_isotropy_on_anisotropic_boxes(fl):
    # Test 7: equal components on boxes with unequal sides.
    specs = [dict(lattice=0, dims=(512, 64, 1), lam=_lam(0, 1.7), kBT=1e-4, rho0=1.0, seed=s) for s in range(2)]
    specs += [dict(lattice=1, dims=(96, 48, 24), lam=_lam(1, 1.7), kBT=1e-4, rho0=1.0, seed=s) for s in range(2)]
    samples = _run_batch(fl, specs, warm=1000, total=6000, every=100)
    for lat in (0, 1):
        D = 3 if lat else 2
        r = np.concatenate([_velocity_ratio(samples[i], D, 1e-4) for i, d in enumerate(specs)
                            if d["lattice"] == lat])
        comp = r.mean(axis=0)
        assert np.abs(comp - 1.0).max() <= 1e-2, (lat, comp)
        assert comp.max() / comp.min() - 1.0 <= 1e-2, (lat, comp)


def test_galilean_drift_comoving_equipartition(fl):
    # The headline physics at 64^3: drift (0.05, 0.02, 0), 1e-3 density perturbation,
    # kBT 1e-4, shear rate 1.6. Fluctuations about the box mean velocity obey
    # equipartition; the drift itself is conserved.
    u0 = (0.05, 0.02, 0.0)
    specs = [dict(lattice=1, dims=(64, 64, 64), lam=_lam(1, 1.6), kBT=1e-4, rho0=1.0, seed=s) for s in range(4)]
    samples = _run_batch(fl, specs, warm=1000, total=6000, every=100, u0=[u0] * 4, amp=1e-3)
    r = np.concatenate([_velocity_ratio(s, 3, 1e-4) for s in samples])
    comp = r.mean(axis=0)
    assert np.abs(comp - 1.0).max() <= 1e-2, comp
    assert 3.0 * r.mean(axis=1).std(ddof=1) / np.sqrt(r.shape[0]) <= 5e-3
    for s in samples:
        for x in s:
            # mass and momentum conserved: the box mean of rho u stays rho0 u0 (perturbation
            # mean ~1e-3 / sqrt(N) of rho0)
            mom = np.array(x["mom"]) / x["sites"]
            assert np.abs(mom - np.array(u0)).max() <= 1e-5


def test_velocity_fluctuations_gaussian(fl, oracle_mod):
    # Test 8: the single-site velocity components are normal: skewness 0, kurtosis 3
    # (64^3 sites of one snapshot; the sampling errors are about 0.005 and 0.01).
    with fl.Lattice(1, (64, 64, 64), _lam(1, 1.5), 1e-4, 1.0, 3) as lat:
        lat.step(2000)
        f = lat.populations()
    cv, _, _ = oracle_mod.tables(1)  # velocities in the paper's order
    rho = f.sum(axis=0)
    for a in range(3):
        u = np.tensordot(cv[:, a].astype(float), f, axes=(0, 0)) / rho
        z = (u - u.mean()) / u.std()
        assert abs(np.mean(z ** 3)) <= 0.02
        assert abs(np.mean(z ** 4) - 3.0) <= 0.05


def _precision_stats(fl, storage, kbt, ref):
    dims = tuple(ref["dims"])
    with fl.Lattice(1, dims, _lam(1, ref["omega_shear"]), kbt, ref["rho0"], ref["seed"], storage) as lat:
        lat.step(ref["first"])
        uu, kk = [], []
        for k in range(ref["first"], ref["last"] + 1, ref["every"]):
            s = lat.stats()
            assert s["step"] == k
            uu.append(np.array(s["uu"][:3]) - np.array(s["u_mean"][:3]) ** 2)
            kk.append(np.diag(s["k_cov"]))
            if k < ref["last"]:
                lat.step(ref["every"])
    return np.mean(uu), np.mean(kk, axis=0)


@pytest.mark.parametrize("kbt", [1e-5, 1e-4])
def test_storage_precision_against_oracle_replica(fl, kbt, oracle_mod):
    # The 256^3 precision workload on its 32^3 replica: same seed, same steps as the FP64
    # oracle's stored statistics (tests/oracle_ref): the error of equipartition and of
    # every mode variance at each storage width.
    with open(os.path.join(HERE, "oracle_ref", "precision_d3q27_32cube.json")) as fh:
        ref = json.load(fh)
    ser = ref["series"][repr(kbt)]
    uu_ref = np.mean([np.array(x["uu"][:3]) - np.array(x["u_mean"][:3]) ** 2 for x in ser])
    kk_ref = np.mean([x["kk"] for x in ser], axis=0)
    noisy = np.arange(4, 27)
    # Bounds: FP32 storage rounds each value to 2^-24 of itself and follows the oracle's
    # trajectory (1e-5); 16-bit storage rounds each deviation to 2^-8 (BF16) or 2^-11
    # (FP16) of itself every step, an unbiased perturbation whose effect on second
    # moments is of order 2^-18 (1e-3 leaves a wide margin; measured about 1e-5).
    for storage, tol in ((0, 1e-5), (1, 1e-3), (2, 1e-3)):
        uu, kk = _precision_stats(fl, storage, kbt, ref)
        e_uu = uu / uu_ref - 1.0
        e_kk = np.abs(kk[noisy] / kk_ref[noisy] - 1.0).max()
        print(f"precision kBT={kbt:g} storage={storage}: equipartition error {e_uu:+.2e}, "
              f"max mode-variance error {e_kk:.2e}")
        assert abs(e_uu) <= tol, (storage, e_uu)
        assert e_kk <= tol, (storage, kk[noisy] / kk_ref[noisy])


def test_c1_statistics_follow_the_oracle(fl, oracle_mod):
    # Config 1: D2Q9 64x64 at rest, kBT 1e-4, every non-conserved mode at rate 1.25
    # (tau 0.8), seed 42, 1000 steps. The GPU (FP32) and the oracle (FP64) run the same
    # noise, so their sampled <u_a^2> and mode variances agree sample by sample.
    lam = np.full(9, 1.25)
    lam[:3] = 1.0
    dims = (64, 64, 1)
    every = 50
    with fl.Lattice(0, dims, lam, 1e-4, 1.0, 42) as lat:
        fo = lat.populations()
        worst_u, worst_k, ratios = 0.0, 0.0, []
        for k in range(0, 1001, every):
            if k >= 100:
                sg = lat.stats()
                so = oracle_mod.stats(0, dims, fo)
                du = np.abs(np.array(sg["uu"][:2]) - so["uu"][:2]) / so["uu"][:2]
                dk = np.abs(np.diag(sg["k_cov"])[3:9] - np.diag(so["k_cov"])[3:9]) / np.diag(so["k_cov"])[3:9]
                worst_u, worst_k = max(worst_u, du.max()), max(worst_k, dk.max())
                ratios.append(so["uu"][:2].mean() / _target(1e-4))
            if k < 1000:
                lat.step(every)
                fo = oracle_mod.run(0, dims, lam, 1e-4, 42, fo, k, every)
    print(f"C1: GPU vs oracle, worst relative difference <u^2> {worst_u:.1e}, mode variances {worst_k:.1e}; "
          f"oracle <u^2>/target averaged over steps 100-1000: {np.mean(ratios):.4f}")
    assert worst_u <= 1e-4 and worst_k <= 1e-4
    # 4096 sites x 19 samples: the 3-sigma sampling error of the average is about 3 %
    assert abs(np.mean(ratios) - 1.0) <= 0.05
