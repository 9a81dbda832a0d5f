"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs, element by element.

Tolerance (the stated 1e-5 on populations after 100 FP32 steps), measured against the
population scale: max_i,x |f_gpu - f_oracle| / (w_i rho0) <= 1e-5. The plain ratio
|f_gpu - f_oracle| / |f_oracle| is not used: at the paper's temperatures a population
fluctuates by sqrt(3 kBT / w_i) of its weight (25 % for a D3Q27 corner at kBT = 1e-4) and
single populations pass through zero, where that ratio is unbounded even between two
FP64 runs. Reduced-precision storage is checked one step at a time against the rounding
bound of its format.
"""
import numpy as np
import pytest

from _gram_tol import mean_tol, uu_tol

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def fl():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_16486_gb300 as fl

    return fl


def _lam(lattice, shear, rest=1.0):
    if lattice == 0:
        lam = np.full(9, rest)
        lam[:3] = 1.0
        lam[[4, 5]] = shear
    else:
        lam = np.full(27, rest)
        lam[:4] = 1.0
        lam[[7, 8, 9]] = shear
    return lam


def _err(a, b, lattice, rho0=1.0):
    """max |a - b| / (w_i rho0) over populations i and sites."""
    q = 9 if lattice == 0 else 27
    if lattice == 0:
        w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    else:
        w = np.array([8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8)
    w = w.reshape((q,) + (1,) * (a.ndim - 1)) if a.shape[0] == q else w
    return float((np.abs(a - b) / (w * rho0)).max())


def _run_pair(fl, oracle_mod, lattice, dims, lam, kBT, seed, steps, u0=(0, 0, 0), amp=0.0,
              pseed=0, rho0=1.0, storage=0, variant=0):
    with fl.Lattice(lattice, dims, lam, kBT, rho0, seed, storage) as lat:
        if variant:
            lat.variant = variant
        lat.init_uniform(u0, amp, pseed)
        f0 = lat.populations()
        lat.step(steps)
        assert lat.step_count == steps
        fg = lat.populations()
    fo = oracle_mod.run(lattice, dims, lam, kBT, seed, f0, 0, steps)
    return f0, fg, fo


def test_d2q9_64x64_fp64_config_parity(fl, oracle_mod):
    # D2Q9 64x64, rho0 = 1 at rest, kBT = 1e-4, every non-conserved mode at omega = 1.25
    # (tau = 0.8), Philox seed 42: the first 100 steps.
    lam = _lam(0, 1.25, 1.25)
    f0, fg, fo = _run_pair(fl, oracle_mod, 0, (64, 64, 1), lam, 1e-4, 42, 100)
    assert np.abs(fg - f0).max() > 1e-4  # the noise moved the state
    assert _err(fg, fo, 0) <= TOL


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6, 7, 8])
def test_d3q27_drift_perturbed_ragged_box(fl, oracle_mod, variant):
    # The headline workload's physics (drift (0.05, 0.02, 0), 1e-3 density perturbation,
    # kBT = 1e-4, shear omega = 1.6) on a box spanning three x-blocks (one site per thread)
    # or two (two sites per thread) with a ragged tail, for every step-kernel variant.
    lam = _lam(1, 1.6)
    f0, fg, fo = _run_pair(fl, oracle_mod, 1, (300, 7, 5), lam, 1e-4, 0, 100, (0.05, 0.02, 0.0),
                           1e-3, 0, variant=variant)
    assert _err(fg, fo, 1) <= TOL


@pytest.mark.parametrize("variant,storage,dims", [(7, 0, (40, 9, 6)), (8, 0, (40, 9, 6)), (7, 0, (70, 5, 3)),
                                                   (7, 1, (40, 9, 6)), (8, 2, (24, 13, 4))])
def test_d3q27_row_blocks_narrow_box(fl, oracle_mod, variant, storage, dims):
    # Blocks of four rows (variants 7, 8) on boxes whose rows are shorter than a one-row
    # block, with a ragged last row group (ny not a multiple of 4) and a row longer than
    # one warp's 64 sites; FP32 to the population tolerance, 16-bit storage one step against
    # the rounding bound of its width.
    lam = _lam(1, 1.6)
    if storage == 0:
        f0, fg, fo = _run_pair(fl, oracle_mod, 1, dims, lam, 2e-4, 11, 60, (0.05, 0.02, -0.01), 1e-3, 3,
                               variant=variant)
        assert _err(fg, fo, 1) <= TOL
        return
    bits = 8 if storage == 1 else 11
    c, w, _ = oracle_mod.tables(1)
    with fl.Lattice(1, dims, lam, 2e-4, 1.0, 11, storage) as lat:
        lat.variant = variant
        assert lat.variant == variant
        lat.init_uniform((0.05, 0.02, -0.01), 1e-3, 3)
        lat.step(3)
        f0 = lat.populations()
        lat.step(1)
        got = lat.populations()
    ref = oracle_mod.run(1, dims, lam, 2e-4, 11, f0, 3, 1)
    wq = w.reshape(-1, 1, 1, 1)
    bound = np.abs(ref - wq) * 2.0 ** -bits * 1.01 + 2e-6 * np.abs(ref) + 3e-8
    assert float((np.abs(got - ref) / bound).max()) <= 1.0


def test_d3q27_general_rates(fl, oracle_mod):
    rng = np.random.default_rng(5)
    lam = np.ones(27)
    lam[4:] = rng.uniform(0.3, 1.95, 23)
    f0, fg, fo = _run_pair(fl, oracle_mod, 1, (19, 11, 13), lam, 3e-4, 123456789012345, 100,
                           (0.02, -0.03, 0.01), 1e-3, 5)
    assert _err(fg, fo, 1) <= TOL


@pytest.mark.parametrize("variant", [1, 3, 4, 5, 6, 7])
def test_d2q9_paper_rates(fl, oracle_mod, variant):
    # D2Q9 with the paper's rates (L_4 = L_5 = omega, every other mode 1): the
    # specialised path that forms only the shear central moments.
    lam = _lam(0, 1.7)
    f0, fg, fo = _run_pair(fl, oracle_mod, 0, (128, 21, 1), lam, 3e-4, 5, 100, (0.03, -0.02), 1e-3, 4,
                           variant=variant)
    assert _err(fg, fo, 0) <= TOL


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6, 7, 8])
def test_d2q9_general_rates_ragged(fl, oracle_mod, variant):
    rng = np.random.default_rng(6)
    lam = np.ones(9)
    lam[3:] = rng.uniform(0.3, 1.95, 6)
    f0, fg, fo = _run_pair(fl, oracle_mod, 0, (200, 37, 1), lam, 5e-4, 9, 100, (-0.04, 0.03), 1e-3, 2,
                           variant=variant)
    assert _err(fg, fo, 0) <= TOL


@pytest.mark.parametrize("lattice,dims", [(1, (1, 1, 1)), (1, (2, 3, 1)), (1, (5, 1, 4)), (1, (1, 6, 2)),
                                          (0, (1, 7, 1)), (0, (3, 1, 1)), (0, (2, 2, 1))])
def test_degenerate_boxes(fl, oracle_mod, lattice, dims):
    lam = _lam(lattice, 1.7, 1.1)
    f0, fg, fo = _run_pair(fl, oracle_mod, lattice, dims, lam, 1e-3, 77, 25, (0.01, -0.02, 0.03), 1e-3, 1)
    assert _err(fg, fo, lattice) <= TOL


@pytest.mark.parametrize("lattice,dims", [(0, (16, 12, 1)), (1, (8, 6, 5))])
def test_zero_noise_from_rest_is_exactly_at_rest(fl, lattice, dims):
    # Test 1: kBT = 0 from rest; the stored deviations stay exactly zero.
    with fl.Lattice(lattice, dims, _lam(lattice, 1.6), 0.0, 1.0, 42) as lat:
        lat.step(31)
        st = lat.stats()
        f = lat.populations()
    assert np.all(st["uu"] == 0.0) and np.all(st["u_mean"] == 0.0)
    assert st["mass"] == pytest.approx(np.prod(dims), rel=1e-12)
    with fl.Lattice(lattice, dims, _lam(lattice, 1.6), 0.0, 1.0, 42) as lat:
        f_rest = lat.populations()
    assert np.array_equal(f, f_rest)


@pytest.mark.parametrize("lattice,dims", [(0, (10, 6, 1)), (1, (6, 5, 4))])
def test_set_get_roundtrip_both_parities(fl, lattice, dims):
    rng = np.random.default_rng(8)
    q = 9 if lattice == 0 else 27
    with fl.Lattice(lattice, dims, _lam(lattice, 1.3), 1e-4, 1.0, 3) as lat:
        for steps in (0, 1):
            lat.step(steps)
            f = lat.populations()
            g = f * (1 + 1e-3 * rng.standard_normal(f.shape))
            lat.set_populations(g)
            back = lat.populations()
            # FP32 storage of the deviation g - w rho0
            assert np.abs(back - g).max() <= 1e-7 * np.abs(g).max()
            sites = rng.integers(0, np.prod(dims), 17)
            sp = lat.sites_populations(sites)
            flat = back.reshape(q, -1)
            assert np.array_equal(sp, flat[:, sites].T)


def test_autotune_leaves_the_state_unchanged(fl):
    lam = _lam(1, 1.6)
    with fl.Lattice(1, (64, 20, 18), lam, 1e-4, 1.0, 3) as lat:
        lat.init_uniform((0.05, 0.02, 0.0), 1e-3, 0)
        lat.step(3)
        before = lat.populations()
        chosen = lat.autotune(4)
        assert chosen in (1, 2, 3, 4, 5, 6, 7, 8) and lat.variant == chosen
        assert lat.step_count == 3
        assert np.array_equal(lat.populations(), before)
        lat.variant = 1
        lat.step(5)
        a = lat.populations()
    with fl.Lattice(1, (64, 20, 18), lam, 1e-4, 1.0, 3) as lat:
        lat.init_uniform((0.05, 0.02, 0.0), 1e-3, 0)
        lat.variant = 1
        lat.step(8)
        assert np.array_equal(lat.populations(), a)


def test_autotune_cache_file(tmp_path):
    # FLBM_AUTOTUNE_CACHE: the first process tunes and appends its choice; a second process
    # reads it and returns the same variant without trials (the state is not touched).
    import os
    import subprocess
    import sys

    cache = tmp_path / "tune.txt"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys, numpy as np; sys.path.insert(0, %r)\n"
        "import paper_2602_16486_gb300 as fl\n"
        "lam = np.ones(27); lam[[7, 8, 9]] = 1.6\n"
        "with fl.Lattice(1, (64, 32, 16), lam, 1e-4, 1.0, 3) as lat:\n"
        "    lat.init_uniform((0.02, 0.0, 0.0), 1e-3, 1)\n"
        "    f0 = lat.populations()\n"
        "    v = lat.autotune(4)\n"
        "    assert np.array_equal(lat.populations(), f0) and lat.step_count == 0\n"
        "    print('VARIANT', v)\n" % root)
    env = dict(os.environ, FLBM_AUTOTUNE_CACHE=str(cache))
    first = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True)
    assert first.returncode == 0, first.stderr
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and "\t" in lines[0]
    v1 = int(first.stdout.split("VARIANT")[1])
    assert int(lines[0].split("\t")[1]) == v1
    second = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True)
    assert second.returncode == 0, second.stderr
    assert int(second.stdout.split("VARIANT")[1]) == v1
    assert len(cache.read_text().splitlines()) == 1  # read from the file, not tuned again


def test_checkpoint_resume_is_bitwise(fl):
    lam = _lam(1, 1.5)
    with fl.Lattice(1, (12, 10, 9), lam, 1e-4, 1.0, 11) as a:
        a.init_uniform((0.02, 0.0, -0.01), 1e-3, 4)
        a.step(7)
        blob = a.save()
        a.step(8)
        fa = a.populations()
    with fl.Lattice(1, (12, 10, 9), _lam(1, 1.9), 5e-3, 2.0, 999) as b:
        b.load(blob)
        assert b.step_count == 7
        b.step(8)
        fb = b.populations()
    assert np.array_equal(fa, fb)


def test_stats_match_oracle_on_same_state(fl, oracle_mod):
    for lattice, dims, u0 in ((0, (64, 48, 1), (0.03, -0.01)), (1, (20, 16, 12), (0.05, 0.02, 0.0))):
        lam = _lam(lattice, 1.6)
        with fl.Lattice(lattice, dims, lam, 1e-3, 1.0, 21) as lat:
            lat.init_uniform(u0, 1e-3, 3)
            lat.step(13)
            st = lat.stats()
            f = lat.populations()
        ref = oracle_mod.stats(lattice, dims, f)
        n = np.prod(dims)
        assert st["sites"] == n and st["nonfinite"] == 0
        assert st["mass"] == pytest.approx(ref["mass"], rel=1e-7)
        np.testing.assert_allclose(st["mom"], ref["mom"], rtol=1e-5, atol=1e-6 * n)
        # near-zero means: the reduction's own error (tests/_gram_tol.py) sets the floor
        assert np.all(np.abs(np.asarray(st["u_mean"]) - ref["u_mean"])
                      <= 1e-5 * np.abs(ref["u_mean"]) + 1e-9 + mean_tol(ref["uu"][:3], n))
        assert np.all(np.abs(np.asarray(st["uu"]) - ref["uu"]) <= 1e-5 * np.abs(ref["uu"]) + uu_tol(ref["uu"], n))
        scale = np.sqrt(np.abs(np.diag(ref["k_cov"])))
        np.testing.assert_allclose(st["k_mean"], ref["k_mean"], atol=1e-5 * scale.max() + 1e-9)
        np.testing.assert_allclose(st["k_cov"], ref["k_cov"], rtol=1e-4,
                                   atol=1e-5 * np.outer(scale, scale).max())


@pytest.mark.parametrize("steps", [12, 13])
@pytest.mark.parametrize("lattice,dims", [(0, (512, 6, 1)), (1, (256, 6, 5)), (1, (512, 2, 3))])
def test_stats_row_tiles_match_oracle(fl, oracle_mod, lattice, dims, steps):
    # nx a multiple of the reduction's 256-site tile: every tile lies inside one row and the
    # kernel takes y, z and the periodic offsets from the tile (both parities).
    lam = _lam(lattice, 1.6)
    u0 = (0.04, -0.02, 0.01)
    with fl.Lattice(lattice, dims, lam, 1e-3, 1.0, 5) as lat:
        lat.init_uniform(u0, 1e-3, 9)
        lat.step(steps)
        st = lat.stats()
        f = lat.populations()
    ref = oracle_mod.stats(lattice, dims, f)
    n = np.prod(dims)
    assert st["sites"] == n and st["nonfinite"] == 0
    assert st["mass"] == pytest.approx(ref["mass"], rel=1e-7)
    assert np.all(np.abs(np.asarray(st["u_mean"]) - ref["u_mean"])
                  <= 1e-5 * np.abs(ref["u_mean"]) + 1e-9 + mean_tol(ref["uu"][:3], n))
    assert np.all(np.abs(np.asarray(st["uu"]) - ref["uu"]) <= 1e-5 * np.abs(ref["uu"]) + uu_tol(ref["uu"], n))
    scale = np.sqrt(np.abs(np.diag(ref["k_cov"])))
    np.testing.assert_allclose(st["k_mean"], ref["k_mean"], atol=1e-5 * scale.max() + 1e-9)
    np.testing.assert_allclose(st["k_cov"], ref["k_cov"], rtol=1e-4, atol=1e-5 * np.outer(scale, scale).max())


def test_sample_ring_matches_stats(fl):
    lam = _lam(0, 1.25, 1.25)
    with fl.Lattice(0, (40, 30, 1), lam, 1e-4, 1.0, 1) as lat:
        direct = []
        for _ in range(5):
            lat.step(3)
            lat.sample()
            direct.append(lat.stats())
        got = lat.fetch_samples()
    assert [g["step"] for g in got] == [3, 6, 9, 12, 15]
    for g, d in zip(got, direct):
        # Same kernel on the same state; block sums meet in FP64 atomics whose order varies.
        for key in ("mass", "uu", "k_cov"):
            np.testing.assert_allclose(g[key], d[key], rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("storage,bits", [(1, 8), (2, 11)])
def test_reduced_precision_one_step_bound(fl, oracle_mod, storage, bits):
    # (nx = 70 and 20 with 16-bit storage: rows of 140 / 40 bytes, so the pipelined
    # variant does not apply and the two-site kernel runs; the pipelined 16-bit path is
    # covered by test_reduced_precision_pipelined.)
    # One step from the stored state: the only error beyond FP32 arithmetic is the
    # rounding of each stored deviation d* to the format (relative 2^-bits).
    for lattice, dims in ((0, (70, 9, 1)), (1, (20, 7, 6))):
        lam = _lam(lattice, 1.6)
        with fl.Lattice(lattice, dims, lam, 1e-4, 1.0, 5, storage) as lat:
            lat.init_uniform((0.0, 0.0, 0.0), 1e-3, 2)
            lat.step(3)
            f0 = lat.populations()
            lat.step(1)
            fg = lat.populations()
        fo = oracle_mod.run(lattice, dims, lam, 1e-4, 5, f0, 3, 1)
        q = 9 if lattice == 0 else 27
        w = oracle_mod.tables(lattice)[1].reshape((q,) + (1,) * 3)
        dev = np.abs(fo - w)
        # 3e-8 covers the absolute spacing of FP16 subnormals (2^-24) below 6.1e-5.
        assert np.all(np.abs(fg - fo) <= dev * 2.0 ** -bits * 1.01 + 2e-6 * np.abs(fo) + 3e-8), \
            float((np.abs(fg - fo) / (dev * 2.0 ** -bits + 1e-30)).max())


@pytest.mark.parametrize("variant,storage,bits", [(5, 0, None), (2, 0, None), (5, 1, 8), (5, 2, 11)])
@pytest.mark.parametrize("pre_steps", [3, 4])
def test_full_size_headline_sampled_sites(fl, oracle_mod, variant, storage, bits, pre_steps):
    # D3Q27 256^3 in the benchmark's launch configuration (variant 5, the one the autotuner
    # picks, and variant 2), FP32 and 16-bit storage, an odd and an even update: the oracle
    # recomputes the collision of 48 sampled sites (the periodic seams among them) from the
    # GPU's pre-step populations and compares it with what the GPU streamed into the
    # neighbours. FP32: the 1e-5 population tolerance; 16-bit: each stored deviation is
    # rounded to 2^-bits of itself (as in test_reduced_precision_one_step_bound).
    dims = (256, 256, 256)
    lam = _lam(1, 1.6)
    c, w, _ = oracle_mod.tables(1)
    rng = np.random.default_rng(9)
    nx, ny, nz = dims
    xs = rng.integers(0, nx, 48)
    ys = rng.integers(0, ny, 48)
    zs = rng.integers(0, nz, 48)
    xs[:4] = [0, nx - 1, 0, nx - 1]  # include the periodic seams
    ys[:4] = [0, ny - 1, ny - 1, 0]
    zs[:4] = [nz - 1, 0, 0, nz - 1]
    sites = xs + nx * (ys + ny * zs)
    with fl.Lattice(1, dims, lam, 1e-4, 1.0, 0, storage) as lat:
        lat.variant = variant
        assert lat.variant == variant
        lat.init_uniform((0.05, 0.02, 0.0), 1e-3, 0)
        lat.step(pre_steps)  # the next update has the parity of pre_steps
        pre = lat.sites_populations(sites)
        lat.step(1)
        worst = 0.0
        for k, s in enumerate(sites):
            x, y, z = xs[k], ys[k], zs[k]
            eta = oracle_mod.site_eta(1, 0, pre_steps, int(s))
            fstar, _ = oracle_mod.collide_site(1, pre[k], lam, 1e-4, eta)
            dest = ((x + c[:, 0]) % nx) + nx * (((y + c[:, 1]) % ny) + ny * ((z + c[:, 2]) % nz))
            post = lat.sites_populations(dest)
            got = post[np.arange(27), np.arange(27)]
            if bits is None:
                worst = max(worst, float((np.abs(got - fstar) / w).max()))
            else:
                bound = np.abs(fstar - w) * 2.0 ** -bits * 1.01 + 2e-6 * np.abs(fstar) + 3e-8
                worst = max(worst, float((np.abs(got - fstar) / bound).max()))
    assert worst <= (TOL if bits is None else 1.0), worst


@pytest.mark.parametrize("storage", [1, 2])
def test_reduced_precision_pipelined_matches_pair_kernel(fl, storage):
    # The pipelined kernels and the two-site kernels perform identical arithmetic (rolled
    # or not); with 16-bit storage their stored results must agree bit for bit.
    lam = _lam(1, 1.6)
    out = []
    for variant in (2, 3, 4, 5, 6):
        with fl.Lattice(1, (64, 9, 7), lam, 1e-4, 1.0, 5, storage) as lat:
            lat.variant = variant
            assert lat.variant == variant
            lat.init_uniform((0.05, 0.02, 0.0), 1e-3, 2)
            lat.step(9)
            out.append(lat.populations())
    for o in out[1:]:
        assert np.array_equal(out[0], o)


@pytest.mark.parametrize("lattice,dims", [(0, (16, 12, 1)), (1, (8, 6, 5)), (1, (40, 3, 2))])
def test_pipelined_small_rows_fewer_threads_than_populations(fl, oracle_mod, lattice, dims):
    # Rows of 8 or 4 sites give blocks of 4 or 8 threads, fewer than Q bulk copies per tile.
    lam = _lam(lattice, 1.6, 1.2)
    f0, fg, fo = _run_pair(fl, oracle_mod, lattice, dims, lam, 1e-4, 12, 20, (0.02, 0.01, -0.01), 1e-3, 3,
                           variant=4)
    assert _err(fg, fo, lattice) <= TOL


@pytest.mark.parametrize("pre_steps", [3, 4])
@pytest.mark.parametrize("lattice", [2, 3])
def test_full_size_other_lattices_sampled_sites(fl, oracle_mod, lattice, pre_steps):
    # The benchmark's other lattices at 256^3 with its physics (drift, perturbation, kBT,
    # shear rate 1.6; the isotropic variant's deviators at the shear rate too) in the
    # launch configuration the autotuner picks there (variant 5): the oracle recomputes the
    # collision of 32 sampled sites (the periodic seams among them) from the GPU's pre-step
    # populations and compares it with what the GPU streamed into the neighbours.
    dims = (256, 256, 256)
    q = 27 if lattice == 2 else 19
    lam = np.ones(q)
    lam[[5, 6, 7, 8, 9] if lattice == 2 else [7, 8, 9]] = 1.6
    c, w, _ = oracle_mod.tables(lattice)
    rng = np.random.default_rng(10 + lattice)
    nx, ny, nz = dims
    xs, ys, zs = rng.integers(0, nx, 32), rng.integers(0, ny, 32), rng.integers(0, nz, 32)
    xs[:4] = [0, nx - 1, 0, nx - 1]
    ys[:4] = [0, ny - 1, ny - 1, 0]
    zs[:4] = [nz - 1, 0, 0, nz - 1]
    sites = xs + nx * (ys + ny * zs)
    with fl.Lattice(lattice, dims, lam, 1e-4, 1.0, 0) as lat:
        lat.variant = 5
        assert lat.variant == 5
        lat.init_uniform((0.05, 0.02, 0.0), 1e-3, 0)
        lat.step(pre_steps)
        pre = lat.sites_populations(sites)
        lat.step(1)
        worst = 0.0
        for k, s in enumerate(sites):
            x, y, z = xs[k], ys[k], zs[k]
            eta = oracle_mod.site_eta(lattice, 0, pre_steps, int(s))
            fstar, _ = oracle_mod.collide_site(lattice, pre[k], lam, 1e-4, eta)
            dest = ((x + c[:, 0]) % nx) + nx * (((y + c[:, 1]) % ny) + ny * ((z + c[:, 2]) % nz))
            got = lat.sites_populations(dest)[np.arange(q), np.arange(q)]
            worst = max(worst, float((np.abs(got - fstar) / w).max()))
    assert worst <= TOL, worst
