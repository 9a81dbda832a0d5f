"""GPU parity of batched ensembles (flbm_batch_*): every lattice of a batch against the
FP64 oracle run alone with the same parameters, and against a single context.

Tolerance as for single lattices: max |f_gpu - f_oracle| / (w_i rho0) <= 1e-5.
"""
import numpy as np
import pytest

from _gram_tol import sum_tol, uu_tol

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def fl():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_16486_gb300 as fl

    return fl


def _w(lattice):
    if lattice == 0:
        return np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    return np.array([8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8)


def _err(a, b, lattice, rho0=1.0):
    w = _w(lattice).reshape((-1, 1, 1, 1))
    return float((np.abs(a - b) / (w * rho0)).max())


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


def _general(lattice, seed):
    rng = np.random.default_rng(seed)
    q, d = (9, 2) if lattice == 0 else (27, 3)
    lam = np.ones(q)
    lam[d + 1:] = rng.uniform(0.3, 1.95, q - d - 1)
    return lam


def _specs(general=False):
    # Even and odd nx for both lattices (paired and unpaired sites), a degenerate box,
    # kBT over two decades, rho0 != 1, own seeds (one above 2^32).
    s = [
        dict(lattice=1, dims=(12, 10, 6), lam=_lam(1, 1.6), kBT=1e-4, rho0=1.0, seed=11),
        dict(lattice=1, dims=(9, 7, 5), lam=_lam(1, 1.9), kBT=3e-4, rho0=1.0, seed=12),
        dict(lattice=0, dims=(34, 20, 1), lam=_lam(0, 1.3), kBT=1e-3, rho0=1.0, seed=13),
        dict(lattice=0, dims=(33, 17, 1), lam=_lam(0, 0.7), kBT=1e-5, rho0=1.3, seed=14),
        dict(lattice=1, dims=(2, 3, 1), lam=_lam(1, 1.2), kBT=2e-4, rho0=1.0, seed=(1 << 40) + 15),
        dict(lattice=0, dims=(600, 3, 1), lam=_lam(0, 1.98), kBT=1e-4, rho0=1.0, seed=16),
        # rows of one and three sites: every pair slot of a row is the lone last one, or
        # one pair and one lone site
        dict(lattice=1, dims=(1, 5, 3), lam=_lam(1, 1.4), kBT=1e-4, rho0=1.0, seed=17),
        dict(lattice=0, dims=(3, 7, 1), lam=_lam(0, 1.1), kBT=2e-4, rho0=1.0, seed=18),
    ]
    if general:
        s[0]["lam"] = _general(1, 21)
        s[3]["lam"] = _general(0, 22)
    return s


_U0 = [(0.05, 0.02, 0.0), (-0.03, 0.01, 0.02), (0.04, -0.02, 0.0), (0.0, 0.03, 0.0),
       (0.01, 0.01, 0.01), (-0.05, 0.0, 0.0), (0.02, -0.01, 0.03), (-0.02, 0.04, 0.0)]


def _init(batch):
    f0 = []
    for i in range(len(batch)):
        lat = batch.lattice(i)
        lat.init_uniform(_U0[i], 1e-3, 100 + i)
        f0.append(lat.populations())
    return f0


@pytest.mark.parametrize("form", [0, 1, 2, 3])
@pytest.mark.parametrize("general", [False, True])
def test_batch_members_match_oracle(fl, oracle_mod, general, form):
    specs = _specs(general)
    with fl.Batch(specs) as b:
        b.shape = (128, form)
        f0 = _init(b)
        b.step(3)
        b.step(4)  # a second captured shape, then a replay below
        b.step(3)
        b.sync()
        assert b.step_count == 10
        for i, d in enumerate(specs):
            lat = b.lattice(i)
            assert lat.step_count == 10
            fg = lat.populations()
            fo = oracle_mod.run(d["lattice"], d["dims"], d["lam"], d["kBT"], d["seed"], f0[i], 0, 10)
            assert np.abs(fg - f0[i]).max() > 0.0
            assert _err(fg, fo, d["lattice"], d["rho0"]) <= TOL, i


@pytest.mark.parametrize("general", [False, True])
def test_batch_equals_single_contexts(fl, general):
    # Each lattice of the batch against a single context with the same parameters and
    # the same initial state. With general rates the arithmetic is the same code on the
    # same constants (bitwise); the paper-structure form builds its amplitudes from
    # sqrt(kBT) on the device, which may move the last bit.
    specs = _specs(general)
    with fl.Batch(specs) as b:
        f0 = _init(b)
        b.step(25)
        fb = [b.lattice(i).populations() for i in range(len(specs))]
    for i, d in enumerate(specs):
        with fl.Lattice(d["lattice"], d["dims"], d["lam"], d["kBT"], d["rho0"], d["seed"]) as lat:
            lat.variant = 3
            lat.set_populations(f0[i])
            lat.step(25)
            fs = lat.populations()
        general_member = general and i in (0, 3)
        if general_member and d["dims"][0] % 2 == 0:
            assert np.array_equal(fb[i], fs), i
        else:
            assert _err(fb[i], fs, d["lattice"], d["rho0"]) <= 1e-6, i


@pytest.mark.parametrize("form", [0, 1, 2, 3])
@pytest.mark.parametrize("threads", [64, 128, 256])
def test_batch_shapes_same_result(fl, threads, form):
    # Every launch shape computes the same update, bit for bit; calls of several sizes
    # start on both parities.
    if form == 2 and threads > 128:
        pytest.skip("form 2 takes at most 128 threads per block")
    specs = _specs(False)
    with fl.Batch(specs) as b:
        _init(b)
        b.shape = (threads, form)
        assert b.shape == (threads, form)
        b.step(2)
        b.step(3)
        b.step(1)
        b.step(3)
        b.sync()
        assert b.step_count == 9
        got = [b.lattice(i).populations() for i in range(len(specs))]
    with fl.Batch(specs) as b:
        _init(b)
        b.step(9)
        ref = [b.lattice(i).populations() for i in range(len(specs))]
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)


@pytest.mark.parametrize("shape3,shape2", [((128, 0), (64, 2)), ((64, 3), (256, 0)), ((128, 2), (128, 3))])
def test_batch_type_shapes_same_result(fl, shape3, shape2):
    # Each lattice type in its own per-step shape computes the same update, bit for bit;
    # the persistent form refuses per-type shapes and launches every type alike.
    specs = _specs(False)
    with fl.Batch(specs) as b:
        _init(b)
        b.set_type_shape(fl.FLBM_D3Q27, *shape3)
        b.set_type_shape(fl.FLBM_D2Q9, *shape2)
        assert b.type_shape(fl.FLBM_D3Q27) == shape3 and b.type_shape(fl.FLBM_D2Q9) == shape2
        assert b.shape == shape3
        b.step(3)
        b.step(4)
        b.sync()
        got = [b.lattice(i).populations() for i in range(len(specs))]
        b.shape = (128, 1)
        assert b.type_shape(fl.FLBM_D2Q9) == (128, 1)
        with pytest.raises(fl.FlbmError) as e:
            b.set_type_shape(fl.FLBM_D2Q9, 64, 0)
        assert e.value.status == fl.FLBM_ESTATE
    with fl.Batch(specs) as b:
        _init(b)
        b.step(7)
        ref = [b.lattice(i).populations() for i in range(len(specs))]
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)


def test_batch_autotune_leaves_state(fl):
    specs = _specs(False)
    with fl.Batch(specs) as b:
        _init(b)
        b.step(3)
        before = [b.lattice(i).populations() for i in range(len(specs))]
        t, f = b.autotune(4)
        assert t in (64, 128, 256) and f in (0, 1, 2, 3) and b.shape == (t, f)
        assert b.step_count == 3
        after = [b.lattice(i).populations() for i in range(len(specs))]
        for x, y in zip(before, after):
            assert np.array_equal(x, y)
        b.step(5)
        tuned = [b.lattice(i).populations() for i in range(len(specs))]
    with fl.Batch(specs) as b:
        _init(b)
        b.step(8)
        ref = [b.lattice(i).populations() for i in range(len(specs))]
    for x, y in zip(tuned, ref):
        assert np.array_equal(x, y)


def test_batch_member_rules_and_stats(fl, oracle_mod):
    specs = _specs(False)
    with fl.Batch(specs) as b:
        _init(b)
        lat = b.lattice(0)
        with pytest.raises(fl.FlbmError) as e:
            lat.step(1)
        assert e.value.status == fl.FLBM_ESTATE
        with pytest.raises(fl.FlbmError) as e:
            lat.variant = 2
        assert e.value.status == fl.FLBM_ESTATE
        fl.flbm_destroy(lat.ctx)  # ignored for a borrowed handle
        b.step(4)
        with pytest.raises(fl.FlbmError) as e:
            lat.init_uniform((0, 0, 0), 0.0, 0)
        assert e.value.status == fl.FLBM_ESTATE
        blob = lat.save()
        b.step(1)
        with pytest.raises(fl.FlbmError) as e:  # a checkpoint of another step
            lat.load(blob)
        assert e.value.status == fl.FLBM_ESTATE
        # statistics of a member: FP64 reduction against the oracle's
        for i, d in enumerate(specs):
            m = b.lattice(i)
            st = m.stats()
            so = oracle_mod.stats(d["lattice"], d["dims"], m.populations())
            assert st["step"] == 5
            # sum of rho - rho0 over the sites: the reduction's own error (tests/_gram_tol.py)
            n = int(np.prod(d["dims"]))
            drho2 = n * (so["k_cov"][0, 0] - 2 * d["rho0"] * so["k_mean"][0] + d["rho0"] ** 2)
            assert abs(st["mass"] - so["mass"]) <= 1e-9 * so["mass"] + sum_tol(drho2)
            # per-site products in FP32, sums in FP64: relative to the largest component, plus
            # the reduction's own error (tests/_gram_tol.py; some members have a few sites)
            scale = np.abs(so["uu"]).max()
            assert np.all(np.abs(np.asarray(st["uu"]) - so["uu"]) <= 1e-6 * scale + uu_tol(so["uu"], n))
        with pytest.raises(fl.FlbmError):
            b.lattice(len(specs))


def test_batch_stats_of_members_match_oracle(fl, oracle_mod):
    # flbm_batch_stats(b, i) of a D3Q27 and a D2Q9 member of one mixed batch (even and odd
    # rows), after an odd and an even number of steps, against the oracle's statistics of
    # the same populations (Sec. III: statistics over ensembles of runs).
    specs = _specs(False)
    with fl.Batch(specs) as b:
        _init(b)
        for steps in (5, 2):
            b.step(steps)
            for i in (0, 3):
                d = specs[i]
                st = b.stats(i)
                ref = oracle_mod.stats(d["lattice"], d["dims"], b.lattice(i).populations())
                n = int(np.prod(d["dims"]))
                assert st["step"] == b.step_count and st["sites"] == n and st["nonfinite"] == 0
                assert st["mass"] == pytest.approx(ref["mass"], rel=1e-7)
                u2 = np.abs(ref["uu"][:3]).max()
                np.testing.assert_allclose(st["mom"], ref["mom"], rtol=1e-5, atol=1e-6 * n)
                np.testing.assert_allclose(st["u_mean"], ref["u_mean"], rtol=1e-5, atol=1e-5 * np.sqrt(u2))
                np.testing.assert_allclose(st["uu"], ref["uu"], rtol=1e-5, atol=1e-6 * u2)
                scale = np.sqrt(np.abs(np.diag(ref["k_cov"])))
                np.testing.assert_allclose(st["k_mean"], ref["k_mean"], atol=1e-5 * scale.max() + 1e-9)
                np.testing.assert_allclose(st["k_cov"], ref["k_cov"], rtol=1e-4,
                                           atol=1e-5 * np.outer(scale, scale).max())
                # the same record as flbm_stats on the borrowed member handle
                same = b.lattice(i).stats()
                np.testing.assert_allclose(same["k_cov"], st["k_cov"], rtol=1e-12,
                                           atol=1e-12 * np.outer(scale, scale).max())
        for bad in (-1, len(specs)):
            with pytest.raises(fl.FlbmError) as e:
                b.stats(bad)
            assert e.value.status == fl.FLBM_EINVAL


def test_batch_invalid_specs(fl):
    good = _specs(False)[:2]
    bad = [dict(good[0]), dict(good[1])]
    bad[1]["dims"] = (4, 4, 4)
    bad[1]["lattice"] = 0  # D2Q9 with nz = 4
    bad[1]["lam"] = np.full(9, 1.5)
    with pytest.raises(fl.FlbmError) as e:
        fl.Batch(bad)
    assert e.value.status == fl.FLBM_EINVAL and "specs[1]" in str(e.value)
    with pytest.raises(fl.FlbmError):
        fl.flbm_batch_create([])
    with fl.Batch(good) as b:
        with pytest.raises(fl.FlbmError):
            b.shape = (96, 0)
        with pytest.raises(fl.FlbmError):
            b.shape = (256, 2)
        with pytest.raises(fl.FlbmError):
            b.shape = (128, 4)
        with pytest.raises(fl.FlbmError):
            b.step(-1)
        b.step(0)
        assert b.step_count == 0
        assert fl.flbm_batch_uses_graph(b.handle) in (0, 1)


def test_persistent_wait_timeout_reported_and_recoverable(fl):
    # The persistent form's completion waits are bounded: a launch whose waits can never
    # be satisfied (test hook) gives up after 2000 polls per wait, reports FLBM_ETIMEOUT at
    # the next sync, leaves the step count at the last completed launch, and the batch
    # keeps working afterwards. No GPU fault, trap or hang is involved.
    specs = _specs(False)
    with fl.Batch(specs) as b:
        _init(b)
        b.shape = (128, 1)
        fl.flbm_batch_test_wait_timeout(b.handle, 2000)
        b.step(3)
        with pytest.raises(fl.FlbmError) as e:
            b.sync()
        assert e.value.status == fl.FLBM_ETIMEOUT
        assert b.step_count == 0
        f0 = _init(b)  # allowed again at step 0
        b.step(5)
        b.sync()
        got = [b.lattice(i).populations() for i in range(len(specs))]
    with fl.Batch(specs) as b:
        ref0 = _init(b)
        b.step(5)
        ref = [b.lattice(i).populations() for i in range(len(specs))]
    for x, y in zip(f0, ref0):
        assert np.array_equal(x, y)
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)


def test_batch_at_the_lattice_limit(fl, oracle_mod):
    # FLBM_BATCH_MAX_LATTICES lattices (the by-value table of the kernel arguments is
    # full), mixed types, sizes and parities, every launch form; one more is refused.
    n = fl.FLBM_BATCH_MAX_LATTICES
    rng = np.random.default_rng(7)
    specs = []
    for j in range(n):
        if j % 2:
            dims = tuple(int(v) for v in rng.integers(1, 6, 3))
            specs.append(dict(lattice=1, dims=dims, lam=_lam(1, 1.0 + 0.9 * rng.random()), kBT=1e-4, rho0=1.0,
                              seed=5000 + j))
        else:
            dims = (int(rng.integers(1, 12)), int(rng.integers(1, 9)), 1)
            specs.append(dict(lattice=0, dims=dims, lam=_lam(0, 1.0 + 0.9 * rng.random()), kBT=1e-4, rho0=1.0,
                              seed=5000 + j))
    with pytest.raises(fl.FlbmError) as e:
        fl.Batch(specs + [specs[0]])
    assert e.value.status == fl.FLBM_EINVAL
    results = []
    for form in (0, 1, 2, 3):
        with fl.Batch(specs) as b:
            b.shape = (64 if form != 1 else 128, form)
            f0 = []
            for i in range(n):
                b.lattice(i).init_uniform((0.02, -0.01, 0.01), 1e-3, i)
                if i in (0, 1, n - 2, n - 1):
                    f0.append(b.lattice(i).populations())
            b.step(4)
            b.sync()
            results.append([b.lattice(i).populations() for i in (0, 1, n - 2, n - 1)])
    for r in results[1:]:
        for x, y in zip(r, results[0]):
            assert np.array_equal(x, y)
    for k, i in enumerate((0, 1, n - 2, n - 1)):
        d = specs[i]
        fo = oracle_mod.run(d["lattice"], d["dims"], d["lam"], d["kBT"], d["seed"], f0[k], 0, 4)
        assert _err(results[0][k], fo, d["lattice"], d["rho0"]) <= TOL, i


def test_batch_zero_temperature_members(fl, oracle_mod):
    # kBT = 0 (Test 1 of the paper): the batch kernels still draw the normals but scale
    # them by zero, so a member at rest stays exactly at rest and a drifting member follows
    # the deterministic oracle; a noisy member beside them is unaffected.
    specs = [
        dict(lattice=1, dims=(10, 6, 5), lam=_lam(1, 1.5), kBT=0.0, rho0=1.0, seed=1),
        dict(lattice=0, dims=(31, 12, 1), lam=_lam(0, 1.7), kBT=0.0, rho0=1.2, seed=2),
        dict(lattice=1, dims=(9, 7, 4), lam=_lam(1, 1.3), kBT=0.0, rho0=1.0, seed=3),
        dict(lattice=0, dims=(16, 10, 1), lam=_lam(0, 1.2), kBT=1e-4, rho0=1.0, seed=4),
    ]
    with fl.Batch(specs) as b:
        b.lattice(0).init_uniform((0.0, 0.0, 0.0), 0.0, 0)
        b.lattice(1).init_uniform((0.0, 0.0, 0.0), 0.0, 0)
        b.lattice(2).init_uniform((0.03, -0.02, 0.01), 1e-3, 5)
        b.lattice(3).init_uniform((0.0, 0.0, 0.0), 1e-3, 6)
        f0 = [b.lattice(i).populations() for i in range(len(specs))]
        b.step(12)
        got = [b.lattice(i).populations() for i in range(len(specs))]
    for i in (0, 1):
        assert np.array_equal(got[i], f0[i]), i
    for i in (2, 3):
        d = specs[i]
        fo = oracle_mod.run(d["lattice"], d["dims"], d["lam"], d["kBT"], d["seed"], f0[i], 0, 12)
        assert _err(got[i], fo, d["lattice"], d["rho0"]) <= TOL, i


def test_c5_ensemble_full_size_sampled_members(fl, oracle_mod):
    # The batched-ensemble workload at full size (256 lattices, 9.3 M sites, drawn as the
    # benchmark draws them) in the launch shape the autotuner picks, as the benchmark times
    # it: whole small members of both lattice types and both side parities against the
    # oracle over three steps (both parities), and the largest D3Q27 members with an even
    # and an odd side on sampled sites (their periodic seams among them) over one step.
    import bench

    specs = bench.draw_ensemble()
    n = len(specs)
    sizes = [int(np.prod(d["dims"])) for d in specs]
    picks, bigs = [], []
    for parity in (0, 1):
        for lattice in (0, 1):
            cand = [i for i in range(n) if specs[i]["lattice"] == lattice and specs[i]["dims"][0] % 2 == parity]
            if cand:
                picks.append(min(cand, key=lambda i: sizes[i]))
                if lattice == 1:
                    bigs.append(max(cand, key=lambda i: sizes[i]))
    c, w, _ = oracle_mod.tables(1)
    rng = np.random.default_rng(3)
    samples = {}
    for i in bigs:
        nx, ny, nz = specs[i]["dims"]
        xs, ys, zs = rng.integers(0, nx, 24), rng.integers(0, ny, 24), rng.integers(0, nz, 24)
        xs[:4] = [0, nx - 1, 0, nx - 1]
        ys[:4] = [0, ny - 1, ny - 1, 0]
        zs[:4] = [nz - 1, 0, 0, nz - 1]
        sites = xs + nx * (ys + ny * zs)
        dests = [((x + c[:, 0]) % nx) + nx * (((y + c[:, 1]) % ny) + ny * ((z + c[:, 2]) % nz))
                 for x, y, z in zip(xs, ys, zs)]
        samples[i] = (sites, dests)
    with fl.Batch(specs) as b:
        for i in range(n):
            b.lattice(i).init_uniform((0.0, 0.0, 0.0), 0.0, 0)
        b.autotune(4)
        b.step(2)
        f0 = {i: b.lattice(i).populations() for i in picks}
        pre = {i: b.lattice(i).sites_populations(samples[i][0]) for i in bigs}
        b.step(1)
        post = {i: [b.lattice(i).sites_populations(dst) for dst in samples[i][1]] for i in bigs}
        b.step(2)
        got = {i: b.lattice(i).populations() for i in picks}
    for i in bigs:
        d = specs[i]
        worst = 0.0
        for k, s in enumerate(samples[i][0]):
            eta = oracle_mod.site_eta(1, d["seed"], 2, int(s))
            fstar, _ = oracle_mod.collide_site(1, pre[i][k], d["lam"], d["kBT"], eta)
            worst = max(worst, float((np.abs(post[i][k][np.arange(27), np.arange(27)] - fstar) / w).max()))
        assert worst <= TOL, (i, d["dims"], worst)
    for i in picks:
        e = specs[i]
        fo = oracle_mod.run(e["lattice"], e["dims"], e["lam"], e["kBT"], e["seed"], f0[i], 2, 3)
        assert _err(got[i], fo, e["lattice"], e["rho0"]) <= TOL, (i, e["dims"])
