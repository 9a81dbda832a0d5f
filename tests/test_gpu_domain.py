"""GPU checks of the slab decomposition (flbm_domain_*, flbm_create_slab): a lattice split
along z into slabs, in one process on one GPU, evolves bitwise like the whole lattice,
because the noise is keyed on the global site and every slot crosses a slab face by copy
(the periodic streaming of Eq. streaming across the decomposition)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fl():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_16486_gb300 as fl

    return fl


def _lam(lattice, shear=1.6, rest=1.0, general=False):
    q = 19 if lattice == 3 else 27
    lam = np.full(q, rest)
    lam[:4] = 1.0
    lam[[7, 8, 9]] = shear
    if lattice == 2:
        lam[[5, 6]] = shear
    if general:
        lam[4:] = np.random.default_rng(3).uniform(0.4, 1.9, q - 4)
    return lam


def _same_stats(got, ref):
    # The per-site values are bitwise the same, but the reduction sums a tile's sites in
    # FP32 (tensor-core Gram fragments, flushed to FP64 every few tiles), so grouping the
    # sites by slab moves each sum by FP32 rounding of the partial sums: compare at that
    # level, relative to the size of the summed terms.
    assert got["mass"] == pytest.approx(ref["mass"], rel=1e-9)
    d = np.abs(np.diag(ref["k_cov"]))
    assert np.all(np.abs(np.asarray(got["k_cov"]) - ref["k_cov"]) <= 1e-6 * np.sqrt(np.outer(d, d)))
    assert np.all(np.abs(np.asarray(got["k_mean"]) - ref["k_mean"]) <= 1e-6 * np.sqrt(d))
    u2 = np.abs(ref["uu"][:3]).max()
    assert np.all(np.abs(np.asarray(got["uu"]) - ref["uu"]) <= 1e-6 * u2)
    assert np.all(np.abs(np.asarray(got["u_mean"]) - ref["u_mean"]) <= 1e-6 * np.sqrt(u2))


CASES = [  # lattice, dims, slabs, variant, general rates
    (1, (24, 10, 9), 2, 2, False),   # D3Q27, paper rates, two-site kernel, slabs of 5 and 4 planes
    (1, (24, 10, 9), 3, 5, True),    # D3Q27, general rates, three slabs
    (1, (23, 6, 7), 2, 1, False),    # D3Q27, odd nx: one site per thread
    (2, (20, 8, 6), 2, 2, False),    # isotropic D3Q27
    (3, (18, 8, 10), 4, 2, False),   # D3Q19, four slabs
    (1, (16, 6, 4), 4, 2, False),    # one plane per slab
    (1, (16, 6, 5), 1, 2, False),    # one slab: its own neighbour
]


@pytest.mark.parametrize("lattice,dims,nslabs,variant,general", CASES)
def test_domain_steps_bitwise_like_the_whole_lattice(fl, lattice, dims, nslabs, variant, general):
    lam = _lam(lattice, general=general)
    kBT, rho0, seed = 2e-4, 1.0, 77
    with fl.Lattice(lattice, dims, lam, kBT, rho0, seed) as whole, \
            fl.Domain(lattice, dims, lam, kBT, rho0, seed, nslabs=nslabs) as dom:
        assert len(dom) == nslabs
        whole.variant = variant
        dom.variant = variant
        whole.init_uniform((0.04, -0.02, 0.01), 1e-3, 9)
        dom.init_uniform((0.04, -0.02, 0.01), 1e-3, 9)
        assert np.array_equal(dom.populations(), whole.populations())
        for n in (7, 1, 4):  # odd, even, even states
            whole.step(n)
            dom.step(n)
            assert dom.step_count == whole.step_count
            fw, fd = whole.populations(), dom.populations()
            assert np.array_equal(fd, fw), f"step {whole.step_count}: max |diff| {np.abs(fd - fw).max():.3e}"
            sw, sd = whole.stats(), dom.stats()
            assert sd["sites"] == sw["sites"] and sd["step"] == sw["step"] and sd["nonfinite"] == 0
            _same_stats(sd, sw)


def test_domain_set_populations_in_an_odd_state(fl):
    # Populations written into a domain in an odd AA state land in the right slab's slots
    # (some of a slab's arriving populations live in its neighbour's planes).
    lattice, dims = 1, (12, 6, 8)
    lam = _lam(lattice)
    with fl.Lattice(lattice, dims, lam, 1e-4, 1.0, 5) as whole, \
            fl.Domain(lattice, dims, lam, 1e-4, 1.0, 5, nslabs=3) as dom:
        whole.init_uniform((0.02, 0.0, -0.03), 1e-3, 1)
        whole.step(3)
        f = whole.populations()
        dom.init_uniform()
        dom.step(3)  # same step count (odd), other state
        dom.set_populations(f)
        assert np.array_equal(dom.populations(), f)
        whole.step(5)
        dom.step(5)
        assert np.array_equal(dom.populations(), whole.populations())


def test_single_rank_slab_lattice_matches_whole(fl):
    # The multi-process driver (paper_2602_16486_gb300.slab) with one rank: the halo moves
    # by device copies between views of the caller-owned buffer.
    import torch

    from paper_2602_16486_gb300 import slab

    lattice, dims = 1, (16, 8, 6)
    lam = _lam(lattice)
    s = slab.SlabLattice(lattice, dims, lam, 3e-4, 1.0, 21, rank=0, world=1)
    try:
        with fl.Lattice(lattice, dims, lam, 3e-4, 1.0, 21) as whole:
            s.init_uniform((0.03, 0.01, 0.0), 1e-3, 2)
            whole.init_uniform((0.03, 0.01, 0.0), 1e-3, 2)
            s.step(5)
            whole.step(5)
            st, sw = s.stats(), whole.stats()
            assert st["sites"] == sw["sites"]
            _same_stats(st, sw)
            # the owned planes of the slab's array hold the whole lattice's state
            s.step(1)
            whole.step(1)
            loc = fl.flbm_get_populations(s.ctx, lattice, (dims[0], dims[1], dims[2] + 2))
            assert np.array_equal(loc[:, 1:dims[2] + 1], whole.populations())
    finally:
        s.close()
        torch.cuda.synchronize()


def test_slab_rules(fl):
    lam = _lam(1)
    with pytest.raises(fl.FlbmError) as e:
        fl.Domain(0, (8, 8, 1), np.ones(9), 1e-4, 1.0, 0, nslabs=2)
    assert e.value.status == fl.FLBM_EINVAL
    with pytest.raises(fl.FlbmError) as e:
        fl.Domain(1, (8, 8, 3), lam, 1e-4, 1.0, 0, nslabs=4)  # more slabs than planes
    assert e.value.status == fl.FLBM_EINVAL
    ctx = fl.flbm_create_slab(1, (8, 8, 6), 2, 3, lam, 1e-4, 1.0, 0)
    try:
        with pytest.raises(fl.FlbmError) as e:
            fl.flbm_step(ctx, 2)  # one step per call
        assert e.value.status == fl.FLBM_EINVAL
        with pytest.raises(fl.FlbmError) as e:
            fl.flbm_autotune(ctx, 4)
        assert e.value.status == fl.FLBM_ESTATE
        fl.flbm_set_step_variant(ctx, 4)
        assert fl.flbm_get_step_variant(ctx) == 2  # the pipelined kernel walks whole boxes
        assert fl.flbm_stats(ctx)["sites"] == 8 * 8 * 3
    finally:
        fl.flbm_destroy(ctx)
