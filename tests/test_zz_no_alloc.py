"""flbm_stats_noalloc: the statistics for callers that cannot allocate GPU memory (an
application whose own pool owns the device-memory budget, a service whose footprint must
not change once running). Its accumulators live in a static device array instead of a
cudaMalloc'd buffer; its results must equal those of flbm_stats on the same state.
Collected last on purpose, so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _lam(q):
    lam = np.full(q, 1.3)
    lam[: (3 if q == 9 else 4)] = 1.0
    return lam


def _q(lattice):
    return {0: 9, 1: 27, 2: 27, 3: 19}[lattice]


def _close(got, ref, atol, what):
    got, ref = np.asarray(got, dtype=float), np.asarray(ref, dtype=float)
    bad = np.abs(got - ref) > atol
    assert not bad.any(), f"{what}: {int(bad.sum())} entries differ, max |diff| {np.abs(got - ref).max():.3e}"


def _assert_same_stats(got, ref):
    # Both sides sum the same per-site terms with FP64 atomics whose order varies from run
    # to run, so each entry is compared against the size of the terms summed into it
    # (about 1e-16 relative per addition), not against its own value, which can be a
    # near-cancellation (the mean of a noise mode).
    assert got["sites"] == ref["sites"] and got["nonfinite"] == 0
    assert got["step"] == -1
    tol = 1e-11
    n = ref["sites"]
    d = np.abs(np.diag(ref["k_cov"]))
    u2 = np.abs(ref["uu"][:3]).max()
    assert got["mass"] == pytest.approx(ref["mass"], rel=tol)
    _close(got["mom"], ref["mom"], tol * n * np.sqrt(d[0] * u2), "mom")
    _close(got["u_mean"], ref["u_mean"], tol * np.sqrt(u2), "u_mean")
    _close(got["uu"], ref["uu"], tol * u2, "uu")
    _close(got["k_mean"], ref["k_mean"], tol * np.sqrt(d), "k_mean")
    _close(got["k_cov"], ref["k_cov"], tol * np.sqrt(np.outer(d, d)), "k_cov")


@pytest.mark.parametrize("lattice,dims,storage", [
    (1, (24, 18, 10), 0),   # D3Q27 FP32, even nx: the pair-row path
    (0, (96, 64, 1), 1),    # D2Q9 BF16
    (1, (23, 10, 9), 0),    # D3Q27 FP32, odd nx: one site per row slot
    (2, (20, 12, 8), 2),    # isotropic D3Q27, FP16
    (3, (18, 10, 12), 0),   # D3Q19 FP32
    (3, (15, 8, 6), 1),     # D3Q19 BF16, odd nx
])
def test_noalloc_stats_equal_flbm_stats_on_two_calls_in_a_row(lattice, dims, storage):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_16486_gb300 as fl

    q = _q(lattice)
    nbytes = fl.flbm_required_bytes(lattice, dims, storage)
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")  # caller-owned populations
    stream = torch.cuda.Stream()
    ctx = fl.flbm_create_ex(lattice, dims, _lam(q), 1e-3, 1.0, 17, storage, stream.cuda_stream,
                            buf.data_ptr(), nbytes)
    try:
        fl.flbm_init_uniform(ctx, (0.03, -0.02, 0.01), 1e-3, 5)
        for steps in (5, 2):  # odd, then odd again: parity 1 and the next parity 1 state
            fl.flbm_step(ctx, steps)
            ref = fl.flbm_stats(ctx)
            parity = fl.flbm_get_step(ctx) & 1
            for _ in range(2):  # two calls in a row share (and re-zero) the scratch
                got = fl.flbm_stats_noalloc(lattice, dims, storage, parity, 1.0, buf.data_ptr(),
                                            stream.cuda_stream)
                _assert_same_stats(got, ref)
        fl.flbm_step(ctx, 1)  # even parity
        ref = fl.flbm_stats(ctx)
        got = fl.flbm_stats_noalloc(lattice, dims, storage, 0, 1.0, buf.data_ptr(), stream.cuda_stream)
        _assert_same_stats(got, ref)
    finally:
        fl.flbm_destroy(ctx)


def test_noalloc_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_16486_gb300 as fl

    buf = torch.empty(27 * 8 * 8 * 8 * 4 + 256, dtype=torch.uint8, device="cuda")
    ptr = buf.data_ptr()
    assert ptr % 256 == 0
    cases = [
        ((1, (8, 8, 8), 0, 2, 1.0), ptr),    # parity
        ((1, (8, 8, 8), 0, 0, -1.0), ptr),   # rho0
        ((5, (8, 8, 8), 0, 0, 1.0), ptr),    # lattice
        ((1, (8, 8, 8), 0, 0, 1.0), ptr + 4),  # one FP32 element off: rejected on the host
        ((1, (8, 8, 8), 0, 0, 1.0), ptr + 8),  # pair-aligned but not 256-byte aligned
    ]
    for args, p in cases:
        with pytest.raises(fl.FlbmError) as ei:
            fl.flbm_stats_noalloc(*args, p)
        assert ei.value.status == fl.FLBM_EINVAL
