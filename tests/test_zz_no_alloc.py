"""flbm_stats_noalloc: the statistics for callers that cannot allocate GPU memory (a
memory pool that owns the device budget, a fixed footprint, a stream capture). Its
accumulators live in a static device array instead of a cudaMalloc'd buffer; its
results must equal those of flbm_stats on the same state. Collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _lam(q):
    lam = np.full(q, 1.3)
    lam[: (3 if q == 9 else 4)] = 1.0
    return lam


@pytest.mark.parametrize("lattice,dims,storage", [(1, (24, 18, 10), 0), (0, (96, 64, 1), 1)])
def test_noalloc_stats_equal_flbm_stats_on_two_calls_in_a_row(lattice, dims, storage):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_16486_gb300 as fl

    q = 9 if lattice == 0 else 27
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
                assert got["sites"] == ref["sites"] and got["nonfinite"] == 0
                assert got["step"] == -1
                for key in ("mass", "mom", "u_mean", "uu", "k_mean", "k_cov"):
                    np.testing.assert_allclose(got[key], ref[key], rtol=1e-12, atol=1e-300, err_msg=key)
        fl.flbm_step(ctx, 1)  # even parity
        ref = fl.flbm_stats(ctx)
        got = fl.flbm_stats_noalloc(lattice, dims, storage, 0, 1.0, buf.data_ptr(), stream.cuda_stream)
        np.testing.assert_allclose(got["k_cov"], ref["k_cov"], rtol=1e-12, atol=1e-300)
    finally:
        fl.flbm_destroy(ctx)


def test_noalloc_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_16486_gb300 as fl

    buf = torch.empty(27 * 8 * 8 * 8 * 4, dtype=torch.uint8, device="cuda")
    for args in ((1, (8, 8, 8), 0, 2, 1.0), (1, (8, 8, 8), 0, 0, -1.0), (5, (8, 8, 8), 0, 0, 1.0)):
        with pytest.raises(fl.FlbmError) as ei:
            fl.flbm_stats_noalloc(*args, buf.data_ptr())
        assert ei.value.status == fl.FLBM_EINVAL
