"""ctypes binding of libflbm.so (include/flbm.h), function for function, same names.

Argument marshalling only: numpy arrays and Python numbers are converted to the C
types, status codes other than FLBM_OK become ``FlbmError``. Every step of the
computation runs in the CUDA kernels of the library. There is no fallback: if the
library is missing or cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libflbm.so")

FLBM_D2Q9, FLBM_D3Q27, FLBM_D3Q27_ISO, FLBM_D3Q19 = 0, 1, 2, 3
FLBM_FP32, FLBM_BF16, FLBM_FP16 = 0, 1, 2
FLBM_OK, FLBM_EINVAL, FLBM_ENOMEM, FLBM_ECUDA, FLBM_ENUMERIC, FLBM_ETIMEOUT, FLBM_ESTATE = range(7)
STATUS_NAMES = {0: "FLBM_OK", 1: "FLBM_EINVAL", 2: "FLBM_ENOMEM", 3: "FLBM_ECUDA",
                4: "FLBM_ENUMERIC", 5: "FLBM_ETIMEOUT", 6: "FLBM_ESTATE"}
Q_OF = {FLBM_D2Q9: 9, FLBM_D3Q27: 27, FLBM_D3Q27_ISO: 27, FLBM_D3Q19: 19}
D_OF = {FLBM_D2Q9: 2, FLBM_D3Q27: 3, FLBM_D3Q27_ISO: 3, FLBM_D3Q19: 3}


class FlbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class flbm_stats_t(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64),
        ("sites", ctypes.c_int64),
        ("nonfinite", ctypes.c_int64),
        ("lattice", ctypes.c_int32),
        ("q", ctypes.c_int32),
        ("mass", ctypes.c_double),
        ("mom", ctypes.c_double * 3),
        ("u_mean", ctypes.c_double * 3),
        ("uu", ctypes.c_double * 6),
        ("k_mean", ctypes.c_double * 27),
        ("k_cov", ctypes.c_double * (27 * 27)),
    ]

    def to_dict(self):
        q = self.q
        return {
            "step": self.step, "sites": self.sites, "nonfinite": self.nonfinite,
            "lattice": self.lattice, "q": q, "mass": self.mass,
            "mom": np.array(self.mom[:]), "u_mean": np.array(self.u_mean[:]),
            "uu": np.array(self.uu[:]), "k_mean": np.array(self.k_mean[:q]),
            "k_cov": np.array(self.k_cov[:q * q]).reshape(q, q),
        }


class flbm_lattice_spec(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("dims", ctypes.c_int64 * 3),
        ("lambda_", ctypes.c_double * 27),
        ("kBT", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


FLBM_BATCH_MAX_LATTICES = 512


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    i64p = ctypes.POINTER(ctypes.c_int64)
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "flbm_required_bytes": (ctypes.c_size_t, [ctypes.c_int, i64p, ctypes.c_int]),
        "flbm_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, i64p, dp, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64]),
        "flbm_create_ex": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, i64p, dp, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_uint64, ctypes.c_int, vp, vp,
                                          ctypes.c_size_t]),
        "flbm_destroy": (None, [vp]),
        "flbm_init_uniform": (ctypes.c_int, [vp, dp, ctypes.c_double, ctypes.c_uint64]),
        "flbm_step": (ctypes.c_int, [vp, ctypes.c_int64]),
        "flbm_get_step": (ctypes.c_int64, [vp]),
        "flbm_stats": (ctypes.c_int, [vp, ctypes.POINTER(flbm_stats_t)]),
        "flbm_sample": (ctypes.c_int, [vp]),
        "flbm_fetch_samples": (ctypes.c_int, [vp, ctypes.POINTER(flbm_stats_t), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int)]),
        "flbm_set_sample_capacity": (ctypes.c_int, [vp, ctypes.c_int]),
        "flbm_sample_capacity": (ctypes.c_int, [vp]),
        "flbm_get_populations": (ctypes.c_int, [vp, dp, ctypes.c_size_t]),
        "flbm_set_populations": (ctypes.c_int, [vp, dp, ctypes.c_size_t]),
        "flbm_get_sites": (ctypes.c_int, [vp, i64p, ctypes.c_size_t, dp]),
        "flbm_checkpoint_bytes": (ctypes.c_size_t, [vp]),
        "flbm_save": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
        "flbm_load": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
        "flbm_sync": (ctypes.c_int, [vp]),
        "flbm_set_step_variant": (ctypes.c_int, [vp, ctypes.c_int]),
        "flbm_get_step_variant": (ctypes.c_int, [vp]),
        "flbm_set_collision": (ctypes.c_int, [vp, ctypes.c_int]),
        "flbm_get_collision": (ctypes.c_int, [vp]),
        "flbm_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "flbm_stats_noalloc": (ctypes.c_int, [ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_double, vp, vp, ctypes.POINTER(flbm_stats_t)]),
        "flbm_last_error": (ctypes.c_char_p, []),
        "flbm_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(flbm_lattice_spec),
                                             ctypes.c_int, vp]),
        "flbm_batch_destroy": (None, [vp]),
        "flbm_batch_size": (ctypes.c_int, [vp]),
        "flbm_batch_lattice": (vp, [vp, ctypes.c_int]),
        "flbm_batch_step": (ctypes.c_int, [vp, ctypes.c_int64]),
        "flbm_batch_stats": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(flbm_stats_t)]),
        "flbm_batch_get_step": (ctypes.c_int64, [vp]),
        "flbm_batch_set_shape": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
        "flbm_batch_get_shape": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
        "flbm_batch_set_type_shape": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "flbm_batch_get_type_shape": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                     ctypes.POINTER(ctypes.c_int)]),
        "flbm_batch_autotune": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int)]),
        "flbm_batch_uses_graph": (ctypes.c_int, [vp]),
        "flbm_batch_sync": (ctypes.c_int, [vp]),
        "flbm_batch_test_wait_timeout": (ctypes.c_int, [vp, ctypes.c_uint32]),
        "flbm_slab_required_bytes": (ctypes.c_size_t, [ctypes.c_int, i64p, ctypes.c_int64, ctypes.c_int]),
        "flbm_create_slab": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, i64p, ctypes.c_int64, ctypes.c_int64,
                                            dp, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_int, vp,
                                            vp, ctypes.c_size_t]),
        "flbm_slab_halo": (ctypes.c_int, [ctypes.c_int, i64p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, i64p, i64p,
                                          ctypes.POINTER(ctypes.c_int), i64p]),
        "flbm_domain_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, i64p, dp, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int)]),
        "flbm_domain_destroy": (None, [vp]),
        "flbm_domain_size": (ctypes.c_int, [vp]),
        "flbm_domain_slab": (vp, [vp, ctypes.c_int]),
        "flbm_domain_init_uniform": (ctypes.c_int, [vp, dp, ctypes.c_double, ctypes.c_uint64]),
        "flbm_domain_step": (ctypes.c_int, [vp, ctypes.c_int64]),
        "flbm_domain_get_step": (ctypes.c_int64, [vp]),
        "flbm_domain_set_step_variant": (ctypes.c_int, [vp, ctypes.c_int]),
        "flbm_domain_stats": (ctypes.c_int, [vp, ctypes.POINTER(flbm_stats_t)]),
        "flbm_domain_get_populations": (ctypes.c_int, [vp, dp, ctypes.c_size_t]),
        "flbm_domain_set_populations": (ctypes.c_int, [vp, dp, ctypes.c_size_t]),
        "flbm_domain_sync": (ctypes.c_int, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _check(status):
    if status != FLBM_OK:
        raise FlbmError(status, _lib.flbm_last_error().decode())
    return status


def _dims(dims):
    d = [int(x) for x in dims] + [1] * (3 - len(dims))
    return (ctypes.c_int64 * 3)(*d)


def _lambda(lattice, lam):
    q = Q_OF.get(lattice)  # an unknown lattice is reported by the library itself
    arr = np.ascontiguousarray(np.asarray(lam, dtype=np.float64))
    if q is not None and arr.size != q:
        raise ValueError(f"lambda needs {q} entries, got {arr.size}")
    return arr


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---- the C ABI, name for name -----------------------------------------------------------
def flbm_required_bytes(lattice, dims, storage=FLBM_FP32):
    return int(_lib.flbm_required_bytes(int(lattice), _dims(dims), int(storage)))


def flbm_create(lattice, dims, lam, kBT, rho0, seed):
    ctx = ctypes.c_void_p()
    lam = _lambda(lattice, lam)
    _check(_lib.flbm_create(ctypes.byref(ctx), int(lattice), _dims(dims), _dp(lam), float(kBT),
                            float(rho0), int(seed) & 0xFFFFFFFFFFFFFFFF))
    return ctx


def flbm_create_ex(lattice, dims, lam, kBT, rho0, seed, storage=FLBM_FP32, cuda_stream=None,
                   dev_buf=None, dev_buf_bytes=0):
    ctx = ctypes.c_void_p()
    lam = _lambda(lattice, lam)
    _check(_lib.flbm_create_ex(ctypes.byref(ctx), int(lattice), _dims(dims), _dp(lam), float(kBT),
                               float(rho0), int(seed) & 0xFFFFFFFFFFFFFFFF, int(storage),
                               ctypes.c_void_p(cuda_stream or 0) if cuda_stream else None,
                               ctypes.c_void_p(dev_buf) if dev_buf else None, int(dev_buf_bytes)))
    return ctx


def flbm_destroy(ctx):
    _lib.flbm_destroy(ctx)


def flbm_init_uniform(ctx, u0=(0.0, 0.0, 0.0), rho_perturb_amp=0.0, perturb_seed=0):
    u = np.ascontiguousarray(np.asarray(list(u0) + [0.0] * (3 - len(u0)), dtype=np.float64))
    _check(_lib.flbm_init_uniform(ctx, _dp(u), float(rho_perturb_amp), int(perturb_seed)))


def flbm_step(ctx, n=1):
    _check(_lib.flbm_step(ctx, int(n)))


def flbm_get_step(ctx):
    return int(_lib.flbm_get_step(ctx))


def flbm_stats(ctx, allow_nonfinite=False):
    out = flbm_stats_t()
    st = _lib.flbm_stats(ctx, ctypes.byref(out))
    if st == FLBM_ENUMERIC and allow_nonfinite:
        return out.to_dict()
    _check(st)
    return out.to_dict()


def flbm_sample(ctx):
    _check(_lib.flbm_sample(ctx))


def flbm_fetch_samples(ctx, max_n=None, allow_nonfinite=False):
    cap = int(_lib.flbm_sample_capacity(ctx))
    max_n = cap if max_n is None else int(max_n)
    buf = (flbm_stats_t * max(max_n, 1))()
    n = ctypes.c_int(0)
    st = _lib.flbm_fetch_samples(ctx, buf, max_n, ctypes.byref(n))
    if not (st == FLBM_ENUMERIC and allow_nonfinite):
        _check(st)
    return [buf[k].to_dict() for k in range(n.value)]


def flbm_set_sample_capacity(ctx, cap):
    _check(_lib.flbm_set_sample_capacity(ctx, int(cap)))


def flbm_sample_capacity(ctx):
    return int(_lib.flbm_sample_capacity(ctx))


def flbm_get_populations(ctx, lattice, dims):
    q = Q_OF[lattice]
    d = [int(x) for x in dims] + [1] * (3 - len(dims))
    out = np.empty((q, d[2], d[1], d[0]), dtype=np.float64)
    _check(_lib.flbm_get_populations(ctx, _dp(out), out.size))
    return out


def flbm_set_populations(ctx, f):
    arr = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    _check(_lib.flbm_set_populations(ctx, _dp(arr), arr.size))


def flbm_get_sites(ctx, lattice, sites):
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    out = np.empty((s.size, Q_OF[lattice]), dtype=np.float64)
    _check(_lib.flbm_get_sites(ctx, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), s.size, _dp(out)))
    return out


def flbm_checkpoint_bytes(ctx):
    return int(_lib.flbm_checkpoint_bytes(ctx))


def flbm_save(ctx, host_ptr=None, nbytes=None):
    """Save into a caller buffer (address, size) or, by default, a new bytearray."""
    if host_ptr is None:
        n = flbm_checkpoint_bytes(ctx)
        buf = bytearray(n)
        cbuf = (ctypes.c_char * n).from_buffer(buf)
        _check(_lib.flbm_save(ctx, ctypes.cast(cbuf, ctypes.c_void_p), n))
        return buf
    _check(_lib.flbm_save(ctx, ctypes.c_void_p(host_ptr), int(nbytes)))
    return None


def flbm_load(ctx, blob=None, host_ptr=None, nbytes=None):
    if blob is not None:
        n = len(blob)
        cbuf = (ctypes.c_char * n).from_buffer(blob)
        _check(_lib.flbm_load(ctx, ctypes.cast(cbuf, ctypes.c_void_p), n))
    else:
        _check(_lib.flbm_load(ctx, ctypes.c_void_p(host_ptr), int(nbytes)))


def flbm_sync(ctx):
    _check(_lib.flbm_sync(ctx))


def flbm_stats_noalloc(lattice, dims, storage, parity, rho0, dev_populations, cuda_stream=None,
                       allow_nonfinite=False):
    """Statistics of a caller-owned device population array; the library allocates
    nothing for this call (see include/flbm.h)."""
    out = flbm_stats_t()
    st = _lib.flbm_stats_noalloc(int(lattice), _dims(dims), int(storage), int(parity), float(rho0),
                                 ctypes.c_void_p(dev_populations),
                                 ctypes.c_void_p(cuda_stream) if cuda_stream else None,
                                 ctypes.byref(out))
    if not (st == FLBM_ENUMERIC and allow_nonfinite):
        _check(st)
    return out.to_dict()


def flbm_set_step_variant(ctx, variant):
    _check(_lib.flbm_set_step_variant(ctx, int(variant)))


def flbm_get_step_variant(ctx):
    return int(_lib.flbm_get_step_variant(ctx))


FLBM_COLLISION_CM = 0
FLBM_COLLISION_RAW = 1


def flbm_set_collision(ctx, model):
    _check(_lib.flbm_set_collision(ctx, int(model)))


def flbm_get_collision(ctx):
    return int(_lib.flbm_get_collision(ctx))


def flbm_autotune(ctx, trial_steps=10):
    chosen = ctypes.c_int(-1)
    _check(_lib.flbm_autotune(ctx, int(trial_steps), ctypes.byref(chosen)))
    return chosen.value


def flbm_last_error():
    return _lib.flbm_last_error().decode()


def _spec(d):
    """One flbm_lattice_spec from a dict: lattice, dims, lam (Q rates), kBT, rho0, seed."""
    lattice = int(d["lattice"])
    lam = _lambda(lattice, d["lam"])
    s = flbm_lattice_spec()
    s.lattice = lattice
    s.reserved = 0
    dd = [int(x) for x in d["dims"]] + [1] * (3 - len(d["dims"]))
    for a in range(3):
        s.dims[a] = dd[a]
    for v in range(lam.size):
        s.lambda_[v] = float(lam[v])
    s.kBT = float(d["kBT"])
    s.rho0 = float(d.get("rho0", 1.0))
    s.seed = int(d.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    return s


def flbm_batch_create(specs, cuda_stream=None):
    arr = (flbm_lattice_spec * max(len(specs), 1))(*[_spec(d) for d in specs])
    b = ctypes.c_void_p()
    _check(_lib.flbm_batch_create(ctypes.byref(b), arr, len(specs),
                                  ctypes.c_void_p(cuda_stream) if cuda_stream else None))
    return b


def flbm_batch_destroy(b):
    _lib.flbm_batch_destroy(b)


def flbm_batch_size(b):
    return int(_lib.flbm_batch_size(b))


def flbm_batch_lattice(b, i):
    h = _lib.flbm_batch_lattice(b, int(i))
    if not h:
        raise FlbmError(FLBM_EINVAL, _lib.flbm_last_error().decode())
    return ctypes.c_void_p(h)


def flbm_batch_step(b, n=1):
    _check(_lib.flbm_batch_step(b, int(n)))


def flbm_batch_stats(b, i, allow_nonfinite=False):
    out = flbm_stats_t()
    st = _lib.flbm_batch_stats(b, int(i), ctypes.byref(out))
    if not (st == FLBM_ENUMERIC and allow_nonfinite):
        _check(st)
    return out.to_dict()


def flbm_batch_get_step(b):
    return int(_lib.flbm_batch_get_step(b))


FLBM_BATCH_STEP, FLBM_BATCH_PERSISTENT, FLBM_BATCH_STEP_OCC, FLBM_BATCH_STEP_ROLLED = 0, 1, 2, 3


def flbm_batch_set_shape(b, threads, form):
    _check(_lib.flbm_batch_set_shape(b, int(threads), int(form)))


def flbm_batch_get_shape(b):
    t = ctypes.c_int(-1)
    f = ctypes.c_int(-1)
    _check(_lib.flbm_batch_get_shape(b, ctypes.byref(t), ctypes.byref(f)))
    return t.value, f.value


def flbm_batch_set_type_shape(b, lattice, threads, form):
    _check(_lib.flbm_batch_set_type_shape(b, int(lattice), int(threads), int(form)))


def flbm_batch_get_type_shape(b, lattice):
    t = ctypes.c_int(-1)
    f = ctypes.c_int(-1)
    _check(_lib.flbm_batch_get_type_shape(b, int(lattice), ctypes.byref(t), ctypes.byref(f)))
    return t.value, f.value


def flbm_batch_autotune(b, trial_steps=10):
    """Returns (threads, form) of the fastest launch shape."""
    t = ctypes.c_int(-1)
    f = ctypes.c_int(-1)
    _check(_lib.flbm_batch_autotune(b, int(trial_steps), ctypes.byref(t), ctypes.byref(f)))
    return t.value, f.value


def flbm_batch_uses_graph(b):
    return int(_lib.flbm_batch_uses_graph(b))


def flbm_batch_sync(b):
    _check(_lib.flbm_batch_sync(b))


def flbm_batch_test_wait_timeout(b, polls):
    _check(_lib.flbm_batch_test_wait_timeout(b, int(polls)))


def flbm_slab_required_bytes(lattice, dims, z_count, storage=FLBM_FP32):
    return int(_lib.flbm_slab_required_bytes(int(lattice), _dims(dims), int(z_count), int(storage)))


def flbm_create_slab(lattice, dims, z_begin, z_count, lam, kBT, rho0, seed, storage=FLBM_FP32, cuda_stream=None,
                     dev_buf=None, dev_buf_bytes=0):
    ctx = ctypes.c_void_p()
    lam = _lambda(lattice, lam)
    _check(_lib.flbm_create_slab(ctypes.byref(ctx), int(lattice), _dims(dims), int(z_begin), int(z_count), _dp(lam),
                                 float(kBT), float(rho0), int(seed) & 0xFFFFFFFFFFFFFFFF, int(storage),
                                 ctypes.c_void_p(cuda_stream) if cuda_stream else None,
                                 ctypes.c_void_p(dev_buf) if dev_buf else None, int(dev_buf_bytes)))
    return ctx


def flbm_slab_halo(lattice, dims, z_count, phase, side):
    """(send_offsets, recv_offsets, region_len) of one halo message, in elements."""
    so = (ctypes.c_int64 * 9)()
    ro = (ctypes.c_int64 * 9)()
    n = ctypes.c_int(0)
    ln = ctypes.c_int64(0)
    _check(_lib.flbm_slab_halo(int(lattice), _dims(dims), int(z_count), int(phase), int(side), so, ro,
                               ctypes.byref(n), ctypes.byref(ln)))
    return [int(so[k]) for k in range(n.value)], [int(ro[k]) for k in range(n.value)], int(ln.value)


def flbm_domain_create(lattice, dims, lam, kBT, rho0, seed, storage=FLBM_FP32, nslabs=2, devices=None):
    d = ctypes.c_void_p()
    lam = _lambda(lattice, lam)
    devs = (ctypes.c_int * int(nslabs))(*[int(x) for x in devices]) if devices is not None else None
    _check(_lib.flbm_domain_create(ctypes.byref(d), int(lattice), _dims(dims), _dp(lam), float(kBT), float(rho0),
                                   int(seed) & 0xFFFFFFFFFFFFFFFF, int(storage), int(nslabs), devs))
    return d


def flbm_domain_destroy(d):
    _lib.flbm_domain_destroy(d)


def flbm_domain_size(d):
    return int(_lib.flbm_domain_size(d))


def flbm_domain_slab(d, k):
    ctx = _lib.flbm_domain_slab(d, int(k))
    if not ctx:
        raise FlbmError(FLBM_EINVAL, _lib.flbm_last_error().decode())
    return ctypes.c_void_p(ctx)


def flbm_domain_init_uniform(d, u0=(0.0, 0.0, 0.0), rho_perturb_amp=0.0, perturb_seed=0):
    u = np.ascontiguousarray(np.asarray(list(u0) + [0.0] * (3 - len(u0)), dtype=np.float64))
    _check(_lib.flbm_domain_init_uniform(d, _dp(u), float(rho_perturb_amp), int(perturb_seed)))


def flbm_domain_step(d, n=1):
    _check(_lib.flbm_domain_step(d, int(n)))


def flbm_domain_get_step(d):
    return int(_lib.flbm_domain_get_step(d))


def flbm_domain_set_step_variant(d, variant):
    _check(_lib.flbm_domain_set_step_variant(d, int(variant)))


def flbm_domain_stats(d, allow_nonfinite=False):
    out = flbm_stats_t()
    st = _lib.flbm_domain_stats(d, ctypes.byref(out))
    if not (st == FLBM_ENUMERIC and allow_nonfinite):
        _check(st)
    return out.to_dict()


def flbm_domain_get_populations(d, lattice, dims):
    q = Q_OF[lattice]
    out = np.empty((q, int(dims[2]), int(dims[1]), int(dims[0])), dtype=np.float64)
    _check(_lib.flbm_domain_get_populations(d, _dp(out), out.size))
    return out


def flbm_domain_set_populations(d, f):
    arr = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    _check(_lib.flbm_domain_set_populations(d, _dp(arr), arr.size))


def flbm_domain_sync(d):
    _check(_lib.flbm_domain_sync(d))


# ---- a thin owner object over the same calls ---------------------------------------------
class Lattice:
    """Owns one context; methods forward to the C ABI calls of the same name."""

    def __init__(self, lattice, dims, lam, kBT, rho0=1.0, seed=0, storage=FLBM_FP32,
                 cuda_stream=None, dev_buf=None, dev_buf_bytes=0, _borrowed=None):
        self.lattice = int(lattice)
        self.dims = tuple(int(x) for x in dims) + (1,) * (3 - len(dims))
        self.q = Q_OF[self.lattice]
        self.storage = storage
        self._owned = _borrowed is None
        if _borrowed is not None:
            self.ctx = _borrowed
        else:
            self.ctx = flbm_create_ex(lattice, self.dims, lam, kBT, rho0, seed, storage, cuda_stream,
                                      dev_buf, dev_buf_bytes)

    @property
    def sites(self):
        return self.dims[0] * self.dims[1] * self.dims[2]

    def init_uniform(self, u0=(0.0, 0.0, 0.0), amp=0.0, perturb_seed=0):
        flbm_init_uniform(self.ctx, u0, amp, perturb_seed)

    def step(self, n=1):
        flbm_step(self.ctx, n)

    @property
    def step_count(self):
        return flbm_get_step(self.ctx)

    def stats(self, allow_nonfinite=False):
        return flbm_stats(self.ctx, allow_nonfinite)

    def sample(self):
        flbm_sample(self.ctx)

    def fetch_samples(self, max_n=None, allow_nonfinite=False):
        return flbm_fetch_samples(self.ctx, max_n, allow_nonfinite)

    def populations(self):
        return flbm_get_populations(self.ctx, self.lattice, self.dims)

    def set_populations(self, f):
        flbm_set_populations(self.ctx, f)

    def sites_populations(self, sites):
        return flbm_get_sites(self.ctx, self.lattice, sites)

    def save(self):
        return flbm_save(self.ctx)

    def load(self, blob):
        flbm_load(self.ctx, blob)

    def sync(self):
        flbm_sync(self.ctx)

    def autotune(self, trial_steps=10):
        return flbm_autotune(self.ctx, trial_steps)

    @property
    def collision(self):
        """FLBM_COLLISION_CM (the paper's scheme) or FLBM_COLLISION_RAW (raw moments)."""
        return flbm_get_collision(self.ctx)

    @collision.setter
    def collision(self, model):
        flbm_set_collision(self.ctx, model)

    @property
    def variant(self):
        return flbm_get_step_variant(self.ctx)

    @variant.setter
    def variant(self, v):
        flbm_set_step_variant(self.ctx, v)

    def close(self):
        if self.ctx:
            if self._owned:
                flbm_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns a batch of independent lattices (flbm_batch_*); ``lattice(i)`` gives a
    non-owning Lattice view of member i for the read and exchange calls."""

    def __init__(self, specs, cuda_stream=None):
        self.specs = [dict(d) for d in specs]
        self.handle = flbm_batch_create(self.specs, cuda_stream)
        self._views = [None] * len(self.specs)

    def __len__(self):
        return len(self.specs)

    def lattice(self, i):
        if not 0 <= int(i) < len(self.specs):
            flbm_batch_lattice(self.handle, i)  # raises FLBM_EINVAL with the library's message
        if self._views[i] is None:
            d = self.specs[i]
            self._views[i] = Lattice(d["lattice"], d["dims"], None, None,
                                     _borrowed=flbm_batch_lattice(self.handle, i))
        return self._views[i]

    def step(self, n=1):
        flbm_batch_step(self.handle, n)

    @property
    def step_count(self):
        return flbm_batch_get_step(self.handle)

    def stats(self, i, allow_nonfinite=False):
        """Statistics of member i (flbm_batch_stats)."""
        return flbm_batch_stats(self.handle, i, allow_nonfinite)

    @property
    def shape(self):
        """(threads per block, launch form)."""
        return flbm_batch_get_shape(self.handle)

    @shape.setter
    def shape(self, tf):
        flbm_batch_set_shape(self.handle, tf[0], tf[1])

    def type_shape(self, lattice):
        """(threads per block, launch form) of one lattice type as launched."""
        return flbm_batch_get_type_shape(self.handle, lattice)

    def set_type_shape(self, lattice, threads, form):
        flbm_batch_set_type_shape(self.handle, lattice, threads, form)

    def autotune(self, trial_steps=10):
        return flbm_batch_autotune(self.handle, trial_steps)

    @property
    def uses_graph(self):
        return flbm_batch_uses_graph(self.handle) == 1

    def sync(self):
        flbm_batch_sync(self.handle)

    def close(self):
        if self.handle:
            for v in self._views:
                if v is not None:
                    v.ctx = None
            flbm_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Domain:
    """Owns a domain (flbm_domain_*): one lattice split along z into slabs."""

    def __init__(self, lattice, dims, lam, kBT, rho0=1.0, seed=0, storage=FLBM_FP32, nslabs=2, devices=None):
        self.lattice = int(lattice)
        self.dims = tuple(int(x) for x in dims)
        self.handle = flbm_domain_create(lattice, self.dims, lam, kBT, rho0, seed, storage, nslabs, devices)

    def __len__(self):
        return flbm_domain_size(self.handle)

    def init_uniform(self, u0=(0.0, 0.0, 0.0), amp=0.0, perturb_seed=0):
        flbm_domain_init_uniform(self.handle, u0, amp, perturb_seed)

    def step(self, n=1):
        flbm_domain_step(self.handle, n)

    @property
    def step_count(self):
        return flbm_domain_get_step(self.handle)

    @property
    def variant(self):
        return flbm_get_step_variant(flbm_domain_slab(self.handle, 0))

    @variant.setter
    def variant(self, v):
        flbm_domain_set_step_variant(self.handle, v)

    def stats(self, allow_nonfinite=False):
        return flbm_domain_stats(self.handle, allow_nonfinite)

    def populations(self):
        return flbm_domain_get_populations(self.handle, self.lattice, self.dims)

    def set_populations(self, f):
        flbm_domain_set_populations(self.handle, f)

    def sync(self):
        flbm_domain_sync(self.handle)

    def close(self):
        if self.handle:
            flbm_domain_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
