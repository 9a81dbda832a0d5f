"""FP64 CPU oracle of the fluctuating central-moment LBM step (arXiv:2602.16486).

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package. The product
path (``paper_2602_16486_gb300``) never imports it and shares no code with it.

This module is argument marshalling (numpy <-> ctypes) around ``flbm_oracle.cpp``;
every piece of arithmetic lives in that file, which cites the paper section by
section. ``build()`` compiles it with g++ (FP64, no fast-math, no FMA contraction).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flbm_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

D2Q9 = 0
D3Q27 = 1
D3Q27_ISO = 2  # D3Q27 with trace/deviator normal-stress modes (flbm_oracle.cpp)
D3Q19 = 3
_Q = {D2Q9: 9, D3Q27: 27, D3Q27_ISO: 27, D3Q19: 19}
_D = {D2Q9: 2, D3Q27: 3, D3Q27_ISO: 3, D3Q19: 3}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (skipped if up to date)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    i64p = ctypes.POINTER(ctypes.c_int64)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_q.argtypes = [ctypes.c_int]
    lib.oracle_q.restype = ctypes.c_int
    lib.oracle_tables.argtypes = [ctypes.c_int, ip, dp, dp]
    lib.oracle_basis.argtypes = [ctypes.c_int, ctypes.c_int, dp]
    lib.oracle_basis.restype = ctypes.c_double
    lib.oracle_T.argtypes = [ctypes.c_int, dp, dp]
    lib.oracle_hermite.argtypes = [ip, ip, ctypes.c_int]
    lib.oracle_hermite.restype = ctypes.c_double
    lib.oracle_feq.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
    lib.oracle_philox.argtypes = [u32p, u32p, u32p]
    lib.oracle_uniform.argtypes = [ctypes.c_uint32]
    lib.oracle_uniform.restype = ctypes.c_double
    lib.oracle_normals_block.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                         ctypes.c_uint32, ctypes.c_uint32, dp]
    lib.oracle_site_eta.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_uint32, dp]
    lib.oracle_collide_site.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, dp, dp, dp]
    lib.oracle_collide_site.restype = ctypes.c_int
    lib.oracle_init_uniform.argtypes = [ctypes.c_int, i64p, ctypes.c_double, dp, ctypes.c_double,
                                        ctypes.c_uint64, dp]
    lib.oracle_run.argtypes = [ctypes.c_int, i64p, dp, ctypes.c_double, ctypes.c_uint64,
                               ctypes.c_uint64, ctypes.c_int64, dp, ctypes.c_int]
    lib.oracle_run.restype = ctypes.c_int64
    lib.oracle_stats.argtypes = [ctypes.c_int, i64p, dp, dp]
    lib.oracle_collide_site_model.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double, dp, dp, dp]
    lib.oracle_collide_site_model.restype = ctypes.c_int
    lib.oracle_run_model.argtypes = [ctypes.c_int, ctypes.c_int, i64p, dp, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.c_uint64, ctypes.c_int64, dp, ctypes.c_int]
    lib.oracle_run_model.restype = ctypes.c_int64
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _dims(lat, dims):
    d = [int(x) for x in dims] + [1] * (3 - len(dims))
    if lat == D2Q9 and d[2] != 1:
        raise ValueError("D2Q9 needs nz == 1")
    return np.array(d, dtype=np.int64)


def Q(lat):
    return _Q[lat]


def D(lat):
    return _D[lat]


def tables(lat):
    """Return (c[Q,3] int, w[Q], b[Q]) with b_v = sum_i w_i M_vi^2 computed in FP64."""
    lib = _load()
    q = _Q[lat]
    c = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    b = np.zeros(q)
    lib.oracle_tables(lat, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w), _dp(b))
    return c, w, b


def basis(lat, v, cbar):
    cb = _f64(list(cbar) + [0.0] * (3 - len(cbar)), 3)
    return _load().oracle_basis(lat, int(v), _dp(cb))


def T(lat, u):
    q = _Q[lat]
    uu = _f64(list(u) + [0.0] * (3 - len(u)), 3)
    out = np.zeros((q, q))
    _load().oracle_T(lat, _dp(uu), _dp(out))
    return out


def hermite(c, idx):
    ci = np.ascontiguousarray(np.asarray(list(c) + [0] * (3 - len(c)), dtype=np.int32))
    ii = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    ip = ctypes.POINTER(ctypes.c_int)
    return _load().oracle_hermite(ci.ctypes.data_as(ip), ii.ctypes.data_as(ip), len(idx))


def feq(lat, rho, u):
    q = _Q[lat]
    uu = _f64(list(u) + [0.0] * (3 - len(u)), 3)
    out = np.zeros(q)
    _load().oracle_feq(lat, float(rho), _dp(uu), _dp(out))
    return out


def philox(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    up = ctypes.POINTER(ctypes.c_uint32)
    _load().oracle_philox(c.ctypes.data_as(up), k.ctypes.data_as(up), out.ctypes.data_as(up))
    return out


def uniform(w):
    return _load().oracle_uniform(int(w) & 0xFFFFFFFF)


def normals_block(seed, step, site, tag, blk):
    z = np.zeros(4)
    _load().oracle_normals_block(int(seed), int(step), int(site), int(tag), int(blk), _dp(z))
    return z


def site_eta(lat, seed, step, site):
    eta = np.zeros(_Q[lat])
    _load().oracle_site_eta(lat, int(seed), int(step), int(site), _dp(eta))
    return eta


CM = 0   # collision models: central moments (the paper's scheme)
RAW = 1  # raw moments (T = M); with a uniform rate, fluctuating BGK


def collide_site(lat, f, lam, kBT, eta, model=CM):
    """Return (f_star[Q], k_pre[Q]) for one site with given normals eta[Q]; k_pre are the
    pre-collision moments of the model's basis (central for CM, raw for RAW)."""
    q = _Q[lat]
    f = _f64(f, q)
    lam = _f64(lam, q)
    eta = _f64(eta, q)
    fs = np.zeros(q)
    k = np.zeros(q)
    rc = _load().oracle_collide_site_model(lat, int(model), _dp(f), _dp(lam), float(kBT), _dp(eta), _dp(fs),
                                           _dp(k))
    if rc != 0:
        raise FloatingPointError("singular collision matrix")
    return fs, k


def init_uniform(lat, dims, rho0, u0=(0.0, 0.0, 0.0), amp=0.0, perturb_seed=0):
    """Equilibrium state f[Q, nz, ny, nx] at rho0 (optionally perturbed) and velocity u0."""
    d = _dims(lat, dims)
    q = _Q[lat]
    f = np.zeros((q, d[2], d[1], d[0]))
    uu = _f64(list(u0) + [0.0] * (3 - len(u0)), 3)
    _load().oracle_init_uniform(lat, d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                float(rho0), _dp(uu), float(amp), int(perturb_seed), _dp(f))
    return f


def run(lat, dims, lam, kBT, seed, f, step0=0, nsteps=1, threads=0, model=CM):
    """Advance a copy of f[Q, nz, ny, nx] by nsteps steps; returns the new state."""
    d = _dims(lat, dims)
    q = _Q[lat]
    g = np.array(f, dtype=np.float64, copy=True, order="C")
    if g.size != q * int(np.prod(d)):
        raise ValueError("population array has the wrong size")
    lam = _f64(lam, q)
    bad = _load().oracle_run_model(lat, int(model), d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(lam),
                                   float(kBT), int(seed), int(step0), int(nsteps), _dp(g), int(threads))
    if bad:
        raise FloatingPointError(f"{bad} singular collision matrices")
    return g.reshape(q, d[2], d[1], d[0])


def stats(lat, dims, f):
    """Statistics of a state (pre-collision): dict of FP64 arrays (see oracle_stats)."""
    d = _dims(lat, dims)
    q = _Q[lat]
    g = _f64(f, q * int(np.prod(d)))
    out = np.zeros(13 + q + q * q + 1)
    _load().oracle_stats(lat, d.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(g), _dp(out))
    return {
        "mass": out[0],
        "mom": out[1:4].copy(),
        "u_mean": out[4:7].copy(),
        "uu": out[7:13].copy(),
        "k_mean": out[13:13 + q].copy(),
        "k_cov": out[13 + q:13 + q + q * q].reshape(q, q).copy(),
        "nonfinite": int(out[13 + q + q * q]),
        "sites": int(np.prod(d)),
    }
