"""Writes precision_d3q27_32cube.json: FP64 oracle statistics of the D3Q27 32^3 replica
of the 256^3 storage-precision workload (rho0 = 1 at rest, Lambda_shear = 1.6, every
other non-conserved mode at rate 1; kBT 1e-5 and 1e-4; seed 7). Calls only the oracle.

    python tests/oracle_ref/make_precision_ref.py [--threads N]
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402

DIMS = (32, 32, 32)
OMEGA = 1.6
SEED = 7
KBTS = (1e-5, 1e-4)
FIRST, LAST, EVERY = 100, 400, 10
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "precision_d3q27_32cube.json")


def lam():
    v = np.ones(27)
    v[[7, 8, 9]] = OMEGA
    return v


def series(kbt, threads):
    f = oracle.init_uniform(1, DIMS, 1.0)
    step, out = 0, []
    while step <= LAST:
        if step >= FIRST:
            s = oracle.stats(1, DIMS, f)
            out.append({"step": step, "uu": s["uu"].tolist(), "u_mean": s["u_mean"].tolist(),
                        "kk": np.diag(s["k_cov"]).tolist()})
        if step == LAST:
            break
        n = EVERY if step >= FIRST else FIRST
        f = oracle.run(1, DIMS, lam(), kbt, SEED, f, step, n, threads)
        step += n
    return out


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--threads", type=int, default=0)
    a = p.parse_args()
    ref = {"lattice": "D3Q27", "dims": list(DIMS), "rho0": 1.0, "omega_shear": OMEGA, "seed": SEED,
           "first": FIRST, "last": LAST, "every": EVERY, "series": {}}
    for kbt in KBTS:
        ref["series"][repr(kbt)] = series(kbt, a.threads)
        print(f"kBT {kbt}: {len(ref['series'][repr(kbt)])} samples", flush=True)
    with open(OUT, "w") as fh:
        json.dump(ref, fh, indent=0)


if __name__ == "__main__":
    main()
