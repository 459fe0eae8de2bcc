"""Write the oracle's per-pair results for the full-size workloads to
``tests/golden/oracle_<workload>.npz``.

Calls only ``oracle`` (the plain FP64 CPU implementation) and the seeded input
generator ``paper_2011_07209_gb300.synth``; nothing here touches the CUDA
path.  The oracle runs at CG tolerance 1e-13 (the "discrete truth": the
discrete equations of the method solved far below the 1e-9 the workloads ask
for), so that the GPU's error against it is the GPU's own.

Each file holds, for one cell:
  rows      int16 [n_pairs][8]  (i, j, k0, k1, k2, g0, g1, g2), the unique pair list
  pair_e    float64 [n_pairs]   int_PE rho v of each pair
  pair_sig  float64 [n_pairs][3][3]  the pair's stress integrand (Eq. sxx_working, before w and the sum)
  pair_ncg  int32 [n_pairs]     oracle CG iterations
  e_xx, dedh, stress            cell totals (Eqs. exxGen_mlwf, sxx_working, pixx_working)
  lattice, lattice0, n, r_pair, r_pe, r_me, tol, n_aux, n_stcl
  centres_sha256, oracle_sha256  fingerprints of the inputs and of the oracle source

Usage:  python tests/golden/make_oracle_golden.py [workload ...]
(workloads: water64 triclinic128 batch3 traj256_s0 traj256_s1; default all).
Run time on 8 host cores: about 4 hours for all of them.
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2011_07209_gb300 import synth  # noqa: E402

TRUTH_TOL = 1e-13
TRAJ_SEED = synth.SEED_BASE + 500


def sha(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def oracle_sha() -> str:
    with open(os.path.join(ROOT, "oracle", "exx_oracle.c"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def cells(name: str):
    """(file stem, MLWF set, R_pair, R_PE, R_ME, lattice0 or None) of one workload."""
    if name == "water64":
        c = synth.CONFIGS[2]
        return [("water64", synth.make_config(2), c["r_pair"], c["r_pe"], c["r_me"], None)]
    if name == "triclinic128":
        c = synth.CONFIGS[3]
        return [("triclinic128", synth.make_config(3), c["r_pair"], c["r_pe"], c["r_me"], None)]
    if name == "batch3":
        return [(f"batch3_{k}", ws, 8.0, r_pe, 8.0, None) for k, (nm, ws, r_pe) in enumerate(synth.make_batch(4))]
    if name in ("traj256_s0", "traj256_s1"):
        c = synth.CONFIGS[5]
        ws0 = synth.make_config(5)
        step = int(name[-1])
        steps = synth.trajectory(ws0, step + 1, seed=TRAJ_SEED)
        lat0 = ws0.lattice if step > 0 else None
        return [(name, steps[step], c["r_pair"], c["r_pe"], c["r_me"], lat0)]
    raise ValueError(name)


def run(name: str) -> None:
    for stem, ws, r_pair, r_pe, r_me, lat0 in cells(name):
        t = time.time()
        p = oracle.make_params(r_pair=r_pair, r_pe=r_pe, r_me=r_me, tol=TRUTH_TOL, lattice0=lat0)
        o = oracle.exx(ws, p, want_d=False)
        out = os.path.join(HERE, f"oracle_{stem}.npz")
        np.savez_compressed(
            out, rows=o["pairs"].astype(np.int16), pair_e=o["pair_e"], pair_sig=o["pair_sig"],
            pair_ncg=o["pair_ncg"].astype(np.int32), e_xx=o["e_xx"], dedh=o["dedh"], stress=o["stress"],
            lattice=ws.lattice, lattice0=ws.lattice if lat0 is None else lat0, n=np.asarray(ws.n),
            r_pair=r_pair, r_pe=r_pe, r_me=r_me, tol=TRUTH_TOL, n_aux=o["n_aux"], n_stcl=o["n_stcl"],
            centres_sha256=sha(ws.centres), oracle_sha256=oracle_sha())
        print(f"{stem}: {len(o['pairs'])} pairs, E_xx = {o['e_xx']:.15e}, {time.time() - t:.0f} s", flush=True)


if __name__ == "__main__":
    names = sys.argv[1:] or ["water64", "triclinic128", "batch3", "traj256_s0", "traj256_s1"]
    for nm in names:
        run(nm)
