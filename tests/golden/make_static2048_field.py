"""Writes static2048_field.json: the FP64 reference of the 2048 x 2048 measured
workload, for the accuracy figures bench.py reports next to its timings.

Calls only the oracle (and the seeded scene generator for the inputs):
  * the occupancy raster (oracle.build_grid) and its SHA-256, which pins the
    scene the numbers belong to;
  * u* = the harmonic field (Sec. 3.1, Eq. 1 fixed point) by FP64 conjugate
    gradients to a residual of 1e-12, and its residual;
  * the exit time tau (the expected number of Eq. 1 random-walk steps to a
    fixed cell, (I - J) tau = 1 on free cells), whose maximum turns a residual
    r into the a-posteriori error bound |u - u*| <= tau_max * r;
  * u* at 2048 seeded random free cells, 2048 seeded random free cells where
    u* > 1e-6, and the start cell.

Run from the repository root:  python tests/golden/make_static2048_field.py
(about two minutes on one core)."""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import scenes  # noqa: E402


def main():
    sc = scenes.static2048()
    occ, _, _ = oracle.build_grid(sc)
    ustar, fixed = oracle.solve_field(occ, sc.goal, tol=1e-12)
    r_inf = float(oracle.residual(ustar, fixed)[0])
    tau = oracle.exit_time(fixed, tol=1e-6)
    free = np.argwhere(np.asarray(fixed) == 0)
    rng = np.random.default_rng(2048)
    # most of this cluttered field is below 1e-8 (the potential decays
    # exponentially away from the goal): half the samples uniform over the free
    # cells, half over the free cells where u* > 1e-6
    live = free[ustar[free[:, 0], free[:, 1]] > 1e-6]
    pick = np.concatenate([free[rng.choice(len(free), size=2048, replace=False)],
                           live[rng.choice(len(live), size=min(2048, len(live)), replace=False)]])
    cells = [(int(sc.start[0]), int(sc.start[1]))] + [(int(x), int(y)) for y, x in pick]
    out = {
        "scene": "static2048 (scenes.static2048())",
        "nx": sc.nx, "ny": sc.ny, "goal": list(sc.goal), "start": list(sc.start),
        "occupancy_sha256": hashlib.sha256(np.ascontiguousarray(occ).tobytes()).hexdigest(),
        "reference": "oracle.solve_field: FP64 conjugate gradients to r_inf <= 1e-12",
        "reference_resid_inf": r_inf,
        "tau_max": float(tau.max()),
        "cells": [[x, y] for x, y in cells],
        "u_star": [repr(float(ustar[y, x])) for x, y in cells],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "static2048_field.json")
    with open(path, "w") as f:
        json.dump(out, f)
        f.write("\n")
    print(path, "tau_max", out["tau_max"], "r*", r_inf)


if __name__ == "__main__":
    main()
