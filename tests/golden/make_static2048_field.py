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
    u* > 1e-6, and the start cell;
  * the Eq. 3 descent index (the 4-neighbour of largest u*, i.e. of smallest
    phi*, in the order +x, -x, +y, -y) at 4096 seeded random free cells where
    phi* > 0.99 (u* < 0.01) and the two largest neighbour values differ by
    more than twice the reference's own error bound tau_max * r* (so the
    reference decides the direction), with that margin; and how many free
    cells with phi* > 0.99 there are and how many of them are such near-ties.

Run from the repository root:  python tests/golden/make_static2048_field.py
(a few minutes on one core)."""
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
    # Eq. 3 descent index where phi* > 0.99, excluding the reference's near-ties
    bound = float(tau.max()) * r_inf
    flat = free[ustar[free[:, 0], free[:, 1]] < 0.01]
    ys, xs = flat[:, 0], flat[:, 1]
    nb = np.stack([ustar[ys, xs + 1], ustar[ys, xs - 1], ustar[ys + 1, xs], ustar[ys - 1, xs]], axis=1)
    order = np.argsort(-nb, axis=1, kind="stable")
    top = np.take_along_axis(nb, order[:, :2], axis=1)
    margin = top[:, 0] - top[:, 1]
    decided = margin > 2.0 * bound
    cand = np.flatnonzero(decided)
    dpick = cand[np.random.default_rng(2049).choice(len(cand), size=min(4096, len(cand)), replace=False)]
    out = {
        "scene": "static2048 (scenes.static2048())",
        "nx": sc.nx, "ny": sc.ny, "goal": list(sc.goal), "start": list(sc.start),
        "occupancy_sha256": hashlib.sha256(np.ascontiguousarray(occ).tobytes()).hexdigest(),
        "reference": "oracle.solve_field: FP64 conjugate gradients to r_inf <= 1e-12",
        "reference_resid_inf": r_inf,
        "tau_max": float(tau.max()),
        "cells": [[x, y] for x, y in cells],
        "u_star": [repr(float(ustar[y, x])) for x, y in cells],
        "descent": {
            "definition": "index of the 4-neighbour with the largest u* (order +x, -x, +y, -y) at free cells "
                          "with phi* > 0.99, where the two largest neighbour values differ by more than "
                          "2 tau_max r*",
            "free_cells_phi_above_0.99": int(len(flat)),
            "near_ties_excluded": int((~decided).sum()),
            "oracle_error_bound": bound,
            "cells": [[int(xs[i]), int(ys[i])] for i in dpick],
            "index": [int(order[i, 0]) for i in dpick],
            "margin": [repr(float(margin[i])) for i in dpick],
            "u_star": [repr(float(ustar[ys[i], xs[i]])) for i in dpick],
        },
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "static2048_field.json")
    with open(path, "w") as f:
        json.dump(out, f)
        f.write("\n")
    print(path, "tau_max", out["tau_max"], "r*", r_inf)


if __name__ == "__main__":
    main()
