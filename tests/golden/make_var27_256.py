"""Writes var27_256_oracle.json: the oracle's results on the full-size
256^3 27-point variable-coefficient workload (problems.config(2)), sampled so
that the fixture stays small.

Calls only the oracle (oracle/ssamg.py) and the input generators
(problems/).  Contents:

* levels 0-4 of the hierarchy (Sections 3.1-3.3): cell count, coarsening
  direction, the largest |coefficient| of the level, and at 256 sampled
  cells (plus the eight corners of the box) all 27 stencil entries in
  offset-code order ((ox+1) + 3 (oy+1) + 9 (oz+1)), the smoother diagonal
  omega M^-1 (Eq. relax0/relax1) and, for levels 0-3, the interpolation
  weights PW, PE (Eq. prolEx; zero at coarse points);
* PCG with one V(1,1) cycle per iteration (Section 4) from x0 = 0 to
  ||r|| <= 1e-8 ||b||: iteration count, recursive and true relative
  residuals, ||x||_2, and x at 2,048 sampled cells.

Runs for tens of minutes on one host core and needs ~20 GB of memory:

    python tests/golden/make_var27_256.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import problems as P  # noqa: E402
from oracle import ssamg as O  # noqa: E402

OUT = os.path.join(HERE, "var27_256_oracle.json")
NLEV = 5
NSAMPLE = 256
NX = 2048


def code_of(o):
    return (o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1)


def sample_cells(n, shape, gen):
    nz, ny, nx = shape
    corners = [((k * (nz - 1)) * ny + j * (ny - 1)) * nx + i * (nx - 1)
               for k in (0, 1) for j in (0, 1) for i in (0, 1)]
    cells = np.concatenate([np.array(corners, np.int64), gen.int_range(NSAMPLE, 0, n - 1)])
    return np.unique(cells)


def main():
    t0 = time.time()
    prob = P.config(2)
    h = O.setup(prob)
    print(f"setup {time.time() - t0:.0f} s, {len(h.levels)} levels", flush=True)
    gen = P.SplitMix64(41)
    levels = []
    for l in range(NLEV):
        lev = h.levels[l]
        shp = lev.shape(0)
        cells = sample_cells(lev.n, shp, gen)
        coef = np.zeros((len(cells), 27))
        cmax = 0.0
        for o, a in lev.S[0].items():
            flat = np.asarray(a).reshape(-1)
            coef[:, code_of(o)] = flat[cells]
            cmax = max(cmax, float(np.abs(flat).max()))
        row = {"level": l, "ncells": lev.n, "shape_zyx": list(shp), "dstar": int(lev.dstar[0]),
               "coef_max": cmax, "cells": cells.tolist(), "coef": coef.tolist(),
               "dinv": lev.Dinv[cells].tolist()}
        if l + 1 < len(h.levels) and lev.dstar[0] >= 0:
            row["PW"] = np.asarray(lev.PW[0]).reshape(-1)[cells].tolist()
            row["PE"] = np.asarray(lev.PE[0]).reshape(-1)[cells].tolist()
        levels.append(row)
    t1 = time.time()
    res = O.pcg(h, prob.b[0], tol=1e-8, max_iter=500)
    print(f"pcg {time.time() - t1:.0f} s, {res.iterations} iterations", flush=True)
    xs = gen.int_range(NX, 0, prob.n - 1)
    out = {
        "what": "oracle results on problems.config(2) (1 part 256^3, 27-point variable "
                "coefficients, seed 2), sampled; written by tests/golden/make_var27_256.py",
        "passages": "Sections 3.1-3.4 (hierarchy, smoother), Section 4 (PCG + V(1,1) cycle)",
        "num_levels": len(h.levels),
        "levels": levels,
        "pcg": {"tol": 1e-8, "iterations": res.iterations, "rel_res": res.rel_res,
                "true_rel_res": res.true_rel_res, "x_norm": float(np.linalg.norm(res.x)),
                "cells": xs.tolist(), "x": res.x[xs].tolist()},
    }
    with open(OUT, "w") as f:
        json.dump(out, f)
    print(f"wrote {OUT} ({os.path.getsize(OUT)} bytes) in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
