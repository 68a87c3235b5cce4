"""Write sampled oracle outputs of one full-size FP64 dycore step.

    python tests/golden/make_step_samples.py

Runs the oracle (and nothing else) on the R2B6 grid with 90 levels, the balanced jet
with its 1 m/s wind bump and no theta_v noise (seed 1), one step of dt = 90 s in 5
substeps: the workload the throughput benchmark times. It stores, for a fixed random
sample of cells and edges, every level of every prognostic field, of the two
step-mean mass fluxes and of one tracer (q0 = 1 + z/2 with z the unit-sphere height
of the cell centre) transported with them, plus the L2 norm of each full field, in
r2b6_l90_jet_step_samples.json. The oracle needs about four minutes and 14 GB here.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402

BIS, NLEV, CASE, SEED, NOISE, DT, NSUB = 6, 90, 2, 1, 0.0, 90.0, 5
N_SAMPLE = 24
SAMPLE_SEED = 20251103


def main():
    g = O.build_grid(2, BIS)
    v = O.vertical_grid(NLEV)
    s0 = O.init_state(g, v, SEED, CASE, noise_K=NOISE)
    m0 = O.global_mass(g, v, s0)
    s1, acc = O.dycore_step(g, v, s0, DT, NSUB)
    out = dict(s1, **acc)
    m1 = O.global_mass(g, v, s1)
    # one tracer, q0 = 1 + z/2 (unit-sphere z of the cell centre) at every level,
    # transported with the step's mean fluxes
    q0 = np.repeat(1.0 + 0.5 * g.x_c[:, 2:3], NLEV, axis=1)
    out["tracer"] = O.tracer_step(g, v, q0, s0["rho"], s1["rho"], acc["mflx"], acc["wflx"], DT)
    nc, ne = s0["rho"].shape[0], s0["vn"].shape[0]
    rng = np.random.default_rng(SAMPLE_SEED)
    cells = sorted(set([0, nc - 1] + rng.choice(nc, N_SAMPLE, replace=False).tolist()))
    edges = sorted(set([0, ne - 1] + rng.choice(ne, N_SAMPLE, replace=False).tolist()))
    doc = {
        "source": "oracle one dycore step (make_step_samples.py)",
        "config": {"root": 2, "bisections": BIS, "nlev": NLEV, "case": CASE, "seed": SEED, "noise_K": NOISE,
                   "dt": DT, "nsub": NSUB},
        "cells": cells, "edges": edges,
        "mass": [m0, m1],
        "init": {}, "step": {}, "norm_init": {}, "norm_step": {},
    }
    for f in ("vn", "rho", "theta_v", "exner"):
        idx = edges if f == "vn" else cells
        doc["init"][f] = [[float(x) for x in s0[f][i]] for i in idx]
        doc["norm_init"][f] = float(np.linalg.norm(s0[f]))
    for f in ("vn", "w", "rho", "theta_v", "exner", "mflx", "wflx", "tracer"):
        idx = edges if f in ("vn", "mflx") else cells
        doc["step"][f] = [[float(x) for x in out[f][i]] for i in idx]
        doc["norm_step"][f] = float(np.linalg.norm(out[f]))
    with open(os.path.join(HERE, "r2b6_l90_jet_step_samples.json"), "w") as fh:
        json.dump(doc, fh)


if __name__ == "__main__":
    main()
