"""Write sampled oracle outputs of one full-size FP64 dycore step on terrain-following levels.

    python tests/golden/make_terrain_samples.py

Runs the oracle (and nothing else) on the R2B6 grid with 90 levels over the Gaussian
mountain of the throughput benchmark's terrain variant (1500 m, e-folding radius 800 km,
at 90E 30N), the balanced jet with its 1 m/s wind bump and no theta_v noise (seed 1), one
step of dt = 90 s in 5 substeps. It stores, for a fixed random sample of cells and edges
(half of them on the mountain's slopes), every level of every prognostic field and of the
two step-mean mass fluxes, plus the L2 norm of each full field and the air mass, in
r2b6_l90_jet_terrain_step_samples.json. The oracle needs about six minutes and 20 GB here.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import oracle.terrain as T  # noqa: E402

BIS, NLEV, CASE, SEED, NOISE, DT, NSUB = 6, 90, 2, 1, 0.0, 90.0, 5
H0, RADIUS = 1500.0, 800e3
N_SAMPLE = 12
SAMPLE_SEED = 20251204


def main():
    g = O.build_grid(2, BIS)
    v = O.vertical_grid(NLEV)
    t = T.terrain_geometry(g, v, T.mountain(g.x_c, H0, RADIUS))
    s0 = O.init_state(g, v, SEED, CASE, noise_K=NOISE, terrain=t)
    m0 = T.terrain_mass(g, t, s0)
    s1, acc = T.terrain_step(g, v, t, s0, DT, NSUB)
    out = dict(s1, **acc)
    m1 = T.terrain_mass(g, t, s1)
    nc, ne = s0["rho"].shape[0], s0["vn"].shape[0]
    rng = np.random.default_rng(SAMPLE_SEED)
    hs_e = T.mountain(g.x_e, H0, RADIUS)
    slope_c = np.nonzero((t.hs > 0.2 * H0) & (t.hs < 0.8 * H0))[0]
    slope_e = np.nonzero((hs_e > 0.2 * H0) & (hs_e < 0.8 * H0))[0]
    cells = sorted(set([0, nc - 1] + rng.choice(nc, N_SAMPLE, replace=False).tolist()
                       + rng.choice(slope_c, N_SAMPLE, replace=False).tolist()))
    edges = sorted(set([0, ne - 1] + rng.choice(ne, N_SAMPLE, replace=False).tolist()
                       + rng.choice(slope_e, N_SAMPLE, replace=False).tolist()))
    doc = {
        "source": "oracle one dycore step on terrain-following levels (make_terrain_samples.py)",
        "config": {"root": 2, "bisections": BIS, "nlev": NLEV, "case": CASE, "seed": SEED, "noise_K": NOISE,
                   "dt": DT, "nsub": NSUB, "topo_height_m": H0, "topo_radius_m": RADIUS},
        "cells": cells, "edges": edges,
        "mass": [m0, m1],
        "init": {}, "step": {}, "norm_init": {}, "norm_step": {},
    }
    for f in ("vn", "rho", "theta_v", "exner"):
        idx = edges if f == "vn" else cells
        doc["init"][f] = [[float(x) for x in s0[f][i]] for i in idx]
        doc["norm_init"][f] = float(np.linalg.norm(s0[f]))
    for f in ("vn", "w", "rho", "theta_v", "exner", "mflx", "wflx"):
        idx = edges if f in ("vn", "mflx") else cells
        doc["step"][f] = [[float(x) for x in out[f][i]] for i in idx]
        doc["norm_step"][f] = float(np.linalg.norm(out[f]))
    with open(os.path.join(HERE, "r2b6_l90_jet_terrain_step_samples.json"), "w") as fh:
        json.dump(doc, fh)


if __name__ == "__main__":
    main()
