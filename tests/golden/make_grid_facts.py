"""Write the shortest dual edge of the oracle's R2B0..R2B8 grids.

    python tests/golden/make_grid_facts.py

The mixed-precision tolerances scale with the advective Courant number on the
shortest dual edge; the full-size R2B8 test reads the value from
grid_dual_edge_min.json instead of building the grid in the oracle (about a minute
and 11 GB). Runs only the oracle.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402


def main():
    out = {"source": "oracle grid builder, root 2 (make_grid_facts.py)", "d_e_min_m": {}}
    for bis in range(9):
        out["d_e_min_m"][str(bis)] = float(O.build_grid(2, bis).d_e.min())
    with open(os.path.join(HERE, "grid_dual_edge_min.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
