"""Run one dycore step on a small grid through the C ABI, for kernel profilers (ncu).

    python -m paper_2511_02021_gb300.profile_step BISECTIONS NLEV PRECISION [NSTEPS [NTRACERS [TOPO_M]]]

PRECISION 0 = FP64, 1 = mixed. Builds R2B<BISECTIONS> with NLEV levels, the jet
state with 0.1 K noise (over a Gaussian mountain of TOPO_M metres, radius 800 km,
when TOPO_M > 0), gives it NTRACERS (default 0) tracers, and advances NSTEPS
(default 1) steps of 180 s in 5 substeps.
"""
import sys

import paper_2511_02021_gb300 as P
from paper_2511_02021_gb300 import capi as C


def main(argv):
    bis, nlev, prec = int(argv[1]), int(argv[2]), int(argv[3])
    nsteps = int(argv[4]) if len(argv) > 4 else 1
    ntr = int(argv[5]) if len(argv) > 5 else 0
    topo = float(argv[6]) if len(argv) > 6 else 0.0
    import torch
    torch.cuda.set_device(0)
    P.use_torch_allocator(0)
    P.bind_torch_stream()
    g = C.icon_grid_build(2, bis, nlev)
    s = C.icon_state_init_ex(g, 2, C.ICON_CASE_JET, noise_K=0.1, precision=prec, topo_height_m=topo,
                             topo_radius_m=800e3 if topo > 0 else 0.0)
    if ntr:
        C.icon_state_add_tracers(s, ntr)
        import numpy as np
        xc = C.icon_grid_copy_table(g, "x_c")
        for t in range(ntr):
            C.icon_state_set_tracer(s, g, nlev, t, np.repeat(1.0 + 0.5 * xc[:, 2:3], nlev, axis=1))
    for _ in range(nsteps):
        C.icon_dycore_step(s, 180.0, 5)
    C.icon_state_free(s)
    C.icon_grid_free(g)
    print("ok")


if __name__ == "__main__":
    main(sys.argv)
