"""Workload table: grid sizes, time steps and initial states of the benchmark and
parity configurations (no arithmetic of the method lives here).

The paper's own runs start from reanalysis and spun-up states on the 10 km (R2B8)
and 1.25 km (R2B11) grids with 90 levels (Table 2); these synthetic analytic
states on the same grid family stand in for them.
"""
from dataclasses import dataclass


@dataclass(frozen=True)
class Workload:
    name: str
    bisections: int          # R2B<bisections>
    nlev: int
    case: int                # 0 rest, 1 solid-body rotation, 2 jet + bump, 3 ensemble member
    seed: int
    noise_K: float           # theta_v noise amplitude (K); <0 selects the case default
    dt: float                # s, one dycore step
    nsub: int                # substeps per step
    nsteps: int
    precision: int           # 0 FP64, 1 mixed

    @property
    def cells(self):
        return 20 * 4 ** (self.bisections + 1)


R2B2_SBR = Workload("R2B2-L20-sbr-fp64", 2, 20, 1, 1, 0.01, 300.0, 5, 1, 0)
R2B6_JET = Workload("R2B6-L90-jet-fp64", 6, 90, 2, 1, 0.0, 90.0, 5, 10, 0)
R2B8_JET_MIXED = Workload("R2B8-L90-jet-mixed", 8, 90, 2, 2, 0.1, 22.5, 5, 5, 1)
R2B9_JET_MIXED = Workload("R2B9-L60-jet-mixed", 9, 60, 2, 4, 0.1, 11.0, 5, 3, 1)
# batched ensemble: 32 members on R2B4 (dt 360 s) and 32 on R2B5 (dt 180 s), 60 levels
ENSEMBLE = {"members_b4": 32, "members_b5": 32, "nlev": 60, "seed": 3, "dt_b4": 360.0, "dt_b5": 180.0,
            "nsub": 5, "nsteps": 20, "precision": 1}
