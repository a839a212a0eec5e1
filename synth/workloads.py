"""The synthetic workloads (stand-ins for the paper's cosmological snapshots).

Physical parameters follow the paper's P3M defaults: PM grid n_phi = 2 cbrt(N)
(Eq. phi_gridsize_preference), x_s = 1.25 L_phi and x_r = 4.5 x_s
(Eq. p3m_parameters), softening eps = 0.03 L / cbrt(N) (Table tab:sim_params)
with the B-spline shape (eps_B = 2.8 eps) as default, unit box, G = 1 and
m = 1/N so that G m = 1/N.
"""
from __future__ import annotations

import dataclasses


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n_side: int            # N = n_side^3
    frac_uniform: float    # uniform fraction
    n_spheres: int         # number of Plummer spheres
    b_lo: float            # Plummer scale range (log-uniform); b_lo == b_hi: fixed
    b_hi: float
    seed: int
    n_sub: int = 2         # subtiles per tile per dimension
    description: str = ""

    @property
    def n(self) -> int:
        return self.n_side ** 3

    @property
    def n_phi(self) -> int:
        return 2 * self.n_side

    @property
    def x_s(self) -> float:
        return 1.25 / self.n_phi

    @property
    def x_r(self) -> float:
        return 4.5 * self.x_s

    @property
    def eps(self) -> float:
        return 0.03 / self.n_side

    @property
    def G_m(self) -> float:
        return 1.0 / self.n


WORKLOADS = {
    w.name: w
    for w in [
        Workload("n32k", 32, 0.5, 64, 0.01, 0.01, 1001,
                 description="N=32^3, 50% uniform + 50% in 64 Plummer spheres (b=0.01), PM grid 64^3"),
        Workload("n2m", 128, 0.3, 4096, 1e-3, 1e-2, 1002,
                 description="N=128^3, 30% uniform + 70% in 4096 Plummer spheres (b log-uniform 1e-3..1e-2), PM grid 256^3"),
        Workload("n134m", 512, 0.2, 2 ** 18, 2.5e-4, 2.5e-3, 1003,
                 description="N=512^3, 20% uniform + 80% in 2^18 Plummer spheres (b log-uniform 2.5e-4..2.5e-3), PM grid 1024^3, 8 rungs"),
        Workload("n2m_leapfrog", 128, 0.3, 4096, 1e-3, 1e-2, 1004,
                 description="N=128^3, clustered as the 128^3 set (30% uniform + 4096 spheres), 16-step leapfrog"),
        Workload("n1g", 1024, 0.1, 2 ** 22, 1e-4, 5e-3, 1005,
                 description="N=1024^3, 10% uniform + 90% in 2^22 Plummer spheres (b log-uniform 1e-4..5e-3), PM grid 2048^3"),
    ]
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]
