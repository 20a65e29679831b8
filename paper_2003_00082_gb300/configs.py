"""Workload presets: the five synthetic cylinder-flow workloads the path is measured on.

Each preset names its mesh, velocity recipe, magnetic field, Stuart number,
tolerance and seeds.  The Stuart number N = sigma B_o^2 d / (rho u_inf)
(Eq. 24) with rho = d = u_inf = B_o = 1 (Sect. 3) gives sigma = N.
"""
from __future__ import annotations

from dataclasses import dataclass, field

from . import inputs


@dataclass(frozen=True)
class Workload:
    name: str
    n_theta: int
    n_r: int
    B: tuple = (0.0, 1.0, 1.0)
    stuart: float = 1.0
    tol: float = 1e-8
    seed: int = 0
    steps: int = 1
    vortices: bool = False
    noise_std: float = 0.0
    pressure: bool = False         # also run the pressure Poisson solve (Eq. 15)
    use_x0: bool = False           # previous-step solution as the initial guess
    rho_over_dt: float = 1.0 / inputs.DT
    inner_tol: float = 1e-4
    extra: dict = field(default_factory=dict)

    @property
    def sigma(self) -> float:
        return self.stuart

    @property
    def sizes(self):
        return inputs.ogrid_sizes(self.n_theta, self.n_r)


# Plain CGP potential step at 64x32 (fine ~8.3k nodes), FP64, tol 1e-10, x0 = 0.
# The literal in-plane B = (0, 1, 0) makes div(u x B) vanish in 2-D; the
# timed and parity runs add the B_o k-hat of Eq. 11 (B_o = 1): B = (0, 1, 1).
C1_SMALL = Workload("potential-64x32", 64, 32, B=(0.0, 1.0, 1.0), stuart=1.0, tol=1e-10,
                    seed=0, steps=1, vortices=False, noise_std=1e-3)
C1_LITERAL_B = (0.0, 1.0, 0.0)

# Potential + pressure CGP solves at 512x256 (fine 525,312 nodes), 200 steps of
# an advected vortex train, B = B_o k-hat, N = 1, tol 1e-8, previous-step x0.
C2_SCALE = Workload("potential+pressure-512x256", 512, 256, B=(0.0, 0.0, 1.0), stuart=1.0,
                    tol=1e-8, seed=1, steps=200, vortices=True, noise_std=0.0,
                    pressure=True, use_x0=True)

# Mixed precision on the 64x32 mesh over the 200-step vortex sequence with noise.
C3_MIXED = Workload("mixed-64x32", 64, 32, B=(0.0, 0.0, 1.0), stuart=1.0, tol=1e-8,
                    seed=0, steps=200, vortices=True, noise_std=1e-3, inner_tol=1e-4,
                    use_x0=True)

# Learned initial guess on the 64x32 mesh: train N in {0.5,1,2,5} x 5 seeds x 200
# steps; test N = 3 on seeds 100..104.
C4_LEARNED = Workload("learned-guess-64x32", 64, 32, B=(0.0, 0.0, 1.0), stuart=3.0, tol=1e-8,
                      seed=100, steps=200, vortices=True, noise_std=1e-3, use_x0=True,
                      extra=dict(train_stuart=(0.5, 1.0, 2.0, 5.0), train_seeds=(0, 1, 2, 3, 4),
                                 test_seeds=(100, 101, 102, 103, 104), hidden=64, layers=3))

# 64 uneven instances in one batched launch: n_theta ~ U{64,128,256,512},
# n_r = n_theta/2, N ~ U[0.5, 5], B a unit in-plane vector at a seeded angle
# plus B_o k-hat; FP32 inner PCG with FP64 refinement to 1e-8.
C5_BATCHED = Workload("batched-64-uneven", 0, 0, tol=1e-8, seed=7, steps=1, vortices=True,
                      inner_tol=1e-4, extra=dict(count=64, n_theta_choices=(64, 128, 256, 512),
                                                 stuart_range=(0.5, 5.0)))


def batched_instances(wl: Workload = C5_BATCHED):
    """Draw the per-instance (n_theta, n_r, stuart, B) of the batched workload."""
    import numpy as np
    rng = np.random.default_rng(wl.seed)
    count = wl.extra["count"]
    nth = rng.choice(np.array(wl.extra["n_theta_choices"]), size=count)
    lo, hi = wl.extra["stuart_range"]
    stuart = rng.uniform(lo, hi, size=count)
    ang = rng.uniform(0.0, 2.0 * np.pi, size=count)
    out = []
    for k in range(count):
        out.append(dict(n_theta=int(nth[k]), n_r=int(nth[k]) // 2, stuart=float(stuart[k]),
                        B=inputs.magnetic_field(angle=float(ang[k])), seed=wl.seed * 1000 + k))
    return out
