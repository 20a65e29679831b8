"""Seeded synthetic inputs shared by the CUDA path, its tests and the benchmark.

This module holds no arithmetic of the coarse-grid projection method itself:
it only builds the coarse O-grid mesh around the cylinder and evaluates a
prescribed velocity field at given points.  The fine mesh (the uniform 4-way
split, Sect. 2.3 / Eq. 18) is built independently by the library and by the
oracle; callers evaluate the velocity at whichever fine-node coordinates they
hold.

Mesh (stands in for the paper's Gmsh meshes, Sect. 3, which are not
available): an O-grid around a cylinder of diameter 1 centred at the origin,
outer radius 15, ``n_theta`` periodic nodes per ring and ``n_r`` cells in the
radial direction with geometric stretch ``q`` (default ``1.08 ** (32 / n_r)``,
the 1.08-per-cell stretch at ``n_r = 32`` refined consistently).  Node index
is ``j * n_theta + i`` for ring ``j`` in ``[0, n_r]`` and angle index ``i``.
Each quad is cut along its (i, j)-(i+1, j+1) diagonal; triangles are stored
counter-clockwise.

Velocity (stands in for the paper's flow data): potential flow past the
cylinder at free-stream ``U`` plus an optional train of Lamb-Oseen vortices
(core radius 0.3, circulation +-1 alternating) advected downstream at 0.8 U,
plus optional i.i.d. Gaussian noise per fine-node component.  A step's field
is a pure function of (step, seed), so runs restart from any step.
"""
from __future__ import annotations

import math

import numpy as np

R_IN = 0.5
R_OUT = 15.0
DT = 0.05          # time increment, Sect. 3
N_VORTICES = 7
VORTEX_CORE = 0.3
VORTEX_SPEED = 0.8


def radial_stretch(n_r: int) -> float:
    """Geometric growth factor per radial cell: 1.08 at n_r = 32, refined as 1.08**(32/n_r)."""
    return 1.08 ** (32.0 / n_r)


def ogrid(n_theta: int, n_r: int, q: float | None = None,
          r_in: float = R_IN, r_out: float = R_OUT):
    """Coarse O-grid: returns ``xy`` [(n_r+1)*n_theta, 2] float64 and ``tri`` [2*n_theta*n_r, 3] int32 (CCW)."""
    if n_theta < 3 or n_r < 1:
        raise ValueError("need n_theta >= 3 and n_r >= 1")
    if q is None:
        q = radial_stretch(n_r)
    j = np.arange(n_r + 1, dtype=np.float64)
    if abs(q - 1.0) < 1e-15:
        r = r_in + (r_out - r_in) * j / n_r
    else:
        dr0 = (r_out - r_in) * (q - 1.0) / (q ** n_r - 1.0)
        r = r_in + dr0 * (q ** j - 1.0) / (q - 1.0)
    r[-1] = r_out
    th = 2.0 * np.pi * np.arange(n_theta, dtype=np.float64) / n_theta
    xy = np.empty(((n_r + 1) * n_theta, 2), dtype=np.float64)
    xy[:, 0] = (r[:, None] * np.cos(th)[None, :]).ravel()
    xy[:, 1] = (r[:, None] * np.sin(th)[None, :]).ravel()

    jj, ii = np.meshgrid(np.arange(n_r), np.arange(n_theta), indexing="ij")
    ii = ii.ravel()
    jj = jj.ravel()
    i1 = (ii + 1) % n_theta
    n00 = jj * n_theta + ii
    n10 = jj * n_theta + i1
    n01 = (jj + 1) * n_theta + ii
    n11 = (jj + 1) * n_theta + i1
    t1 = np.stack([n00, n10, n11], axis=1)
    t2 = np.stack([n00, n11, n01], axis=1)
    tri = np.empty((2 * t1.shape[0], 3), dtype=np.int64)
    tri[0::2] = t1
    tri[1::2] = t2
    # orient counter-clockwise
    p0, p1, p2 = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    area2 = (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1])
    neg = area2 < 0
    tri[neg, 1], tri[neg, 2] = tri[neg, 2].copy(), tri[neg, 1].copy()
    return xy, tri.astype(np.int32)


def ogrid_sizes(n_theta: int, n_r: int):
    """Closed-form sizes of the coarse O-grid and its 4-way split (Euler characteristic 0)."""
    n_c = n_theta * (n_r + 1)
    t_c = 2 * n_theta * n_r
    e_c = n_c + t_c
    return dict(n_c=n_c, t_c=t_c, e_c=e_c, nnz=n_c + 2 * e_c, n_f=n_c + e_c, t_f=4 * t_c)


def potential_flow(xy: np.ndarray, U: float = 1.0, a: float = R_IN):
    """Irrotational flow past a cylinder of radius ``a`` at free stream ``U``."""
    x, y = xy[:, 0], xy[:, 1]
    r2 = x * x + y * y
    r4 = r2 * r2
    u = U * (1.0 - a * a * (x * x - y * y) / r4)
    v = -2.0 * U * a * a * x * y / r4
    return u, v


def vortex_centres(step: int, seed: int, U: float = 1.0):
    """Positions and circulations of the advected vortex train at time step ``step``."""
    rng = np.random.default_rng([seed, 0x5EED])
    jitter = rng.uniform(-0.1, 0.1, size=(N_VORTICES, 2))
    k = np.arange(N_VORTICES)
    xc = 1.0 + 2.0 * k + jitter[:, 0] + VORTEX_SPEED * U * step * DT
    yc = np.where(k % 2 == 0, 0.5, -0.5) + jitter[:, 1]
    gamma = np.where(k % 2 == 0, 1.0, -1.0)
    return xc, yc, gamma


def lamb_oseen(xy: np.ndarray, xc, yc, gamma, rc: float = VORTEX_CORE):
    """Sum of Lamb-Oseen vortex velocities u_theta = G/(2 pi rho) (1 - exp(-rho^2/rc^2))."""
    u = np.zeros(xy.shape[0])
    v = np.zeros(xy.shape[0])
    for x0, y0, g in zip(xc, yc, gamma):
        dx = xy[:, 0] - x0
        dy = xy[:, 1] - y0
        rho2 = dx * dx + dy * dy
        s = rho2 / (rc * rc)
        # (1 - exp(-s)) / rho^2, finite as rho -> 0
        with np.errstate(invalid="ignore", divide="ignore"):
            f = np.where(s > 1e-12, -np.expm1(-s) / np.where(rho2 > 0, rho2, 1.0), 1.0 / (rc * rc))
        c = g / (2.0 * math.pi) * f
        u += -c * dy
        v += c * dx
    return u, v


def velocity(xy: np.ndarray, step: int = 0, seed: int = 0, vortices: bool = True,
             noise_std: float = 0.0, U: float = 1.0):
    """Fine-node velocity (u, v) at time step ``step``: potential flow + vortex train + noise."""
    u, v = potential_flow(xy, U)
    if vortices:
        xc, yc, g = vortex_centres(step, seed, U)
        du, dv = lamb_oseen(xy, xc, yc, g)
        u = u + du
        v = v + dv
    if noise_std > 0.0:
        rng = np.random.default_rng([seed, step])
        noise = rng.standard_normal((2, xy.shape[0])) * noise_std
        u = u + noise[0]
        v = v + noise[1]
    return np.ascontiguousarray(u), np.ascontiguousarray(v)


def magnetic_field(angle: float | None = None, b_in_plane=(0.0, 0.0), bz: float = 1.0):
    """B = (Bx, By, Bz): the in-plane part given directly or as a unit vector at ``angle``."""
    if angle is not None:
        return (math.cos(angle), math.sin(angle), bz)
    return (float(b_in_plane[0]), float(b_in_plane[1]), bz)
