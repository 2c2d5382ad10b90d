"""Seeded synthetic inputs: solid masks, initial fluid densities and wall-angle fields.

This module holds geometry only -- no step of the lattice Boltzmann method.  Both the
CUDA path and the FP64 oracle read the arrays it returns, so the two sides see the same
inputs without sharing any of the method's arithmetic.

Every workload follows a test case of arXiv:2102.04709 Section III:

* ``janus_flat``      -- Section III.A (Janus droplet resting on a flat wall)
* ``janus_cylinder``  -- Section III.B (perfect Janus droplet deposited on a cylinder)
* ``capillary``       -- Section III.C (capillary intrusion of ternary fluids)
* ``pillars``         -- Section III.D (compound droplet passing through pillars)

Fluid indices 0, 1, 2 are the paper's red, green, blue.  Angle triples are
(theta_01, theta_20, theta_12) = (theta_rg, theta_br, theta_gb) in degrees, the three
angles of Eq.(17); theta_kl is measured inside fluid k.

Boundary codes (``bc_x``): 0 periodic, 1 modified periodic (labels 0 and 2 swap across the
x seam, Section III.C), 2 Zou-He velocity inlet / pressure outlet (Section III.D),
3 solid walls.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BC_PERIODIC, BC_MODPER, BC_ZOUHE, BC_WALLS = 0, 1, 2, 3


@dataclasses.dataclass
class Workload:
    """One synthetic problem: grid, geometry, material parameters and initial state."""

    name: str
    nx: int
    ny: int
    periodic_y: int
    bc_x: int
    solid: np.ndarray          # uint8 [ny, nx], 1 = solid
    rho: np.ndarray            # float64 [3, ny, nx], initial rho_k (0 at solid nodes)
    angles: np.ndarray         # float64 [ny, nx, 3], read at solid boundary nodes only
    sigma: tuple               # (sigma_01, sigma_02, sigma_12)
    nu: tuple                  # kinematic viscosity of each pure fluid
    beta0: float = 0.7
    u_in: float = 0.0
    rho_out: float = 1.0
    steps: int = 1000
    note: str = ""

    @property
    def n(self) -> int:
        return self.nx * self.ny

    def young_residual(self) -> float:
        """sigma_rg cos(theta_rg) + sigma_br cos(theta_br) + sigma_gb cos(theta_gb), Eq.(18),
        largest magnitude over the wall angles in use."""
        s01, s02, s12 = self.sigma
        a = np.deg2rad(self.angles[self.solid.astype(bool)])
        if a.size == 0:
            return 0.0
        r = s01 * np.cos(a[:, 0]) + s02 * np.cos(a[:, 1]) + s12 * np.cos(a[:, 2])
        return float(np.max(np.abs(r)))


# ----------------------------------------------------------------------------------------
# SplitMix64 (Steele, Lea, Flood 2014): the seeded generator used for pillar layouts
# ----------------------------------------------------------------------------------------
class SplitMix64:
    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


def _grid(nx, ny):
    y, x = np.mgrid[0:ny, 0:nx]
    return x.astype(np.float64), y.astype(np.float64)


def _uniform_angles(nx, ny, triple):
    a = np.empty((ny, nx, 3), dtype=np.float64)
    a[...] = np.asarray(triple, dtype=np.float64)
    return a


def _fill(labels, solid):
    """labels int [ny, nx] in {0,1,2} -> rho [3, ny, nx] with pure fluids, 0 in solids."""
    rho = np.zeros((3,) + labels.shape, dtype=np.float64)
    for k in range(3):
        rho[k][labels == k] = 1.0
    rho[:, solid.astype(bool)] = 0.0
    return rho


def janus_flat(nx=128, ny=64, R=20.0, triple=(90.0, 60.0, 120.0), sigma=(0.01, 0.01, 0.01),
               nu=(1.0 / 6.0,) * 3, steps=1000, name=None):
    """Section III.A: two half-discs (fluid 0 left, fluid 2 right) of radius R centred on the
    bottom wall, inside fluid 1; solid rows y = 0 and y = ny-1 (halfway bounce-back puts the
    wall surface at y = 0.5); periodic in x."""
    x, y = _grid(nx, ny)
    solid = np.zeros((ny, nx), np.uint8)
    solid[0, :] = 1
    solid[ny - 1, :] = 1
    cx, cy = nx / 2.0, 0.5
    inside = (x - cx) ** 2 + (y - cy) ** 2 < R * R
    labels = np.ones((ny, nx), np.int64)
    labels[inside & (x < cx)] = 0
    labels[inside & (x >= cx)] = 2
    return Workload(name or f"janus_flat_{nx}x{ny}", nx, ny, 0, BC_PERIODIC, solid,
                    _fill(labels, solid), _uniform_angles(nx, ny, triple), tuple(sigma),
                    tuple(nu), steps=steps)


def janus_cylinder(nx=512, ny=512, Rs=60.0, Rj=50.0, triple=(90.0, 90.0, 135.0),
                   sigma=(0.01, 0.005, 0.01), nu=(1.0 / 6.0,) * 3, steps=20000, name=None):
    """Section III.B: solid disc of radius Rs at the box centre; a Janus droplet of total
    radius Rj (fluid 0 for x < centre, fluid 2 otherwise) centred on the top of the disc,
    in fluid 1; periodic box."""
    x, y = _grid(nx, ny)
    cx, cy = nx / 2.0, ny / 2.0
    solid = (((x - cx) ** 2 + (y - cy) ** 2) <= Rs * Rs).astype(np.uint8)
    dcy = cy + Rs
    inside = ((x - cx) ** 2 + (y - dcy) ** 2 < Rj * Rj) & (solid == 0)
    labels = np.ones((ny, nx), np.int64)
    labels[inside & (x < cx)] = 0
    labels[inside & (x >= cx)] = 2
    return Workload(name or f"janus_cylinder_{nx}x{ny}", nx, ny, 1, BC_PERIODIC, solid,
                    _fill(labels, solid), _uniform_angles(nx, ny, triple), tuple(sigma),
                    tuple(nu), steps=steps)


def capillary(nx=2048, ny=128, y_lo=24, y_hi=104, s0=256, Lg=256,
              triple=(90.0, 135.0, 45.0), sigma=(0.01, 0.01, 0.01), nu=(0.1, 0.1, 0.1),
              steps=50000, name=None):
    """Section III.C: channel between solid rows y < y_lo and y >= y_hi; fluid 0 for
    x < s0, fluid 1 for s0 <= x < s0 + Lg, fluid 2 beyond; modified periodic in x."""
    x, y = _grid(nx, ny)
    solid = ((y < y_lo) | (y >= y_hi)).astype(np.uint8)
    labels = np.full((ny, nx), 2, np.int64)
    labels[x < s0] = 0
    labels[(x >= s0) & (x < s0 + Lg)] = 1
    return Workload(name or f"capillary_{nx}x{ny}", nx, ny, 0, BC_MODPER, solid,
                    _fill(labels, solid), _uniform_angles(nx, ny, triple), tuple(sigma),
                    tuple(nu), steps=steps)


def place_pillars(nx, ny, count, r_lo, r_hi, x_lo, x_hi, gap, seed, max_tries=200000):
    """Rejection-sample `count` non-overlapping discs (radius U[r_lo, r_hi], centre x in
    [x_lo, x_hi], y in [0, ny) periodic) at least `gap` apart, from SplitMix64(seed)."""
    rng = SplitMix64(seed)
    out = []
    tries = 0
    while len(out) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("pillar placement did not converge")
        r = rng.uniform(r_lo, r_hi)
        cx = rng.uniform(x_lo, x_hi)
        cy = rng.uniform(0.0, float(ny))
        ok = True
        for (px, py, pr) in out:
            dy = abs(cy - py)
            dy = min(dy, ny - dy)
            if math.hypot(cx - px, dy) < r + pr + gap:
                ok = False
                break
        if ok:
            out.append((cx, cy, r))
    return out, rng


def pillars(nx=4096, ny=2048, count=60, r_lo=40.0, r_hi=80.0, x_lo=900.0, x_hi=3900.0,
            gap=8.0, seed=2102, drop=(400.0, 1024.0), r_core=120.0, r_shell=200.0,
            theta=90.0, theta_range=None, u_in=0.01, sigma=(0.01, 0.01, 0.01),
            nu=(0.04, 0.04, 0.04), steps=100000, name=None):
    """Section III.D: circular pillars (seeded), compound droplet (core fluid 0, shell
    fluid 1) in carrier fluid 2; Zou-He velocity inlet at x = 0 and pressure outlet at
    x = nx-1; periodic in y.  Uniform wall angle theta: fluids 0 and 1 both make theta with
    the carrier and meet each other at 90 deg, i.e. the triple (90, 180 - theta, theta),
    which satisfies Eq.(18) for equal tensions.  With ``theta_range=(lo, hi)`` every solid
    node draws its own theta uniformly from that range (same seed stream, after the
    pillars)."""
    pl, rng = place_pillars(nx, ny, count, r_lo, r_hi, x_lo, x_hi, gap, seed)
    x, y = _grid(nx, ny)
    solid = np.zeros((ny, nx), np.uint8)
    for (cx, cy, r) in pl:
        # bounding box of the disc (rows wrap periodically)
        x0, x1 = max(0, int(math.floor(cx - r)) - 1), min(nx, int(math.ceil(cx + r)) + 2)
        rows = np.arange(int(math.floor(cy - r)) - 1, int(math.ceil(cy + r)) + 2) % ny
        xs = np.arange(x0, x1, dtype=np.float64)
        dy = np.abs(rows.astype(np.float64)[:, None] - cy)
        dy = np.minimum(dy, ny - dy)
        hit = ((xs[None, :] - cx) ** 2 + dy ** 2) <= r * r
        sub = solid[rows, x0:x1]
        sub[hit] = 1
        solid[rows, x0:x1] = sub
    dx, dy = x - drop[0], y - drop[1]
    d2 = dx * dx + dy * dy
    labels = np.full((ny, nx), 2, np.int64)
    labels[d2 < r_shell ** 2] = 1
    labels[d2 < r_core ** 2] = 0
    angles = _uniform_angles(nx, ny, (90.0, 180.0 - theta, theta))
    if theta_range is not None:
        ys, xs = np.nonzero(solid)
        th = np.array([rng.uniform(*theta_range) for _ in range(len(ys))], dtype=np.float64)
        angles[ys, xs, 0] = 90.0
        angles[ys, xs, 1] = 180.0 - th
        angles[ys, xs, 2] = th
    return Workload(name or f"pillars_{nx}x{ny}", nx, ny, 1, BC_ZOUHE, solid,
                    _fill(labels, solid), angles, tuple(sigma), tuple(nu), u_in=u_in,
                    rho_out=1.0, steps=steps)


def five_pillars(triple=(90.0, 90.0, 90.0), r_outer=50.0, sigma=0.01, name=None):
    """Section III.D as printed, in units of the outer droplet radius R_o: a 16 R_o x 7.5 R_o box
    (800 x 375 for R_o = 50), five pillars of radius 0.8 R_o centred at (6.9, 3.75), (7.3, 6.2),
    (7.5, 1.6), (9.5, 5.14) and (9.8, 2.54) R_o, a compound droplet at (2, 3.75) R_o: core of
    radius 0.6 R_o in fluid 0 (red), shell of radius R_o in fluid 1 (green), carrier fluid 2
    (blue).  Zou-He velocity inlet / pressure outlet, periodic in y.  Every tension is sigma and
    the viscosities are equal; Re = U R_o / nu = 0.75 and Ca = U nu / sigma = 0.04 then give
    nu = sqrt(0.04 sigma R_o / 0.75) and U = 0.75 nu / R_o.  ``triple`` = (theta_rg, theta_br,
    theta_gb) at every wall node; ``steps`` covers t* = U t / R_o = 40."""
    R = float(r_outer)
    nx, ny = int(round(16 * R)), int(round(7.5 * R))
    nu = math.sqrt(0.04 * sigma * R / 0.75)
    u_in = 0.75 * nu / R
    x, y = _grid(nx, ny)
    solid = np.zeros((ny, nx), np.uint8)
    for cx, cy in ((6.9, 3.75), (7.3, 6.2), (7.5, 1.6), (9.5, 5.14), (9.8, 2.54)):
        dy = np.abs(y - cy * R)
        dy = np.minimum(dy, ny - dy)
        solid[(x - cx * R) ** 2 + dy ** 2 <= (0.8 * R) ** 2] = 1
    d2 = (x - 2.0 * R) ** 2 + (y - 3.75 * R) ** 2
    labels = np.full((ny, nx), 2, np.int64)
    labels[d2 < R * R] = 1
    labels[d2 < (0.6 * R) ** 2] = 0
    return Workload(name or f"five_pillars_{nx}x{ny}", nx, ny, 1, BC_ZOUHE, solid,
                    _fill(labels, solid), _uniform_angles(nx, ny, tuple(triple)), (sigma,) * 3,
                    (nu,) * 3, u_in=u_in, rho_out=1.0, steps=int(round(40.0 * R / u_in)))


# ---- the five standard configurations ---------------------------------------------------
def config1():
    """Janus droplet on a flat wall, 128x64, R = 20, angles 90/60/120, 1000 steps."""
    return janus_flat(name="janus_flat_128x64")


def config2():
    """Perfect Janus droplet on a cylinder, 512x512, disc R = 60, droplet R = 50,
    sigma_02 = 0.005; theta_rg = 90, theta_gb = 135 (theta_bg = 45), theta_br = 90 (Eq.18 has no
    solution for theta_br with these tensions; the residual is reported)."""
    return janus_cylinder(name="janus_cylinder_512x512")


def config3(nu=(0.1, 0.1, 0.1)):
    """Ternary capillary intrusion, 2048x128, channel half-width 40, 50000 steps."""
    return capillary(nu=nu, name="capillary_2048x128")


def config4(theta=90.0):
    """Compound droplet through 60 seeded pillars, 4096x2048, U = 0.01, 100000 steps."""
    return pillars(theta=theta, name=f"pillars_4096x2048_theta{int(theta)}")


def pillars_half(theta=90.0):
    """The pillar case at half the linear size (2048x1024, 60 pillars of radius 20-40, droplet
    core 60 / shell 100): 0.23 GB per population buffer, still above L2; used for detailed
    profiles of the step kernel."""
    return pillars(nx=2048, ny=1024, count=60, r_lo=20.0, r_hi=40.0, x_lo=450.0, x_hi=1950.0,
                   gap=4.0, drop=(200.0, 512.0), r_core=60.0, r_shell=100.0, theta=theta,
                   name=f"pillars_2048x1024_theta{int(theta)}")


def config5():
    """Adjoint case: 512x256, 6 seeded pillars (radius 20-40, centres x in [150, 470]), the
    compound droplet scaled by 1/4 (core 30, shell 50) at (130, 128), per-node theta in
    U[60, 120], U = 0.01, 2000 steps.  The pillar range starts at the droplet's front (x = 180),
    so the shell reaches the pillar centred at (208, 76) within the run and wets it (27 of its
    wall nodes hold under 99 % carrier at step 2000): the angle field influences the centroid,
    and dJ/dtheta is not identically zero."""
    return pillars(nx=512, ny=256, count=6, r_lo=20.0, r_hi=40.0, x_lo=150.0, x_hi=470.0,
                   gap=8.0, seed=4709, drop=(130.0, 128.0), r_core=30.0, r_shell=50.0,
                   theta_range=(60.0, 120.0), steps=2000, name="pillars_512x256_adjoint")


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}
