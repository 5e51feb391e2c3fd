"""Seeded synthetic cases shaped like the paper's experiments.

This module holds no arithmetic of the method: it draws particle placements
with a counter-based generator (SplitMix64) and lists the problem parameters
of each case.  Both the CUDA path and the test oracle take their inputs from
here.

Cases
-----
channel   one cold disk settling in a closed channel (Secs. 3.3-3.4 proportions):
          100 x 400 cells, D = 20 at (50, 300), tau_f = 0.8, rho_s/rho_f = 1.5,
          g = 1e-5, fluid T = 1, particle T = 0, R_lambda = 2, R_cv = 1.5,
          Pr = 0.7, beta = 12.5 (Gr = 100 on D), adiabatic no-slip walls.
cavity    cold disks in a square cavity (Sec. 3.5): side L, N disks of D = 16
          at seeded non-overlapping uniform centres in the upper 60 % with
          gaps >= 2 lu between disks and from the walls, rho_s/rho_f = 1.2,
          bottom wall T = 1, top wall T = 0, adiabatic sides, fluid T = 1,
          particles T = 0, R_lambda = 5 (or per-particle log-uniform in
          [0.1, 10]), R_cv = 2, Pr = 0.71, tau_f = 0.8, sigma_0 = sigma_e =
          sigma_eps = 1 (Sec. 3.5), g = 1e-5, beta from Gr = 100 on the
          cavity height.
"""
from __future__ import annotations

import dataclasses
import math

MASK64 = (1 << 64) - 1


class SplitMix64:
    """Counter-based generator of Steele, Lea & Flood (2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


@dataclasses.dataclass
class Case:
    """Problem parameters (names of include/vlb.h) and the particle arrays."""
    name: str
    params: dict
    x: list
    y: list
    radius: list
    T0: list
    k_ratio: list | None = None
    fixed_T: list | None = None   # particles held at their temperature T0
    semi_minor: list | None = None  # ellipses: semi-minor axes (radius = semi-major axis)
    theta0: list | None = None      # ellipses: initial angle of the major axis

    @property
    def cells(self) -> int:
        return self.params["nx"] * self.params["ny"]


def place_disks(nx: int, ny: int, n: int, diameter: float, seed: int, y_min_frac: float = 0.4,
                gap: float = 2.0, max_tries: int = 2_000_000):
    """Rejection sampling of n disk centres, uniform in
    [R + gap, nx - R - gap] x [max(y_min_frac * ny, 0) + R + gap, ny - R - gap],
    keeping centre distances >= diameter + gap."""
    rng = SplitMix64(seed)
    R = 0.5 * diameter
    x_lo, x_hi = R + gap, nx - R - gap
    y_lo, y_hi = y_min_frac * ny + R + gap, ny - R - gap
    cell = diameter + gap
    grid: dict = {}
    xs, ys = [], []
    tries = 0
    while len(xs) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"could not place {n} disks (placed {len(xs)})")
        x = rng.uniform(x_lo, x_hi)
        y = rng.uniform(y_lo, y_hi)
        gx, gy = int(x // cell), int(y // cell)
        ok = True
        for a in (gx - 1, gx, gx + 1):
            for b in (gy - 1, gy, gy + 1):
                for k in grid.get((a, b), ()):
                    if (xs[k] - x) ** 2 + (ys[k] - y) ** 2 < cell * cell:
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            grid.setdefault((gx, gy), []).append(len(xs))
            xs.append(x)
            ys.append(y)
    return xs, ys


def gr_beta(gr: float, nu: float, g: float, dT: float, D: float) -> float:
    """Volume expansivity giving a Grashof number gr on the diameter (Eq. 32)."""
    return gr * nu * nu / (g * dT * D ** 3)


def channel(precision: str = "fp64") -> Case:
    nu = (0.8 - 0.5) / 3.0
    params = dict(nx=100, ny=400, tau_f=0.8, prandtl=0.7, rho_ratio=1.5, cv_ratio=1.5, k_ratio_default=2.0,
                  gravity=(0.0, -1e-5), beta=gr_beta(100.0, nu, 1e-5, 1.0, 20.0), T_ref=1.0, T_fluid_init=1.0,
                  thermal_wall=(0, 0, 0, 0), wall_T=(0.0, 0.0, 0.0, 0.0), thermal_rates_mode=0,
                  precision=precision)
    return Case("channel 100x400, 1 disk D=20", params, [50.0], [300.0], [10.0], [0.0])


def fixed_temperature_sedimentation(gr: float, length_d: float = 80.0, precision: str = "fp32", hold: int = 1,
                                    diameter: float = 20.0) -> Case:
    """Sedimentation of a disk held at T_c = 0 in a long channel (the paper's
    Sec. 3.3 case, Table 4): D = 20 lu, width 4D, the disk starting D/2
    left of the centreline (x = 1.5 D), rho_r = 1.00232, Re = 40.5, Pr = 0.7,
    Grashof number gr, tau_f = 0.53, R_lambda = R_cv = 1 (hold: 1 reading R11, 2
    reading R11b of how the particle is held); fluid and walls at
    T_h = 1 (T_ref = T_h).  The channel length is not given (length_d
    diameters; the disk starts 10 D below the top)."""
    D = float(diameter)  # 20 cells in the paper (dx = D/20); other values for resolution checks
    nu = (0.53 - 0.5) / 3.0
    u_ref = 40.5 * nu / D
    g = u_ref ** 2 / ((1.00232 - 1.0) * math.pi * D / 2.0)
    nx, ny = int(4 * D), int(length_d * D)
    params = dict(nx=nx, ny=ny, tau_f=0.53, prandtl=0.7, rho_ratio=1.00232, cv_ratio=1.0,
                  k_ratio_default=1.0, gravity=(0.0, -g), beta=gr_beta(gr, nu, g, 1.0, D), T_ref=1.0,
                  T_fluid_init=1.0, thermal_wall=(1, 1, 1, 1), wall_T=(1.0, 1.0, 1.0, 1.0),
                  thermal_rates_mode=0, precision=precision)
    return Case(f"fixed-temperature sedimentation {nx}x{ny}, Gr={gr:g}", params, [1.5 * D], [ny - 10.0 * D],
                [D / 2.0], [0.0], None, [hold])


def ellipse_sedimentation(length_w: float = 30.0, theta0: float = math.pi / 4, x_offset: float = 0.0,
                          precision: str = "fp32") -> Case:
    """Isothermal sedimentation of an elliptical particle in a long channel
    (Sec. 3.2): channel width L = 104 cells (dx = 1/260 cm for L = 0.4 cm),
    semi-axes a = 13 and b = 6.5 cells (0.05 and 0.025 cm), rho_s/rho_f = 1.1,
    nu = 0.01 cm^2/s, |g| = 980 cm/s^2, tau_f = 0.6 (so dt = nu_lu dx^2 / nu
    and g = 980 dt^2 / dx in lattice units); the particle starts at rest in
    the middle of the channel, 3 L below its top, its major axis at theta0 to
    the horizontal (x_offset moves it sideways); no-slip side walls and top,
    the bottom open (fully developed outflow); only the flow matters (beta =
    0, uniform temperature).  The channel is length_w widths long (30 in the
    paper)."""
    W = 104
    dx = 0.4 / W                       # cm
    nu_lu = (0.6 - 0.5) / 3.0
    dt = nu_lu * dx * dx / 0.01        # s
    g = 980.0 * dt * dt / dx           # lattice units
    ny = int(round(length_w * W))
    params = dict(nx=W, ny=ny, tau_f=0.6, prandtl=0.7, rho_ratio=1.1, cv_ratio=1.0, k_ratio_default=1.0,
                  gravity=(0.0, -g), beta=0.0, T_ref=1.0, T_fluid_init=1.0, thermal_wall=(0, 0, 0, 0),
                  wall_T=(0.0, 0.0, 0.0, 0.0), thermal_rates_mode=0, outflow=(0, 0, 1, 0), precision=precision)
    c = Case(f"elliptical particle in a {W}x{ny} channel (a=13, b=6.5, theta0={theta0:.4f})", params,
             [W / 2.0 + x_offset], [ny - 3.0 * W], [13.0], [1.0])
    c.semi_minor = [6.5]
    c.theta0 = [theta0]
    return c


def conjugate_sedimentation(r_cv: float, length_d: float = 40.0, precision: str = "fp32") -> Case:
    """Sedimentation of a cold disk with conjugate heat transfer in a long
    channel (the paper's Sec. 3.4 conjugate case): D = 20 lu, width 4D, the
    disk on the centreline, rho_r = 1.00232, Re = 10.5, Pr = 0.7, Gr = 1000,
    tau_f = 0.53, R_lambda = 1, R_cv as given; T_c = 0 in the disk, T_h = 1 in
    the fluid and on the walls (T_ref = T_h).  The channel length is not
    given (length_d diameters; the disk starts 10 D below the top)."""
    D = 20.0
    nu = (0.53 - 0.5) / 3.0
    u_ref = 10.5 * nu / D                                  # Re = U_ref D / nu
    g = u_ref ** 2 / ((1.00232 - 1.0) * math.pi * D / 2.0)  # U_ref = sqrt((rho_r - 1) |g| pi D / 2)
    nx, ny = int(4 * D), int(length_d * D)
    params = dict(nx=nx, ny=ny, tau_f=0.53, prandtl=0.7, rho_ratio=1.00232, cv_ratio=float(r_cv),
                  k_ratio_default=1.0, gravity=(0.0, -g), beta=gr_beta(1000.0, nu, g, 1.0, D), T_ref=1.0,
                  T_fluid_init=1.0, thermal_wall=(1, 1, 1, 1), wall_T=(1.0, 1.0, 1.0, 1.0),
                  thermal_rates_mode=0, precision=precision)
    return Case(f"conjugate sedimentation {nx}x{ny}, R_cv={r_cv:g}", params, [nx / 2.0], [ny - 10.0 * D],
                [D / 2.0], [0.0])


def cavity(side: int = 2048, n: int = 2048, diameter: float = 16.0, seed: int = 20241031,
           precision: str = "fp32", k_log_uniform: bool = False, gap: float = 2.0) -> Case:
    nu = (0.8 - 0.5) / 3.0
    g = 1e-5
    xs, ys = place_disks(side, side, n, diameter, seed, gap=gap)
    # beta from Gr = 100 on the cavity height (reading R9): with the held
    # bottom and top walls the cavity is a Rayleigh-Benard cell, and Gr on
    # the disk diameter would make it one at Ra ~ 1e11, which leaves the
    # low-Mach range within the configuration's 20,000 steps
    params = dict(nx=side, ny=side, tau_f=0.8, prandtl=0.71, rho_ratio=1.2, cv_ratio=2.0, k_ratio_default=5.0,
                  gravity=(0.0, -g), beta=gr_beta(100.0, nu, g, 1.0, float(side)), T_ref=1.0, T_fluid_init=1.0,
                  thermal_wall=(0, 0, 1, 1), wall_T=(0.0, 0.0, 1.0, 0.0), thermal_rates_mode=1,
                  precision=precision)
    k = None
    if k_log_uniform:
        rng = SplitMix64(seed ^ 0x5DEECE66D)
        k = [10.0 ** rng.uniform(-1.0, 1.0) for _ in range(n)]
    return Case(f"cavity {side}x{side}, {n} disks D={diameter:g}", params, xs, ys, [0.5 * diameter] * n,
                [0.0] * n, k)


def channels(n: int = 256, seed: int = 20241104, w_min: int = 64, w_max: int = 256,
             precision: str = "fp32") -> list:
    """n independent single-disk channels in the proportions of the channel
    case: width W ~ U{w_min..w_max}, length 4 W, disk diameter D = W U[0.1, 0.25]
    released at rest at (W/2, 3 W), rho_s/rho_f ~ U[1.1, 2.0], R_lambda =
    10^U[-1, 1], R_cv = 1.5, tau_f = 0.8, Pr = 0.7, g = 1e-5, beta from Gr = 100
    on the case's D, fluid T = 1, particle T = 0, adiabatic no-slip walls."""
    rng = SplitMix64(seed)
    nu = (0.8 - 0.5) / 3.0
    out = []
    for k in range(n):
        w = w_min + int(rng.next_u64() % (w_max - w_min + 1))
        D = w * rng.uniform(0.1, 0.25)
        rho_r = rng.uniform(1.1, 2.0)
        k_r = 10.0 ** rng.uniform(-1.0, 1.0)
        params = dict(nx=w, ny=4 * w, tau_f=0.8, prandtl=0.7, rho_ratio=rho_r, cv_ratio=1.5, k_ratio_default=k_r,
                      gravity=(0.0, -1e-5), beta=gr_beta(100.0, nu, 1e-5, 1.0, D), T_ref=1.0, T_fluid_init=1.0,
                      thermal_wall=(0, 0, 0, 0), wall_T=(0.0, 0.0, 0.0, 0.0), thermal_rates_mode=0,
                      precision=precision)
        out.append(Case(f"channel {w}x{4 * w}, 1 disk D={D:.3f}", params, [w / 2.0], [3.0 * w], [D / 2.0], [0.0]))
    return out


def served_cases(n: int = 200, seed: int = 20241105, steps: int = 2000, side_log2=(6.0, 10.0),
                 max_particles_log2: float = 9.0, d_range=(8.0, 24.0), max_solid: float = 0.3) -> list:
    """A stream of n sedimentation cases for the served mode: (gap, Case,
    steps) with gap the time since the previous arrival in units of the mean
    (exponential, i.e. Poisson arrivals at rate 1).  Each case is a cavity
    (the cavity case's parameters) of side 2^U[6, 10] (rounded), holding
    floor(2^U[0, 9]) disks of one diameter D ~ U[8, 24] (fewer where their
    area would pass max_solid of the upper 60 %), half of the cases with FP32
    populations and half with FP16 storage."""
    rng = SplitMix64(seed)
    out = []
    for k in range(n):
        gap = -math.log(1.0 - rng.uniform())
        side = int(round(2.0 ** rng.uniform(*side_log2)))
        npart = int(2.0 ** rng.uniform(0.0, max_particles_log2))
        D = rng.uniform(*d_range)
        cap = int(max_solid * 0.6 * side * side / (math.pi * D * D / 4.0))
        npart = max(1, min(npart, cap))
        precision = "fp32" if rng.next_u64() & 1 else "fp16"
        c = cavity(side=side, n=npart, diameter=D, seed=seed + 7919 * (k + 1), precision=precision)
        out.append((gap, c, steps))
    return out
