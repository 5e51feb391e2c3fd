"""FP64 oracle: the volumetric LB method written out phase by phase.

TEST INFRASTRUCTURE ONLY (see the package docstring): only tests, the smoke
check and the benchmark's CPU-baseline leg use this module.

Conventions
-----------
* Lattice units, delta_x = delta_t = c = 1.
* Cell (i, j) covers [i, i+1] x [j, j+1]; its node sits at the cell centre
  (i + 1/2, j + 1/2) -- the volumetric interpretation of Sec. 2 / Fig. 1.
* Fields are numpy arrays indexed [y, x]; populations have shape (9, ny, nx).
* Walls sit on the cell faces of the domain boundary.

Readings of passages the paper leaves open (each one is also listed in the
design notes of the repository):

R1  Solid fraction (Sec. 2, "directly determined by the position"): the exact
    area of disk ∩ cell.  A cell is *solid* for a particle when its four
    corners lie in the closed disk, *fluid* when its nearest point lies at
    distance >= R, else *interface*.  Those two tests run on positions
    rounded to a 2^-20 fixed-point grid, in integers, so that both
    implementations take the same integer decisions.  Several particles may
    own one cell (at most 4); their fractions add, and are scaled down so
    that they sum to 1 if they exceed it (only under contact overlap).
R2  Walls (Sec. 3): halfway bounce-back for f; bounce-back for g at adiabatic
    walls; anti-bounce-back g_i = -gbar_opp(i) + 2 g_i^eq(T_w) at walls held
    at T_w.  A population that crosses a domain corner is handled by the
    wall normal to y.
R3  Time levels (Sec. 2.3, Eq. 8 and the forward-Euler remark at the end of
    Sec. 2.3): the particle state used by the correction of step n -> n+1 is
    advanced explicitly from the force of level n (lagged coupling).
R4  Buoyancy on the fluid (Sec. 3.3) is weighted by (1 - f_s) so that u = u_s
    stays exact in solid cells (Sec. 2.1); the circular dependence between
    T (Eq. 25) and u (Eq. 9) through the buoyancy force is closed by solving
    both at t + dt jointly (closed form below).
R5  Contact (Sec. 2.3 cites Glowinski et al. 2001 without its formula): the
    normalised short-range repulsion
      F_ij = (c_ij / eps_p) * (max(0, R_i + R_j + zeta - d_ij) / zeta)^2
             * (X_i - X_j) / d_ij,
    c_ij = |rho_r - 1| rho_f |g| pi max(R_i, R_j)^2, and its image-particle
    form at walls with eps_w.  It is central (no torque).
R6  Initial state: f* = f^eq(1, 0) corrected with f_s^0 (Eq. 8); the internal
    energy is mixed by volume, eps^0 = (1 - f_s) c_vf T_f + sum_p f_s,p c_vs
    T_p, T^0 = eps^0 / c_v; g^0 = g^eq(eps^0, T^0); q_c^0 = 0 and
    [df_s/dt]^0 = 0.
R7  Domain: fractions exist only for cells inside the domain; a particle may
    not cross a periodic boundary.
R13 Elliptical particles (Sec. 3.2 gives the shape, a = 2b, and its
    orientation, nothing of how it is rasterised or touches others): the
    exact area of ellipse ∩ cell, found in the ellipse's unit-disk frame
    where the cell is a parallelogram; a cell is SOLID when its four corners
    lie in the closed ellipse and FLUID when the ellipse's quadratic form
    stays >= 1 over the cell, both decided in FP64; the orientation theta
    advances as theta + Omega (forward Euler) and sets the raster; mass
    rho_s pi a b, moment of inertia M (a^2 + b^2) / 4; contact between
    particles through the circumscribed disks, with a wall through the
    extent of the ellipse along the wall's normal.
R14 Fully developed outflow (Sec. 3.2, the lower end of the long channel:
    the normal derivative of u vanishes): a population entering through an
    open side takes the value the same population has one cell further in
    (zero normal gradient after streaming), for f and g alike; no wall
    contact there.
R12 Mid-run insertion (the paper has none): a disk added at level n joins the
    particle set and first appears in the raster of level n+1; the correction
    (Eq. 8) and the df_s/dt recursion (Eq. 24) then act on it as on a disk
    moving into cells, so it starts at the temperature of the fluid it
    displaces; its first update has no exchange and no contact force.
"""
from __future__ import annotations

import dataclasses
import functools
import math

import numpy as np

# --------------------------------------------------------------------------
# D2Q9 velocity set (Eq. 2) and the orthogonal moment matrix (Eq. 4).
# --------------------------------------------------------------------------


def lattice_velocities() -> np.ndarray:
    """The nine discrete velocities of Eq. 2 with c = 1, as integers."""
    e = np.zeros((9, 2))
    for i in range(1, 5):
        a = (i - 1) * math.pi / 2.0
        e[i] = (math.cos(a), math.sin(a))
    for i in range(5, 9):
        a = (2 * i - 1) * math.pi / 4.0
        e[i] = (math.sqrt(2.0) * math.cos(a), math.sqrt(2.0) * math.sin(a))
    return np.rint(e).astype(np.int64)


E = lattice_velocities()
EX = E[:, 0].astype(np.float64)
EY = E[:, 1].astype(np.float64)
OPP = np.array([int(np.where((E == -E[i]).all(axis=1))[0][0]) for i in range(9)])

# Eq. 4, row by row.
M = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1, 1],
        [-4, -1, -1, -1, -1, 2, 2, 2, 2],
        [4, -2, -2, -2, -2, 1, 1, 1, 1],
        [0, 1, 0, -1, 0, 1, -1, -1, 1],
        [0, -2, 0, 2, 0, 1, -1, -1, 1],
        [0, 0, 1, 0, -1, 1, 1, -1, -1],
        [0, 0, -2, 0, 2, 1, 1, -1, -1],
        [0, 1, -1, 1, -1, 0, 0, 0, 0],
        [0, 0, 0, 0, 0, 1, -1, 1, -1],
    ],
    dtype=np.float64,
)
MINV = np.linalg.inv(M)

# Free parameters of the thermal LBE fixed in Sec. 2.2.
ALPHA1 = -2.0
ALPHA2 = 1.0
BETA1 = -4.0
BETA2 = 4.0

QBITS = 20  # fixed-point grid of the integer cell tests (reading R1)
MAX_OWNERS = 4


def to_moments(f: np.ndarray) -> np.ndarray:
    """m = M f for every cell (f has shape (9, ...))."""
    return np.tensordot(M, f, axes=(1, 0))


def from_moments(m: np.ndarray) -> np.ndarray:
    """f = M^-1 m for every cell."""
    return np.tensordot(MINV, m, axes=(1, 0))


# --------------------------------------------------------------------------
# Flow LBE (Sec. 2.1): Eqs. 3, 5, 6, 7, 8, 9.
# --------------------------------------------------------------------------


def flow_eq_moments(rho, ux, uy):
    """Equilibrium moments m^eq(rho, u) of Eq. 6."""
    u2 = ux * ux + uy * uy
    return np.stack(
        [
            rho,
            -2.0 * rho + 3.0 * rho * u2,
            rho - 3.0 * rho * u2,
            rho * ux,
            -rho * ux,
            rho * uy,
            -rho * uy,
            rho * (ux * ux - uy * uy),
            rho * ux * uy,
        ]
    )


def force_moments(Fx, Fy, ux, uy):
    """Discrete force term F_m of Eq. 7."""
    Fu = Fx * ux + Fy * uy
    z = np.zeros_like(Fu)
    return np.stack(
        [
            z,
            6.0 * Fu,
            -6.0 * Fu,
            Fx + z,
            -Fx + z,
            Fy + z,
            -Fy + z,
            2.0 * (Fx * ux - Fy * uy),
            Fx * uy + Fy * ux,
        ]
    )


def feq(rho, ux, uy):
    """f^eq(rho, u) = M^-1 m^eq(rho, u) (definition below Eq. 5)."""
    return from_moments(flow_eq_moments(rho, ux, uy))


def flow_rates(tau_f: float, lambda_q: float = 1.0 / 12.0, s_e: float = 1.25,
               s0: float = 1.0, s_j: float = 1.0):
    """Diagonal of S (Eq. 5) with the rules of Sec. 3: s0 = s_j = 1,
    s_e = s_eps, s_p = 1/tau_f and (1/s_p - 1/2)(1/s_q - 1/2) = lambda_q."""
    s_p = 1.0 / tau_f
    s_q = 1.0 / (0.5 + lambda_q / (tau_f - 0.5))
    return np.array([s0, s_e, s_e, s_j, s_q, s_j, s_q, s_p, s_p])


def collide_flow(f, rho, ux, uy, Fx, Fy, S):
    """Post-collision fbar from Eq. 3a: mbar = m - S (m - m^eq) + (I - S/2) F_m."""
    m = to_moments(f)
    meq = flow_eq_moments(rho, ux, uy)
    Fm = force_moments(Fx, Fy, ux, uy)
    s = np.asarray(S, dtype=np.float64).reshape((9,) + (1,) * (f.ndim - 1))
    mbar = m - s * (m - meq) + (1.0 - 0.5 * s) * Fm
    return from_moments(mbar)


def flow_macroscopics(f, Fx, Fy):
    """rho and u of Eq. 9: rho = sum f, rho u = sum e f + F/2."""
    rho = f.sum(axis=0)
    jx = np.tensordot(EX, f, axes=(0, 0))
    jy = np.tensordot(EY, f, axes=(0, 0))
    return rho, (jx + 0.5 * Fx) / rho, (jy + 0.5 * Fy) / rho


# --------------------------------------------------------------------------
# Streaming with walls (Eqs. 3b, 17b; reading R2).
# --------------------------------------------------------------------------


@functools.lru_cache(maxsize=64)
def _source_index(nx, ny, i, periodic):
    """Source cell x - e_i of every cell for the pull form of streaming,
    wrapped on periodic axes; flags where it falls outside the domain."""
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    sx = xx - E[i, 0]
    sy = yy - E[i, 1]
    if periodic[0]:
        sx = sx % nx
    if periodic[1]:
        sy = sy % ny
    out_x = (sx < 0) | (sx >= nx)
    out_y = (sy < 0) | (sy >= ny)
    return yy, xx, np.clip(sy, 0, ny - 1), np.clip(sx, 0, nx - 1), out_x, out_y, sy < 0, sx < 0


def _outflow_copy(dist, i, yy, xx, ox, oy, ylow, xlow, outflow):
    """Zero normal gradient at open sides (reading R14, the fully developed
    condition of Sec. 3.2): a population that would come from outside through
    an open side takes the value the same population has one cell further in,
    f*_i(x) = f*_i(x + n) = dist_i(x - e_i + n) with n the side's inward
    normal.  Returns the mask of cells this applies to and the values.  A
    population crossing a corner takes the rule of the x side when the y
    side is open."""
    ny, nx = yy.shape
    side_x = np.where(xlow, 0, 1)
    side_y = np.where(ylow, 2, 3)
    open_x = np.asarray(outflow, dtype=bool)[side_x] & ox
    open_y = np.asarray(outflow, dtype=bool)[side_y] & oy
    # source one cell in from the crossed side(s): drop the crossing component of -e_i
    sx = np.where(ox, xx, (xx - E[i, 0]) % nx)
    sy = np.where(oy, yy, (yy - E[i, 1]) % ny)
    mask = (open_y & ~ox) | (open_x & ~oy) | (open_x & open_y)
    return mask, dist[i, sy, sx]


def stream_flow(fbar, periodic=(False, False), outflow=(False, False, False, False)):
    """Linear streaming f*_i(x + e_i) = fbar_i(x) (Eq. 3b), written as a
    pull.  Where x - e_i lies outside the domain the population bounces back
    halfway at the wall face: f*_i(x) = fbar_opp(i)(x); through an open
    side (outflow) it takes the zero-gradient value (reading R14)."""
    _, ny, nx = fbar.shape
    out = np.empty_like(fbar)
    for i in range(9):
        yy, xx, sy, sx, ox, oy, ylow, xlow = _source_index(nx, ny, i, tuple(periodic))
        outside = ox | oy
        pulled = fbar[i, sy, sx]
        res = np.where(outside, fbar[OPP[i], yy, xx], pulled)
        if any(outflow):
            mask, copied = _outflow_copy(fbar, i, yy, xx, ox, oy, ylow, xlow, outflow)
            res = np.where(mask, copied, res)
        out[i] = res
    return out


def stream_thermal(gbar, cref, thermal_wall, wall_T, periodic=(False, False), outflow=(False, False, False, False)):
    """Streaming of g (Eq. 17b) as a pull.  At a wall (order x-, x+, y-, y+):
    adiabatic -> g_i(x) = gbar_opp(i)(x); held at T_w ->
    g_i(x) = -gbar_opp(i)(x) + 2 g_i^eq(T_w).  The moving components of
    g^eq (Eq. 19) do not depend on epsilon, so g_i^eq(T_w) is taken from
    M^-1 n^eq(0, T_w)."""
    _, ny, nx = gbar.shape
    out = np.empty_like(gbar)
    geq_wall = [from_moments(thermal_eq_moments(np.zeros(1), np.full(1, float(wall_T[w])), cref))[:, 0]
                for w in range(4)]
    for i in range(9):
        yy, xx, sy, sx, ox, oy, ylow, xlow = _source_index(nx, ny, i, tuple(periodic))
        pulled = gbar[i, sy, sx]
        bounce = gbar[OPP[i], yy, xx]
        # which wall: y walls first (reading R2 for corners)
        wall = np.where(oy, np.where(ylow, 2, 3), np.where(xlow, 0, 1))
        res = np.where(ox | oy, bounce, pulled)
        for w in range(4):
            if thermal_wall[w] == 1:
                geq_w = geq_wall[w][i]
                sel = (ox | oy) & (wall == w)
                res = np.where(sel, -bounce + 2.0 * geq_w, res)
        if any(outflow):
            # open sides: zero normal gradient of g as of f (reading R14); a
            # corner under an open y side takes the x side's rule
            mask, copied = _outflow_copy(gbar, i, yy, xx, ox, oy, ylow, xlow, outflow)
            res = np.where(mask, copied, res)
            corner = ox & oy & np.asarray(outflow, dtype=bool)[np.where(ylow, 2, 3)] & \
                ~np.asarray(outflow, dtype=bool)[np.where(xlow, 0, 1)]
            xw = np.where(xlow, 0, 1)
            cres = bounce.copy()
            for w in (0, 1):
                if thermal_wall[w] == 1:
                    cres = np.where(xw == w, -bounce + 2.0 * geq_wall[w][i], cres)
            res = np.where(corner, cres, res)
        out[i] = res
    return out


# --------------------------------------------------------------------------
# Solid fraction (Sec. 2, reading R1).
# --------------------------------------------------------------------------


def _segment_integral(u, R):
    """P(u) = integral_0^u sqrt(R^2 - t^2) dt for |u| <= R."""
    u = np.clip(u, -R, R)
    return 0.5 * (u * np.sqrt(np.maximum(R * R - u * u, 0.0)) + R * R * np.arcsin(u / R))


def quadrant_area(a, b, R):
    """Area of {(u, v): u^2 + v^2 <= R^2, u <= a, v <= b} (disk at origin).

    For fixed u the admissible v form [-s, min(b, s)], s = sqrt(R^2 - u^2).
    Its length is 2s where s <= b, b + s where -s < b < s, and 0 where
    b <= -s.  With c = sqrt(R^2 - b^2) those regions are |u| >= c (b >= 0),
    |u| < c, and |u| >= c (b < 0); integrating them up to u = a gives the
    result."""
    a = np.clip(np.asarray(a, dtype=np.float64), -R, R)
    b = np.clip(np.asarray(b, dtype=np.float64), -R, R)
    c = np.sqrt(np.maximum(R * R - b * b, 0.0))
    P = lambda u: _segment_integral(u, R)  # noqa: E731
    # u in [-R, -c]: length 2s if b >= 0 else 0
    hi1 = np.minimum(a, -c)
    seg1 = np.where((b >= 0) & (hi1 > -R), 2.0 * (P(hi1) - P(-R)), 0.0)
    # u in [-c, c]: length b + s
    hi2 = np.minimum(a, c)
    seg2 = np.where(hi2 > -c, b * (hi2 + c) + P(hi2) - P(-c), 0.0)
    # u in [c, R]: length 2s if b >= 0 else 0
    seg3 = np.where((b >= 0) & (a > c), 2.0 * (P(a) - P(c)), 0.0)
    return seg1 + seg2 + seg3


def cell_disk_area(x0, x1, y0, y1, X, Y, R):
    """Exact area of disk(X, Y, R) ∩ [x0, x1] x [y0, y1] by inclusion-exclusion
    of quadrant areas."""
    a0, a1 = x0 - X, x1 - X
    b0, b1 = y0 - Y, y1 - Y
    return (quadrant_area(a1, b1, R) - quadrant_area(a0, b1, R)
            - quadrant_area(a1, b0, R) + quadrant_area(a0, b0, R))


def quantise(v) -> np.ndarray:
    """Round to the 2^-20 fixed-point grid of the integer cell tests."""
    return np.rint(np.asarray(v, dtype=np.float64) * float(1 << QBITS)).astype(np.int64)


FLUID, INTERFACE, SOLID = 0, 1, 2


def cell_flags(i, j, Xq, Yq, Rq):
    """Classify cells (i, j) against one disk in fixed point (reading R1):
    SOLID if all four corners are in the closed disk, FLUID if the nearest
    point of the cell is at distance >= R, INTERFACE otherwise."""
    Q = np.int64(1 << QBITS)
    cx0 = i.astype(np.int64) * Q - Xq
    cx1 = cx0 + Q
    cy0 = j.astype(np.int64) * Q - Yq
    cy1 = cy0 + Q
    far2 = np.maximum(cx0 * cx0, cx1 * cx1) + np.maximum(cy0 * cy0, cy1 * cy1)
    nx_ = np.where((cx0 <= 0) & (cx1 >= 0), 0, np.minimum(np.abs(cx0), np.abs(cx1)))
    ny_ = np.where((cy0 <= 0) & (cy1 >= 0), 0, np.minimum(np.abs(cy0), np.abs(cy1)))
    near2 = nx_ * nx_ + ny_ * ny_
    R2 = Rq * Rq
    return np.where(far2 <= R2, SOLID, np.where(near2 >= R2, FLUID, INTERFACE))


@dataclasses.dataclass
class Raster:
    """Per-cell solid fraction and ownership (reading R1)."""
    fs: np.ndarray         # (ny, nx) total solid fraction
    count: np.ndarray      # (ny, nx) number of owners
    owner: np.ndarray      # (ny, nx, 4) particle id, -1 padded, ascending
    flag: np.ndarray       # (ny, nx, 4) INTERFACE or SOLID, 0 padded
    fsp: np.ndarray        # (ny, nx, 4) per-owner fraction (after scaling)


def rasterise(nx, ny, X, Y, R) -> Raster:
    """Solid-fraction field f_s of a set of disks (Sec. 2 and Eq. 8)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    count = np.zeros((ny, nx), dtype=np.int64)
    owner = np.full((ny, nx, MAX_OWNERS), -1, dtype=np.int64)
    flag = np.zeros((ny, nx, MAX_OWNERS), dtype=np.int64)
    fsp = np.zeros((ny, nx, MAX_OWNERS), dtype=np.float64)
    Xq, Yq, Rq = quantise(X), quantise(Y), quantise(R)
    for p in range(X.shape[0]):
        i0 = max(int(math.floor(X[p] - R[p])) - 1, 0)
        i1 = min(int(math.ceil(X[p] + R[p])) + 1, nx - 1)
        j0 = max(int(math.floor(Y[p] - R[p])) - 1, 0)
        j1 = min(int(math.ceil(Y[p] + R[p])) + 1, ny - 1)
        if i1 < i0 or j1 < j0:
            continue
        jj, ii = np.meshgrid(np.arange(j0, j1 + 1), np.arange(i0, i1 + 1), indexing="ij")
        fl = cell_flags(ii, jj, Xq[p], Yq[p], Rq[p])
        sel = fl != FLUID
        if not sel.any():
            continue
        ci, cj, cf = ii[sel], jj[sel], fl[sel]
        area = cell_disk_area(ci.astype(float), ci + 1.0, cj.astype(float), cj + 1.0, X[p], Y[p], R[p])
        val = np.where(cf == SOLID, 1.0, np.clip(area, 0.0, 1.0))
        k = count[cj, ci]
        if (k >= MAX_OWNERS).any():
            raise OverflowError("more than 4 particles own one cell")
        owner[cj, ci, k] = p
        flag[cj, ci, k] = cf
        fsp[cj, ci, k] = val
        count[cj, ci] = k + 1
    tot = fsp.sum(axis=2)
    scale = np.where(tot > 1.0, 1.0 / np.where(tot > 1.0, tot, 1.0), 1.0)
    fsp = fsp * scale[:, :, None]
    return Raster(fs=fsp.sum(axis=2), count=count, owner=owner, flag=flag, fsp=fsp)


# --------------------------------------------------------------------------
# Elliptical particles (Sec. 3.2; reading R13).
# --------------------------------------------------------------------------


def ellipse_frame(px, py, X, Y, a, b, c, s):
    """Coordinates of the points (px, py) in the frame of the ellipse centred
    at (X, Y) with semi-axes a (along its major axis, at angle theta to the
    x axis, c = cos theta, s = sin theta) and b, scaled so that the ellipse is
    the unit disk: (u / a, v / b), u = c dx + s dy, v = -s dx + c dy."""
    dx = px - X
    dy = py - Y
    return (c * dx + s * dy) / a, (c * dy - s * dx) / b


def ellipse_cell_class(i, j, X, Y, a, b, c, s):
    """Class of cell [i, i+1] x [j, j+1] against the closed ellipse
    (reading R13): SOLID when its four corners lie in the ellipse (then the
    convex cell does), FLUID when the smallest value over the cell of
    Q = (u/a)^2 + (v/b)^2 is >= 1 (the cell meets the ellipse at most in one
    point), INTERFACE otherwise.  On each edge P0 + t d, t in [0, 1], Q is a
    convex quadratic in t whose minimum sits at its vertex clamped to
    [0, 1]."""
    corners = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
    qc = []
    for (xa, ya) in corners:
        u, v = ellipse_frame(float(xa), float(ya), X, Y, a, b, c, s)
        qc.append(u * u + v * v)
    if max(qc) <= 1.0:
        return SOLID
    if i <= X <= i + 1 and j <= Y <= j + 1:
        return INTERFACE  # the centre lies in the cell
    qmin = min(qc)
    for k in range(4):
        x0, y0 = corners[k]
        x1, y1 = corners[(k + 1) % 4]
        u0, v0 = ellipse_frame(float(x0), float(y0), X, Y, a, b, c, s)
        u1, v1 = ellipse_frame(float(x1), float(y1), X, Y, a, b, c, s)
        du, dv = u1 - u0, v1 - v0
        A = du * du + dv * dv
        t = min(max(-(u0 * du + v0 * dv) / A, 0.0), 1.0)
        uu, vv = u0 + t * du, v0 + t * dv
        qmin = min(qmin, uu * uu + vv * vv)
    return FLUID if qmin >= 1.0 else INTERFACE


def polygon_unit_disk_area(us, vs):
    """Area of the unit disk intersected with the convex polygon of vertices
    (us[k], vs[k]) in counter-clockwise order, by Green's theorem on the
    boundary of the intersection: the parts of the polygon's edges inside
    the disk contribute (u dv - v du) / 2 = (u_a v_b - u_b v_a) / 2 each, and
    the arcs of the circle between leaving the disk on one edge and entering
    it on a later one contribute half their angle (counter-clockwise)."""
    n = len(us)
    pieces = []  # inside parts of the edges, in boundary order: (start, end)
    for k in range(n):
        u0, v0 = us[k], vs[k]
        u1, v1 = us[(k + 1) % n], vs[(k + 1) % n]
        du, dv = u1 - u0, v1 - v0
        A = du * du + dv * dv
        B = u0 * du + v0 * dv
        C = u0 * u0 + v0 * v0 - 1.0
        disc = B * B - A * C
        if A == 0.0 or disc <= 0.0:
            continue
        r = math.sqrt(disc)
        t0, t1 = max((-B - r) / A, 0.0), min((-B + r) / A, 1.0)
        if t1 <= t0:
            continue
        pieces.append(((u0 + t0 * du, v0 + t0 * dv), (u0 + t1 * du, v0 + t1 * dv), k))
    if not pieces:
        # no edge meets the disk: the disk lies inside the polygon or outside it
        inside = all((us[(k + 1) % n] - us[k]) * (0.0 - vs[k]) - (vs[(k + 1) % n] - vs[k]) * (0.0 - us[k]) >= 0.0
                     for k in range(n))
        return math.pi if inside else 0.0
    area = 0.0
    for m, (pa, pb, k) in enumerate(pieces):
        area += 0.5 * (pa[0] * pb[1] - pb[0] * pa[1])
        qa, _, k2 = pieces[(m + 1) % len(pieces)]  # where the boundary re-enters
        if k2 == (k + 1) % n and math.hypot(qa[0] - pb[0], qa[1] - pb[1]) < 1e-12:
            continue  # the boundary turns at a vertex on the circle: no arc (rounding put it either side)
        ang = math.atan2(pb[0] * qa[1] - pb[1] * qa[0], pb[0] * qa[0] + pb[1] * qa[1])
        if ang < 0.0:
            ang += 2.0 * math.pi
        area += 0.5 * ang
    return area


def ellipse_cell_area(i, j, X, Y, a, b, c, s):
    """Exact area of the ellipse within cell [i, i+1] x [j, j+1]: the map to
    the ellipse's unit-disk frame takes the cell to a parallelogram (same
    orientation, area scaled by 1 / (a b))."""
    corners = [(i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)]
    us, vs = [], []
    for (xa, ya) in corners:
        u, v = ellipse_frame(float(xa), float(ya), X, Y, a, b, c, s)
        us.append(u)
        vs.append(v)
    return a * b * polygon_unit_disk_area(us, vs)


def rasterise_shapes(nx, ny, X, Y, A, B, theta) -> Raster:
    """Solid-fraction field of a set of particles of which those with
    A[p] != B[p] are ellipses (semi-axes A >= B, major axis at angle
    theta[p]) and the others disks of radius A[p] (their cells exactly as
    `rasterise` gives them).  Owners in ascending particle order, at most 4,
    fractions scaled to sum 1 where they pass it."""
    X, Y = np.asarray(X, dtype=np.float64), np.asarray(Y, dtype=np.float64)
    A, B = np.asarray(A, dtype=np.float64), np.asarray(B, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    count = np.zeros((ny, nx), dtype=np.int64)
    owner = np.full((ny, nx, MAX_OWNERS), -1, dtype=np.int64)
    flag = np.zeros((ny, nx, MAX_OWNERS), dtype=np.int64)
    fsp = np.zeros((ny, nx, MAX_OWNERS), dtype=np.float64)
    for p in range(X.shape[0]):
        if A[p] == B[p]:
            one = rasterise(nx, ny, X[p:p + 1], Y[p:p + 1], A[p:p + 1])
            jj, ii = np.nonzero(one.count)
            cells = [(int(i), int(j), int(one.flag[j, i, 0]), float(one.fsp[j, i, 0])) for j, i in zip(jj, ii)]
        else:
            c, s = math.cos(theta[p]), math.sin(theta[p])
            i0, i1 = max(int(math.floor(X[p] - A[p])) - 1, 0), min(int(math.ceil(X[p] + A[p])) + 1, nx - 1)
            j0, j1 = max(int(math.floor(Y[p] - A[p])) - 1, 0), min(int(math.ceil(Y[p] + A[p])) + 1, ny - 1)
            cells = []
            for j in range(j0, j1 + 1):
                for i in range(i0, i1 + 1):
                    cls = ellipse_cell_class(i, j, X[p], Y[p], A[p], B[p], c, s)
                    if cls == FLUID:
                        continue
                    val = 1.0 if cls == SOLID else min(max(ellipse_cell_area(i, j, X[p], Y[p], A[p], B[p], c, s),
                                                           0.0), 1.0)
                    cells.append((i, j, cls, val))
        for i, j, cls, val in cells:
            k = count[j, i]
            if k >= MAX_OWNERS:
                raise OverflowError("more than 4 particles own one cell")
            owner[j, i, k] = p
            flag[j, i, k] = cls
            fsp[j, i, k] = val
            count[j, i] = k + 1
    tot = fsp.sum(axis=2)
    scale = np.where(tot > 1.0, 1.0 / np.where(tot > 1.0, tot, 1.0), 1.0)
    fsp = fsp * scale[:, :, None]
    return Raster(fs=fsp.sum(axis=2), count=count, owner=owner, flag=flag, fsp=fsp)


# --------------------------------------------------------------------------
# Volumetric correction and momentum exchange (Eqs. 8, 27, 28).
# --------------------------------------------------------------------------


def solid_velocity(xc, yc, Ux, Uy, Om, Xc, Yc):
    """Rigid-body velocity u_s(x) = U_c + Omega_c x (x - X_c) of Eq. 27 (2-D)."""
    return Ux - Om * (yc - Yc), Uy + Om * (xc - Xc)


def correct_and_exchange(fstar, ras: Raster, part):
    """Eq. 8 with several owners,
         f = (1 - sum_p f_s,p) f* + sum_p f_s,p f^eq(rho, u_s,p),
    rho = sum f*, and the per-particle force and torque of Eq. 28,
         F_p = - sum_x f_s,p sum_i [f_i^eq(rho, u_s,p) - f*_i] e_i,
         T_p = - sum_x (x - X_p) x f_s,p sum_i [f_i^eq - f*_i] e_i.
    Returns f, F (n, 2), T (n,)."""
    _, ny, nx = fstar.shape
    n = part["x"].shape[0]
    rho = fstar.sum(axis=0)
    f = (1.0 - ras.fs)[None] * fstar
    F = np.zeros((n, 2))
    T = np.zeros(n)
    for k in range(MAX_OWNERS):
        cj, ci = np.nonzero(ras.count > k)
        if cj.size == 0:
            continue
        p = ras.owner[cj, ci, k]
        w = ras.fsp[cj, ci, k]
        xc, yc = ci + 0.5, cj + 0.5
        usx, usy = solid_velocity(xc, yc, part["ux"][p], part["uy"][p], part["omega"][p],
                                  part["x"][p], part["y"][p])
        fe = feq(rho[cj, ci], usx, usy)                       # (9, ncell)
        f[:, cj, ci] += w[None] * fe
        d = fe - fstar[:, cj, ci]
        dFx = -w * np.tensordot(EX, d, axes=(0, 0))
        dFy = -w * np.tensordot(EY, d, axes=(0, 0))
        dT = (xc - part["x"][p]) * dFy - (yc - part["y"][p]) * dFx
        F[:, 0] += np.bincount(p, weights=dFx, minlength=n)
        F[:, 1] += np.bincount(p, weights=dFy, minlength=n)
        T += np.bincount(p, weights=dT, minlength=n)
    return f, F, T


# --------------------------------------------------------------------------
# Thermal LBE (Sec. 2.2): Eqs. 11, 17-25.
# --------------------------------------------------------------------------


def reference_cv(cv_f: float, cv_s: float) -> float:
    """c_v,ref: harmonic mean of the two specific heats (Sec. 2.2)."""
    return 2.0 * cv_f * cv_s / (cv_f + cv_s)


def thermal_eq_moments(eps, T, cref):
    """n^eq(eps, T) of Eq. 19."""
    z = np.zeros_like(eps * T)
    return np.stack([eps + z, -4.0 * eps + (4.0 + ALPHA1) * cref * T,
                     4.0 * eps - (4.0 - ALPHA2) * cref * T, z, z, z, z, z, z])


def source_moments(qc):
    """q_m of Eq. 20."""
    z = np.zeros_like(qc)
    return np.stack([qc, BETA1 * qc, BETA2 * qc, z, z, z, z, z, z])


def geq(eps, T, cref):
    """g^eq = M^-1 n^eq(eps, T) (definition below Eq. 18)."""
    return from_moments(thermal_eq_moments(eps, T, cref))


def fixed_temperature_correction(g, ras, T_p, fixed, cv_s, cref):
    """Particles held at their own temperature (Sec. 3.3, where the particle
    stays at the cold temperature T_c throughout).  fixed[p] = 1 (reading
    R11): in the part of a cell that such a particle covers, the thermal
    populations are replaced by the equilibrium at the particle's
    temperature, in the volumetric form of Eq. 8:
        g = (1 - f_fix) g + sum_{p held} f_s,p g^eq(c_vs T_p, T_p),
    f_fix = sum_{p held} f_s,p.  fixed[p] = 2 (reading R11b): every cell the
    particle owns takes that equilibrium whole (weight 1 in place of f_s,p;
    weights summing above 1 are scaled to 1).  Particles not held
    (fixed[p] = 0) keep the conjugate treatment."""
    fixed = np.asarray(fixed).astype(np.int64)
    ffix = np.zeros(g.shape[1:])
    acc = np.zeros_like(g)
    for k in range(MAX_OWNERS):
        sel = ras.count > k
        if not sel.any():
            continue
        own = np.where(sel, ras.owner[:, :, k], 0)
        mode = np.where(sel, fixed[own], 0)
        w = np.where(mode == 1, ras.fsp[:, :, k], np.where(mode == 2, 1.0, 0.0))
        if not w.any():
            continue
        Tp = T_p[own]
        ffix = ffix + w
        acc = acc + w * geq(cv_s * Tp, Tp, cref)
    over = ffix > 1.0
    acc = np.where(over[None], acc / np.where(over, ffix, 1.0)[None], acc)
    ffix = np.minimum(ffix, 1.0)
    return (1.0 - ffix) * g + acc


def tau_g_of(lam, cref, rho_f=1.0):
    """tau_g from Eq. 22: lambda / rho_f = (4 + alpha1)/6 c_ref (tau_g - 1/2)."""
    return 0.5 + 6.0 * lam / ((4.0 + ALPHA1) * rho_f * cref)


def thermal_rates(tau_g, mode: int = 0):
    """Diagonal of R (Eq. 18) per cell.  Sec. 3: sigma_0 = 1,
    sigma_eps = sigma_e, sigma_q = sigma_j = 1/tau_g and
    (1/sigma_j - 1/2)(1/sigma_e - 1/2) = 1/4 (mode 0); Sec. 3.5:
    sigma_0 = sigma_eps = sigma_e = 1 (mode 1)."""
    sj = 1.0 / tau_g
    if mode == 0:
        se = 1.0 / (0.5 + 0.25 / (tau_g - 0.5))
    else:
        se = np.ones_like(tau_g)
    one = np.ones_like(tau_g)
    return np.stack([one, se, se, sj, sj, sj, sj, se, se])


def collide_thermal(g, eps, T, qc, Rdiag, cref):
    """Post-collision gbar from Eq. 17a:
    nbar = n - R (n - n^eq) + (I - R/2) q_m."""
    n = to_moments(g)
    neq = thermal_eq_moments(eps, T, cref)
    qm = source_moments(qc)
    nbar = n - Rdiag * (n - neq) + (1.0 - 0.5 * Rdiag) * qm
    return from_moments(nbar)


def dfs_dt_update(fs_new, fs_old, dfs_old):
    """[df_s/dt](t + dt) = 2 (f_s(t + dt) - f_s(t)) - [df_s/dt](t)  (Eq. 24)."""
    return 2.0 * (fs_new - fs_old) - dfs_old


def temperature_gradient(g, cref, tau_g):
    """Local gradient scheme of Eq. 23:
    grad T = -6/(4 + alpha1) * sum_i e_i g_i / (c_ref tau_g)."""
    k = -6.0 / (4.0 + ALPHA1)
    gx = k * np.tensordot(EX, g, axes=(0, 0)) / (cref * tau_g)
    gy = k * np.tensordot(EY, g, axes=(0, 0)) / (cref * tau_g)
    return gx, gy


def temperature_prescribed_u(G, cv, cv_f, cv_s, dfs, ux, uy, gTx, gTy):
    """Eq. 25 with a given velocity field:
    T = (sum g - 1/2 c_v u.grad T) / (c_v - 1/2 (c_vs - c_vf) df_s/dt)."""
    return (G - 0.5 * cv * (ux * gTx + uy * gTy)) / (cv - 0.5 * (cv_s - cv_f) * dfs)


def temperature_and_velocity(G, cv, cv_f, cv_s, dfs, rho, jx, jy, fs, bx, by, T_ref, gTx, gTy):
    """Eq. 25 solved jointly with Eq. 9 when the buoyancy force
    F = (1 - f_s) b (T - T_ref), b = -rho_f beta g, depends on T (reading R4).

    With u = u0 + a (T - T_ref), u0 = j/rho, a = (1 - f_s) b / (2 rho),
    Eq. 25 reads T D = G - 1/2 c_v (u0 + a (T - T_ref)).grad T with
    D = c_v - 1/2 (c_vs - c_vf) df_s/dt, which is linear in T."""
    D = cv - 0.5 * (cv_s - cv_f) * dfs
    u0x, u0y = jx / rho, jy / rho
    ax, ay = (1.0 - fs) * bx / (2.0 * rho), (1.0 - fs) * by / (2.0 * rho)
    num = G - 0.5 * cv * ((u0x - ax * T_ref) * gTx + (u0y - ay * T_ref) * gTy)
    den = D + 0.5 * cv * (ax * gTx + ay * gTy)
    T = num / den
    ux = u0x + ax * (T - T_ref)
    uy = u0y + ay * (T - T_ref)
    Fx = (1.0 - fs) * bx * (T - T_ref)
    Fy = (1.0 - fs) * by * (T - T_ref)
    return T, ux, uy, Fx, Fy


def source_term(cv, cv_f, cv_s, ux, uy, gTx, gTy, T, dfs):
    """q_c = -c_v u.grad T + (c_vs - c_vf) T df_s/dt (Eq. 16)."""
    return -cv * (ux * gTx + uy * gTy) + (cv_s - cv_f) * T * dfs


# --------------------------------------------------------------------------
# Particle dynamics (Sec. 2.3): Eqs. 26, 29, 30 and contact (reading R5).
# --------------------------------------------------------------------------


def contact_pairs(X, Y, R, zeta):
    """All pairs i < j with d_ij < R_i + R_j + zeta, ascending (brute force)."""
    n = len(X)
    pairs = []
    for i in range(n):
        for j in range(i + 1, n):
            dx = X[i] - X[j]
            dy = Y[i] - Y[j]
            thr = R[i] + R[j] + zeta
            if dx * dx + dy * dy < thr * thr:
                pairs.append((i, j))
    return pairs


def contact_forces(X, Y, R, prm, pairs, semi_minor=None, theta=None):
    """Contact force on each particle (reading R5); partners are summed in
    ascending id, then walls x-, x+, y-, y+.  An ellipse (semi_minor < R, the
    semi-major axis; major axis at angle theta) meets another particle as its
    circumscribed disk and a wall by its extent along the wall's normal,
    sqrt(a^2 cos^2 + b^2 sin^2) of the angle between major axis and normal
    (reading R13)."""
    n = len(X)
    zeta = prm.contact_range
    gmag = math.hypot(prm.gravity[0], prm.gravity[1])
    scale = abs(prm.rho_ratio - 1.0) * 1.0 * gmag * math.pi
    partners = [[] for _ in range(n)]
    for i, j in pairs:
        partners[i].append(j)
        partners[j].append(i)
    F = np.zeros((n, 2))
    for i in range(n):
        for j in sorted(partners[i]):
            dx = X[i] - X[j]
            dy = Y[i] - Y[j]
            d = math.sqrt(dx * dx + dy * dy)
            gap = R[i] + R[j] + zeta - d
            if gap <= 0.0:
                continue
            c = scale * max(R[i], R[j]) ** 2
            mag = (c / prm.contact_eps_p) * (gap / zeta) ** 2 / d
            F[i, 0] += mag * dx
            F[i, 1] += mag * dy
        c = scale * R[i] ** 2
        walls = [(0, X[i] - 0.0, 1.0, 0.0), (0, prm.nx - X[i], -1.0, 0.0),
                 (1, Y[i] - 0.0, 0.0, 1.0), (1, prm.ny - Y[i], 0.0, -1.0)]
        ext = [R[i], R[i]]  # extent along x and along y
        if semi_minor is not None and semi_minor[i] != R[i]:
            a, b = R[i], semi_minor[i]
            cth, sth = math.cos(theta[i]), math.sin(theta[i])
            ext = [math.sqrt(a * a * cth * cth + b * b * sth * sth), math.sqrt(a * a * sth * sth + b * b * cth * cth)]
        for axis, dist, nxw, nyw in walls:
            if prm.periodic[axis]:
                continue
            if prm.outflow[2 * axis + (0 if (nxw > 0 or nyw > 0) else 1)]:
                continue  # no wall on an open side
            d = 2.0 * dist
            gap = 2.0 * ext[axis] + zeta - d
            if gap <= 0.0:
                continue
            mag = (c / prm.contact_eps_w) * (gap / zeta) ** 2
            F[i, 0] += mag * nxw
            F[i, 1] += mag * nyw
    return F


# --------------------------------------------------------------------------
# Parameters and the coupled time step.
# --------------------------------------------------------------------------


@dataclasses.dataclass
class Params:
    """Problem statement in lattice units (Sec. 3; rho_f = c_vf = 1)."""
    nx: int
    ny: int
    tau_f: float = 0.8
    lambda_q_flow: float = 1.0 / 12.0
    s_e: float = 1.25
    prandtl: float = 0.7
    rho_ratio: float = 1.5
    cv_ratio: float = 1.0
    k_ratio_default: float = 1.0
    gravity: tuple = (0.0, 0.0)
    beta: float = 0.0
    T_ref: float = 1.0
    T_fluid_init: float = 1.0
    thermal_wall: tuple = (0, 0, 0, 0)   # 0 adiabatic, 1 held at wall_T
    wall_T: tuple = (0.0, 0.0, 0.0, 0.0)
    thermal_rates_mode: int = 0
    contact_range: float = 2.0
    contact_eps_p: float = 0.01
    contact_eps_w: float = 0.005
    periodic: tuple = (False, False)
    outflow: tuple = (False, False, False, False)  # open sides x-, x+, y-, y+ (reading R14)

    # derived quantities (Sec. 3)
    @property
    def nu(self):
        return (self.tau_f - 0.5) / 3.0

    @property
    def cv_f(self):
        return 1.0

    @property
    def cv_s(self):
        return self.cv_ratio

    @property
    def lambda_f(self):
        return 1.0 * self.cv_f * self.nu / self.prandtl

    @property
    def cref(self):
        return reference_cv(self.cv_f, self.cv_s)


class Simulation:
    """The coupled step of Sec. 2, phase by phase.

    State at level n: post-correction f, g; rho, u, F, T, eps, q_c; f_s^n
    with its owners; [df_s/dt]^n; per particle X, theta, U, Omega, the
    previous U, Omega and the hydrodynamic force and torque of level n."""

    def __init__(self, prm: Params, x, y, radius, T0, k_ratio=None, ux=None, uy=None, omega=None,
                 fixed_T=None, semi_minor=None, theta=None):
        self.prm = prm
        n = len(x)
        z = np.zeros(n)
        # particles held at their initial temperature T0: 1 reading R11, 2 R11b
        self.fixed_T = np.array(fixed_T if fixed_T is not None else np.zeros(n), dtype=np.int64)
        self.part = {
            "x": np.array(x, dtype=float), "y": np.array(y, dtype=float),
            "r": np.array(radius, dtype=float), "T0": np.array(T0, dtype=float),
            "k": np.array(k_ratio if k_ratio is not None else np.full(n, prm.k_ratio_default), dtype=float),
            "ux": np.array(ux if ux is not None else z, dtype=float),
            "uy": np.array(uy if uy is not None else z, dtype=float),
            "omega": np.array(omega if omega is not None else z, dtype=float),
            "theta": np.array(theta if theta is not None else z, dtype=float),
        }
        # semi-minor axes: an ellipse where it differs from the radius (the
        # semi-major axis), a disk where it equals it (reading R13)
        self.part["b"] = np.array(semi_minor if semi_minor is not None else radius, dtype=float)
        self.part["ux_prev"] = self.part["ux"].copy()
        self.part["uy_prev"] = self.part["uy"].copy()
        self.part["omega_prev"] = self.part["omega"].copy()
        self._set_inertia()
        self.S = flow_rates(prm.tau_f, prm.lambda_q_flow, prm.s_e)
        self.b = (-1.0 * prm.beta * prm.gravity[0], -1.0 * prm.beta * prm.gravity[1])
        self.step_count = 0
        self._init_state()

    # -- helpers ------------------------------------------------------------
    def _set_inertia(self):
        """Mass and moment of inertia of each particle and of its inside fluid
        (Sec. 2.3): an ellipse of semi-axes a, b has area pi a b and polar
        moment M (a^2 + b^2) / 4 (a disk: M R^2 / 2)."""
        a, b = self.part["r"], self.part["b"]
        area = math.pi * a * b
        self.area = area
        self.mass = self.prm.rho_ratio * area                  # M
        self.inertia = 0.25 * self.mass * (a * a + b * b)      # I_c
        self.mass_in = 1.0 * area                              # M_in = rho_f M / rho_s
        self.inertia_in = 0.25 * self.mass_in * (a * a + b * b)  # I_c,in

    def _properties(self, ras: Raster):
        """c_v and lambda of Eq. 11, summed over owners."""
        p = self.prm
        cv = (1.0 - ras.fs) * p.cv_f
        lam = (1.0 - ras.fs) * p.lambda_f
        for k in range(MAX_OWNERS):
            sel = ras.count > k
            if not sel.any():
                continue
            w = np.where(sel, ras.fsp[:, :, k], 0.0)
            kp = self.part["k"][np.where(sel, ras.owner[:, :, k], 0)]
            cv = cv + w * p.cv_s
            lam = lam + w * kp * p.lambda_f
        return cv, lam

    def _raster(self):
        p = self.prm
        P = self.part
        if (P["b"] != P["r"]).any():
            return rasterise_shapes(p.nx, p.ny, P["x"], P["y"], P["r"], P["b"], P["theta"])
        return rasterise(p.nx, p.ny, P["x"], P["y"], P["r"])

    def _init_state(self):
        """Initial state (reading R6)."""
        p = self.prm
        ny, nx = p.ny, p.nx
        self.ras = self._raster()
        ones = np.ones((ny, nx))
        fstar = feq(ones, 0.0 * ones, 0.0 * ones)
        self.f, self.F_mes, self.T_mes = correct_and_exchange(fstar, self.ras, self.part)
        self.cv, lam = self._properties(self.ras)
        self.tau_g = tau_g_of(lam, p.cref)
        eps = (1.0 - self.ras.fs) * p.cv_f * p.T_fluid_init
        for k in range(MAX_OWNERS):
            sel = self.ras.count > k
            if sel.any():
                Tp = self.part["T0"][np.where(sel, self.ras.owner[:, :, k], 0)]
                eps = eps + np.where(sel, self.ras.fsp[:, :, k], 0.0) * p.cv_s * Tp
        self.eps = eps
        self.T = eps / self.cv
        self.qc = np.zeros((ny, nx))
        self.dfs = np.zeros((ny, nx))
        self.g = geq(self.eps, self.T, p.cref)
        rho = self.f.sum(axis=0)
        jx = np.tensordot(EX, self.f, axes=(0, 0))
        jy = np.tensordot(EY, self.f, axes=(0, 0))
        self.Fx = (1.0 - self.ras.fs) * self.b[0] * (self.T - p.T_ref)
        self.Fy = (1.0 - self.ras.fs) * self.b[1] * (self.T - p.T_ref)
        self.rho = rho
        self.ux = (jx + 0.5 * self.Fx) / rho
        self.uy = (jy + 0.5 * self.Fy) / rho
        self.Fc = np.zeros((len(self.part["x"]), 2))
        self.Tc = np.zeros(len(self.part["x"]))
        self.pairs = contact_pairs(self.part["x"], self.part["y"], self.part["r"], p.contact_range)

    def _particle_update(self):
        """Eqs. 26, 29, 30 by forward Euler with backward differences for
        dU/dt and dOmega/dt in F_in, T_in (end of Sec. 2.3)."""
        p = self.prm
        P = self.part
        r = P["r"]
        Fcon = contact_forces(P["x"], P["y"], r, p, self.pairs, semi_minor=P["b"], theta=P["theta"])
        body = (p.rho_ratio - 1.0) * 1.0 * self.area
        F_in_x = -self.mass_in * (P["ux"] - P["ux_prev"])
        F_in_y = -self.mass_in * (P["uy"] - P["uy_prev"])
        T_in = -self.inertia_in * (P["omega"] - P["omega_prev"])
        Fcx = self.F_mes[:, 0] - F_in_x + body * p.gravity[0] + Fcon[:, 0]
        Fcy = self.F_mes[:, 1] - F_in_y + body * p.gravity[1] + Fcon[:, 1]
        Tc = self.T_mes - T_in
        self.Fc = np.stack([Fcx, Fcy], axis=1)
        self.Tc = Tc
        ux_new = P["ux"] + Fcx / self.mass
        uy_new = P["uy"] + Fcy / self.mass
        om_new = P["omega"] + Tc / self.inertia
        P["x"] = P["x"] + P["ux"]
        P["y"] = P["y"] + P["uy"]
        P["theta"] = P["theta"] + P["omega"]
        P["ux_prev"], P["uy_prev"], P["omega_prev"] = P["ux"], P["uy"], P["omega"]
        P["ux"], P["uy"], P["omega"] = ux_new, uy_new, om_new

    def insert_particles(self, x, y, radius, T0, k_ratio=None, ux=None, uy=None, omega=None):
        """Disks added at the current level (mid-run insertion; reading R12):
        they join the particle set with the given centre and velocity and
        first appear in the raster of the next level, where the correction
        (Eq. 8) and the df_s/dt recursion (Eq. 24) act on them as on any disk
        moving into cells; their first update has no exchange and no contact
        force (neither was formed at this level)."""
        n = len(x)
        z = np.zeros(n)
        P = self.part
        new = {"x": x, "y": y, "r": radius, "T0": T0,
               "k": k_ratio if k_ratio is not None else np.full(n, self.prm.k_ratio_default),
               "ux": ux if ux is not None else z, "uy": uy if uy is not None else z,
               "omega": omega if omega is not None else z, "theta": z}
        for key, v in new.items():
            P[key] = np.concatenate([P[key], np.asarray(v, dtype=float)])
        P["b"] = np.concatenate([P["b"], np.asarray(radius, dtype=float)])  # inserted particles are disks
        P["ux_prev"] = np.concatenate([P["ux_prev"], np.asarray(new["ux"], dtype=float)])
        P["uy_prev"] = np.concatenate([P["uy_prev"], np.asarray(new["uy"], dtype=float)])
        P["omega_prev"] = np.concatenate([P["omega_prev"], np.asarray(new["omega"], dtype=float)])
        self._set_inertia()
        self.fixed_T = np.concatenate([self.fixed_T, np.zeros(n, dtype=np.int64)])
        self.F_mes = np.concatenate([self.F_mes, np.zeros((n, 2))])
        self.T_mes = np.concatenate([self.T_mes, z])
        self.Fc = np.concatenate([self.Fc, np.zeros((n, 2))])
        self.Tc = np.concatenate([self.Tc, z])

    def step(self, nsteps: int = 1):
        for _ in range(nsteps):
            self._step()

    def _step(self):
        p = self.prm
        # (1) collisions at level n (Eqs. 3a, 17a)
        fbar = collide_flow(self.f, self.rho, self.ux, self.uy, self.Fx, self.Fy, self.S)
        Rd = thermal_rates(self.tau_g, p.thermal_rates_mode)
        gbar = collide_thermal(self.g, self.eps, self.T, self.qc, Rd, p.cref)
        # (2) streaming (Eqs. 3b, 17b)
        fstar = stream_flow(fbar, p.periodic, p.outflow)
        g = stream_thermal(gbar, p.cref, p.thermal_wall, p.wall_T, p.periodic, p.outflow)
        # (3) particle motion to level n+1 (reading R3), then f_s^{n+1}
        self._particle_update()
        fs_old = self.ras.fs
        self.ras = self._raster()
        # (4) volumetric correction and momentum exchange (Eqs. 8, 28)
        self.f, self.F_mes, self.T_mes = correct_and_exchange(fstar, self.ras, self.part)
        if self.fixed_T.any():
            g = fixed_temperature_correction(g, self.ras, self.part["T0"], self.fixed_T, p.cv_s, p.cref)
        # (5) thermal macroscopics at n+1 (Eqs. 11, 21-25) jointly with rho, u (Eq. 9)
        self.dfs = dfs_dt_update(self.ras.fs, fs_old, self.dfs)
        self.cv, lam = self._properties(self.ras)
        self.tau_g = tau_g_of(lam, p.cref)
        gTx, gTy = temperature_gradient(g, p.cref, self.tau_g)
        G = g.sum(axis=0)
        rho = self.f.sum(axis=0)
        jx = np.tensordot(EX, self.f, axes=(0, 0))
        jy = np.tensordot(EY, self.f, axes=(0, 0))
        T, ux, uy, Fx, Fy = temperature_and_velocity(
            G, self.cv, p.cv_f, p.cv_s, self.dfs, rho, jx, jy, self.ras.fs,
            self.b[0], self.b[1], p.T_ref, gTx, gTy)
        self.g = g
        self.rho, self.ux, self.uy, self.Fx, self.Fy, self.T = rho, ux, uy, Fx, Fy, T
        self.eps = self.cv * T
        self.qc = source_term(self.cv, p.cv_f, p.cv_s, ux, uy, gTx, gTy, T, self.dfs)
        self.pairs = contact_pairs(self.part["x"], self.part["y"], self.part["r"], p.contact_range)
        self.step_count += 1

    # -- outputs -------------------------------------------------------------
    def fields(self):
        return {"rho": self.rho, "ux": self.ux, "uy": self.uy, "T": self.T, "fs": self.ras.fs}

    def particle_state(self):
        P = self.part
        return {"x": P["x"].copy(), "y": P["y"].copy(), "theta": P["theta"].copy(),
                "ux": P["ux"].copy(), "uy": P["uy"].copy(), "omega": P["omega"].copy(),
                "fx": self.Fc[:, 0].copy(), "fy": self.Fc[:, 1].copy(), "torque": self.Tc.copy()}

    def audit(self):
        """Total mass sum f, total internal energy sum eps and sum g."""
        return float(self.f.sum()), float(self.eps.sum()), float(self.g.sum())


class PrescribedFlowThermal:
    """The thermal LBE of Sec. 2.2 on its own, with the velocity field and
    the solid fraction given in advance (the setting of Sec. 3.1, where
    "only the LB equation for temperature field is involved").

    ``fs_of(t)`` returns the solid-fraction field at time t; the velocity is
    uniform.  Properties follow Eq. 11 with c_vf = 1, lambda_s = R_lambda
    lambda_f, c_vs = R_cv."""

    def __init__(self, nx, ny, lambda_f, R_lambda, R_cv, fs_of, T_solid, T_fluid, velocity=(0.0, 0.0),
                 thermal_wall=(0, 0, 0, 0), wall_T=(0.0, 0.0, 0.0, 0.0), periodic=(False, True), mode=0):
        self.nx, self.ny = nx, ny
        self.lambda_f, self.lambda_s = lambda_f, R_lambda * lambda_f
        self.cv_f, self.cv_s = 1.0, R_cv
        self.cref = reference_cv(self.cv_f, self.cv_s)
        self.fs_of = fs_of
        self.u = velocity
        self.walls, self.wall_T, self.periodic, self.mode = thermal_wall, wall_T, periodic, mode
        self.t = 0
        self.fs = fs_of(0)
        self.dfs = np.zeros((ny, nx))
        self.cv, self.tau_g = self._props(self.fs)
        self.T = np.where(self.fs > 0.5, T_solid, T_fluid) * np.ones((ny, nx))
        self.eps = self.cv * self.T
        self.qc = np.zeros((ny, nx))
        self.g = geq(self.eps, self.T, self.cref)

    def _props(self, fs):
        cv = (1.0 - fs) * self.cv_f + fs * self.cv_s
        lam = (1.0 - fs) * self.lambda_f + fs * self.lambda_s
        return cv, tau_g_of(lam, self.cref)

    def step(self, nsteps=1):
        for _ in range(nsteps):
            Rd = thermal_rates(self.tau_g, self.mode)
            gbar = collide_thermal(self.g, self.eps, self.T, self.qc, Rd, self.cref)
            g = stream_thermal(gbar, self.cref, self.walls, self.wall_T, self.periodic)
            self.t += 1
            fs_new = self.fs_of(self.t)
            self.dfs = dfs_dt_update(fs_new, self.fs, self.dfs)
            self.fs = fs_new
            self.cv, self.tau_g = self._props(fs_new)
            gTx, gTy = temperature_gradient(g, self.cref, self.tau_g)
            ux = np.full_like(fs_new, self.u[0])
            uy = np.full_like(fs_new, self.u[1])
            self.T = temperature_prescribed_u(g.sum(axis=0), self.cv, self.cv_f, self.cv_s, self.dfs,
                                              ux, uy, gTx, gTy)
            self.eps = self.cv * self.T
            self.qc = source_term(self.cv, self.cv_f, self.cv_s, ux, uy, gTx, gTy, self.T, self.dfs)
            self.g = g


def slab_fraction(nx, ny, X_interface):
    """f_s of a solid filling x < X_interface (one-dimensional slab)."""
    i = np.arange(nx, dtype=np.float64)
    return np.broadcast_to(np.clip(X_interface - i, 0.0, 1.0), (ny, nx)).copy()


def conjugate_erfc(x, t, X_i, T_h, T_c, lambda_f, R_lambda, R_cv):
    """Closed form of the 1-D transient conjugate problem, Eq. 31 (solid at
    x < X_i initially at T_h, fluid initially at T_c, rho_f = c_vf = 1)."""
    a_s = R_lambda * lambda_f / R_cv
    a_f = lambda_f / 1.0
    e = math.sqrt(R_lambda * R_cv)
    x = np.asarray(x, dtype=np.float64)
    erfc = np.vectorize(math.erfc)
    solid = T_h + (T_c - T_h) / (e + 1.0) * erfc((X_i - x) / (2.0 * math.sqrt(a_s * t)))
    fluid = T_c + (T_h - T_c) * e / (e + 1.0) * erfc((x - X_i) / (2.0 * math.sqrt(a_f * t)))
    return np.where(x < X_i, solid, fluid)


# ---------------------------------------------------------------------------
# The C ABI's entry points over the oracle: the names of include/vlb.h with
# vlbref_ for vlb_, the same inputs in the same order and the same status
# codes, so that one script can drive either side.  Outputs the C ABI writes
# through caller-owned arrays are written into caller-owned numpy arrays of
# the same layout (fields row-major with y slow; xy, uv, force interleaved);
# out-scalars are returned after the status.
# ---------------------------------------------------------------------------
VLBREF_OK, VLBREF_EINVAL, VLBREF_ESTATE = 0, -1, -4
VLBREF_FIELD_RHO, VLBREF_FIELD_UX, VLBREF_FIELD_UY, VLBREF_FIELD_T, VLBREF_FIELD_FS = 1, 2, 4, 8, 16


def _inside(prm, x, y, r):
    """A disk lies inside the walls; on a periodic axis it keeps R + 1 from
    the boundary (reading R7)."""
    mx = r + 1.0 if prm.periodic[0] else r
    my = r + 1.0 if prm.periodic[1] else r
    return r > 0 and mx <= x <= prm.nx - mx and my <= y <= prm.ny - my


def _min_image(d, L, periodic):
    """Separation along an axis of length L; the nearest image on a
    periodic axis."""
    if not periodic:
        return d
    return np.where(d > 0.5 * L, d - L, np.where(d < -0.5 * L, d + L, d)) if isinstance(d, np.ndarray) else (
        d - L if d > 0.5 * L else (d + L if d < -0.5 * L else d))


class _RefHandle:
    def __init__(self, prm: Params):
        self.prm = prm
        self.parts = {k: [] for k in ("x", "y", "r", "T0", "k", "ux", "uy", "omega", "fixed", "b", "theta")}
        self.sim = None
        self.err = ""

    def fail(self, status, msg):
        self.err = msg
        return status


def vlbref_create(p: Params):
    """(status, handle) for the problem p."""
    if p.nx < 2 or p.ny < 2 or not p.tau_f > 0.5:
        return VLBREF_EINVAL, None
    return VLBREF_OK, _RefHandle(p)


def vlbref_add_particles(h, n, xy, radius, T0, k_ratio=None, uv=None, omega=None):
    """Disks before the first step: centres xy[2n], radii, initial
    temperatures, optional conductivity ratios, velocities uv[2n], spins.
    VLBREF_EINVAL for a disk outside the walls or overlapping another."""
    if h.sim is not None:
        return h.fail(VLBREF_ESTATE, "particles must be added before the first step")
    xy = np.asarray(xy, dtype=float).reshape(-1)
    P = h.parts
    for k in range(n):
        x, y, r = float(xy[2 * k]), float(xy[2 * k + 1]), float(radius[k])
        if not _inside(h.prm, x, y, r):
            return h.fail(VLBREF_EINVAL, "a disk lies outside the walls or across a periodic boundary")
        for x2, y2, r2 in zip(P["x"], P["y"], P["r"]):
            dx, dy = _min_image(x - x2, h.prm.nx, h.prm.periodic[0]), _min_image(y - y2, h.prm.ny, h.prm.periodic[1])
            if dx ** 2 + dy ** 2 < (r + r2) ** 2:
                return h.fail(VLBREF_EINVAL, "particles overlap")
        P["x"].append(x)
        P["y"].append(y)
        P["r"].append(r)
        P["T0"].append(float(T0[k]))
        P["k"].append(float(k_ratio[k]) if k_ratio is not None else h.prm.k_ratio_default)
        P["ux"].append(float(uv[2 * k]) if uv is not None else 0.0)
        P["uy"].append(float(uv[2 * k + 1]) if uv is not None else 0.0)
        P["omega"].append(float(omega[k]) if omega is not None else 0.0)
        P["fixed"].append(0)
        P["b"].append(r)
        P["theta"].append(0.0)
    return VLBREF_OK


def vlbref_add_ellipses(h, n, xy, semi_a, semi_b, theta, T0, k_ratio=None, uv=None, omega=None):
    """Elliptical particles before the first step (reading R13): centres
    xy[2n], semi-axes semi_a >= semi_b > 0, major-axis angles theta (radians
    from the x axis), then as vlbref_add_particles.  A particle with
    semi_a == semi_b is a disk.  VLBREF_EINVAL for a particle outside the walls
    (judged by its circumscribed disk) or whose circumscribed disk overlaps
    another's."""
    xy = np.asarray(xy, dtype=float).reshape(-1)
    for k in range(n):
        if not (semi_a[k] >= semi_b[k] > 0.0):
            return h.fail(VLBREF_EINVAL, "semi-axes must satisfy semi_a >= semi_b > 0")
    n0 = len(h.parts["x"])
    st = vlbref_add_particles(h, n, xy, semi_a, T0, k_ratio, uv, omega)
    if st != VLBREF_OK:
        return st
    for k in range(n):
        h.parts["b"][n0 + k] = float(semi_b[k])
        h.parts["theta"][n0 + k] = float(theta[k])
    return VLBREF_OK


def vlbref_set_fixed_temperature(h, first, n, held):
    """Hold particles first .. first + n - 1 at T0 (held[k] != 0), before the first step."""
    if h.sim is not None:
        return h.fail(VLBREF_ESTATE, "fixed temperatures must be set before the first step")
    if first < 0 or n < 0 or first + n > len(h.parts["x"]):
        return h.fail(VLBREF_EINVAL, "particle range")
    for k in range(n):
        h.parts["fixed"][first + k] = int(held[k]) if held[k] in (0, 1, 2) else 1
    return VLBREF_OK


def _ensure(h):
    if h.sim is None:
        P = h.parts
        h.sim = Simulation(h.prm, P["x"], P["y"], P["r"], P["T0"], k_ratio=P["k"], ux=P["ux"], uy=P["uy"],
                           omega=P["omega"], fixed_T=P["fixed"], semi_minor=P["b"], theta=P["theta"])


def vlbref_insert_particles(h, n, xy, radius, T0, k_ratio=None, uv=None, omega=None):
    """Disks between two steps (before the first one: vlbref_add_particles)."""
    if h.sim is None:
        return vlbref_add_particles(h, n, xy, radius, T0, k_ratio, uv, omega)
    xy = np.asarray(xy, dtype=float).reshape(-1)
    uv = None if uv is None else np.asarray(uv, dtype=float).reshape(-1)
    P = h.sim.part
    for k in range(n):
        x, y, r = float(xy[2 * k]), float(xy[2 * k + 1]), float(radius[k])
        if not _inside(h.prm, x, y, r):
            return h.fail(VLBREF_EINVAL, "a disk lies outside the walls or across a periodic boundary")
        dx = _min_image(P["x"] - x, h.prm.nx, h.prm.periodic[0])
        dy = _min_image(P["y"] - y, h.prm.ny, h.prm.periodic[1])
        if (dx ** 2 + dy ** 2 < (P["r"] + r) ** 2).any():
            return h.fail(VLBREF_EINVAL, "particles overlap")
        for j in range(k):
            dx = _min_image(x - float(xy[2 * j]), h.prm.nx, h.prm.periodic[0])
            dy = _min_image(y - float(xy[2 * j + 1]), h.prm.ny, h.prm.periodic[1])
            if dx ** 2 + dy ** 2 < (r + float(radius[j])) ** 2:
                return h.fail(VLBREF_EINVAL, "particles overlap")
    h.sim.insert_particles(xy[0:2 * n:2], xy[1:2 * n:2], list(radius[:n]), list(T0[:n]),
                           k_ratio=None if k_ratio is None else list(k_ratio[:n]),
                           ux=None if uv is None else uv[0:2 * n:2], uy=None if uv is None else uv[1:2 * n:2],
                           omega=None if omega is None else list(omega[:n]))
    return VLBREF_OK


def vlbref_step(h, nsteps):
    """nsteps time steps (the initial state is built by the first call)."""
    if nsteps < 0:
        return h.fail(VLBREF_EINVAL, "nsteps < 0")
    _ensure(h)
    h.sim.step(nsteps)
    return VLBREF_OK


def vlbref_get_fields(h, mask, rho, ux, uy, T, fs):
    """rho, u, T, f_s of the current level into the arrays whose bit is set in mask."""
    _ensure(h)
    f = h.sim.fields()
    for bit, name, out in ((1, "rho", rho), (2, "ux", ux), (4, "uy", uy), (8, "T", T), (16, "fs", fs)):
        if mask & bit:
            if out is None:
                return h.fail(VLBREF_EINVAL, "NULL field array for a selected field")
            np.copyto(np.asarray(out).reshape(h.prm.ny, h.prm.nx), f[name])
    return VLBREF_OK


def vlbref_get_particle_count(h):
    return VLBREF_OK, len(h.parts["x"])


def vlbref_get_particle_state(h, n, xy, theta, uv, omega, force, torque):
    """State of the first n particles: centres, angles, velocities, spins, F_c, T_c."""
    _ensure(h)
    s = h.sim.particle_state()
    if n > len(s["x"]):
        return h.fail(VLBREF_EINVAL, "n exceeds the particle count")
    for out, parts in ((xy, ("x", "y")), (uv, ("ux", "uy")), (force, ("fx", "fy"))):
        if out is not None:
            o = np.asarray(out).reshape(-1)
            o[0:2 * n:2], o[1:2 * n:2] = s[parts[0]][:n], s[parts[1]][:n]
    for out, name in ((theta, "theta"), (omega, "omega"), (torque, "torque")):
        if out is not None:
            np.asarray(out).reshape(-1)[:n] = s[name][:n]
    return VLBREF_OK


def vlbref_get_audit(h):
    """(status, total mass, total internal energy, sum g)."""
    _ensure(h)
    return (VLBREF_OK,) + tuple(h.sim.audit())


def vlbref_get_step(h):
    return VLBREF_OK, (h.sim.step_count if h.sim is not None else 0)


def vlbref_last_error(h):
    return h.err if h is not None else ""


def vlbref_destroy(h):
    if h is not None:
        h.sim = None
