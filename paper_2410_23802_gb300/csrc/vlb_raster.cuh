// Solid fraction of a disk in one lattice cell (Sec. 2: f_s is the volume
// fraction of solid in the cell, fixed by the particle position).
//
// Classification (integer, identical on every device): a cell is SOLID when
// its four corners lie in the closed disk and FLUID when its nearest point is
// at distance >= R, tested on centres and radii rounded to a 2^-20 grid.
// INTERFACE cells get the exact area of disk ∩ cell, computed in cell-local
// coordinates as a polygon (the parts of the cell edges inside the disk) plus
// the circular segments between each chord and its arc -- all quantities are
// O(1), so FP32 keeps ~1e-7 absolute error.
#pragma once

#include <math.h>

#include "vlb_common.cuh"

namespace vlb {

__host__ __device__ __forceinline__ float vsqrt(float v) { return sqrtf(v); }
__host__ __device__ __forceinline__ double vsqrt(double v) { return sqrt(v); }

// Products and sums rounded one by one (no contraction into FMA), so that a
// test gives the same answer in every kernel that makes it.
__host__ __device__ __forceinline__ float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ float add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ double mul_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ double add_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dadd_rn(a, b);
#else
  return a + b;
#endif
}

enum : int { CELL_FLUID = 0, CELL_INTERFACE = 1, CELL_SOLID = 2 };

// An ellipse as the FP64 lattice kernel sees it (the FP32 kernel reads
// ellipses from their band tables and carries none of this).
template <class C>
struct EllPart {};
template <>
struct EllPart<double> {
  int ell;                        // an ellipse
  double ex, ey, ea, eb, ec, es;  // its centre, semi-axes, cos and sin of its angle
};

// One particle as seen from one tile (shared memory).  Coordinates are
// relative to the tile's lower-left corner.
template <class C>
struct PartTile : EllPart<C> {
  long long xq, yq, rq2;  // fixed-point centre and R^2 (2^-20 grid)
  C xh, xl, yh, yl;       // centre as an unevaluated sum hi + lo
  C r, far2, near2;       // radius, quick-reject bounds on the centre distance^2
  C ux, uy, om;           // rigid-body motion (Eq. 27)
  C uxl, uyl;             // low parts of U (U = ux + uxl to FP64 accuracy)
  C lam_s, T0;
  int id;                 // particle id
  int ci, cj;             // cell of the centre (band table origin)
  int fixed;              // held at T0: 1 covered part (reading R11), 2 whole cells (R11b)
  int rx, ry;             // first tile of the particle's range
};

// Integer classification of cell (il, jl) of the tile against one disk.
template <class C>
__host__ __device__ __forceinline__ int cell_class_exact(int il, int jl, const PartTile<C>& p) {
  const long long Q = 1ll << QBITS;
  const long long cx0 = (long long)il * Q - p.xq, cx1 = cx0 + Q;
  const long long cy0 = (long long)jl * Q - p.yq, cy1 = cy0 + Q;
  const long long fx = cx0 * cx0 > cx1 * cx1 ? cx0 * cx0 : cx1 * cx1;
  const long long fy = cy0 * cy0 > cy1 * cy1 ? cy0 * cy0 : cy1 * cy1;
  if (fx + fy <= p.rq2) return CELL_SOLID;
  const long long ax0 = cx0 < 0 ? -cx0 : cx0, ax1 = cx1 < 0 ? -cx1 : cx1;
  const long long ay0 = cy0 < 0 ? -cy0 : cy0, ay1 = cy1 < 0 ? -cy1 : cy1;
  const long long nx = (cx0 <= 0 && cx1 >= 0) ? 0 : (ax0 < ax1 ? ax0 : ax1);
  const long long ny = (cy0 <= 0 && cy1 >= 0) ? 0 : (ay0 < ay1 ? ay0 : ay1);
  if (nx * nx + ny * ny >= p.rq2) return CELL_FLUID;
  return CELL_INTERFACE;
}

// Area of the circular segment cut off by a chord of length L (L <= 2R):
// R^2 (asin z - z sqrt(1 - z^2)), z = L / (2R).
__host__ __device__ __forceinline__ double segment_area(double L, double R) {
  const double z = L / (2.0 * R);
  return R * R * (asin(z) - z * sqrt(fmax(1.0 - z * z, 0.0)));
}
__host__ __device__ __forceinline__ float segment_area(float L, float R) {
  const float z = L / (2.0f * R);
  if (z < 0.25f) {
    // Taylor series of asin z - z sqrt(1 - z^2):
    // 2/3 z^3 + 1/5 z^5 + 3/28 z^7 + 5/72 z^9 + 35/704 z^11 + O(z^13)
    const float z2 = z * z;
    float s = 35.0f / 704.0f;
    s = s * z2 + 5.0f / 72.0f;
    s = s * z2 + 3.0f / 28.0f;
    s = s * z2 + 0.2f;
    s = s * z2 + 2.0f / 3.0f;
    return R * R * s * z2 * z;
  }
  return R * R * (asinf(z) - z * sqrtf(fmaxf(1.0f - z * z, 0.0f)));
}

// Exact area of disk((cx, cy), R) ∩ [0,1]^2 (cell-local coordinates), R >= 1.
//
// Walking the square's boundary counter-clockwise, each edge meets the closed
// disk in one interval (possibly empty), found from that edge's own line.  The
// region's boundary is those intervals joined, between one interval's end and
// the next interval's start, by arcs of the circle; so the area is the polygon
// of the interval end points plus, for every such link, the circular segment
// on its chord.  No entry/exit decision is taken: when rounding puts a circle
// point on one or the other side of a corner, the link's chord is just tiny
// and so is its segment.
template <class C>
__host__ __device__ __forceinline__ C disk_unit_cell_area(C cx, C cy, C R) {
  // The polygon's points are visited in walking order (a_0, b_0, a_1, b_1, ...)
  // and its shoelace terms and link segments summed on the fly, in that order,
  // so no point list is kept.
  C x0 = C(0), y0 = C(0);  // first point (a_0)
  C xp = C(0), yp = C(0);  // last point so far
  bool any = false;
  C twice = C(0), seg = C(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    // edge 0: y = 0, x 0 -> 1; edge 1: x = 1, y 0 -> 1; edge 2: y = 1, x 1 -> 0;
    // edge 3: x = 0, y 1 -> 0
    const bool horiz = (k == 0 || k == 2);
    const C fixed = (k == 1 || k == 2) ? C(1) : C(0);
    const C d = fixed - (horiz ? cy : cx);
    const C ad = d < C(0) ? -d : d;
    if (ad >= R) continue;
    const C s = vsqrt((R - ad) * (R + ad));
    const C c_run = horiz ? cx : cy;
    C lo = c_run - s, hi = c_run + s;
    lo = lo < C(0) ? C(0) : lo;
    hi = hi > C(1) ? C(1) : hi;
    if (!(hi > lo)) continue;
    const bool up = (k == 0 || k == 1);
    const C a = up ? lo : hi, b = up ? hi : lo;  // start and end in walking order
    const C ax = horiz ? a : fixed, ay = horiz ? fixed : a;
    const C bx = horiz ? b : fixed, by = horiz ? fixed : b;
    if (any) {
      // link from the previous interval's end to this start: a chord and its arc
      twice += xp * ay - ax * yp;
      const C lx = ax - xp, ly = ay - yp;
      const C L = vsqrt(lx * lx + ly * ly);
      if (L > C(0)) seg += segment_area(L < C(2) * R ? L : C(2) * R, R);
    } else {
      x0 = ax; y0 = ay;
      any = true;
    }
    twice += ax * by - bx * ay;
    xp = bx; yp = by;
  }
  if (!any) return C(0);
  // closing link from the last end back to the first start
  twice += xp * y0 - x0 * yp;
  {
    const C lx = x0 - xp, ly = y0 - yp;
    const C L = vsqrt(lx * lx + ly * ly);
    if (L > C(0)) seg += segment_area(L < C(2) * R ? L : C(2) * R, R);
  }
  const C area = C(0.5) * twice + seg;
  return area < C(0) ? C(0) : (area > C(1) ? C(1) : area);
}

// Quick class of tile cell (il, jl): CELL_FLUID or CELL_SOLID where the
// centre distance decides it, CELL_BAND where the exact test is needed.  The
// FP32 lattice kernel and the band kernel both take this decision, so it is
// rounded step by step (mul_rn, add_rn) to come out the same in both.
enum : int { CELL_BAND = 3 };
template <class C>
__host__ __device__ __forceinline__ int quick_class(int il, int jl, const PartTile<C>& p) {
  // centre distance from the cell centre (hi/lo sums keep FP32 exact enough)
  const C dx = add_rn(add_rn(add_rn(C(il), C(0.5)), -p.xh), -p.xl);
  const C dy = add_rn(add_rn(add_rn(C(jl), C(0.5)), -p.yh), -p.yl);
  const C d2 = add_rn(mul_rn(dx, dx), mul_rn(dy, dy));
  if (d2 >= p.far2) return CELL_FLUID;   // nearest point > R + 0.04
  if (d2 <= p.near2) return CELL_SOLID;  // farthest corner < R - 0.04
  return CELL_BAND;
}

// ---------------------------------------------------------------------------
// Ellipses (reading R13), in FP64 with every product, sum and quotient
// rounded one at a time, so that the class decisions are those of any other
// FP64 evaluation in the same order (the oracle's among them).
// ---------------------------------------------------------------------------
struct EllFrame { double u, v; };
// Point (px, py) in the ellipse's unit-disk frame: ((c dx + s dy) / a, (c dy - s dx) / b).
__host__ __device__ __forceinline__ EllFrame ellipse_frame(double px, double py, double X, double Y, double a,
                                                           double b, double c, double s) {
  const double dx = add_rn(px, -X), dy = add_rn(py, -Y);
  EllFrame f;
#ifdef __CUDA_ARCH__
  f.u = __ddiv_rn(add_rn(mul_rn(c, dx), mul_rn(s, dy)), a);
  f.v = __ddiv_rn(add_rn(mul_rn(c, dy), -mul_rn(s, dx)), b);
#else
  f.u = (c * dx + s * dy) / a;
  f.v = (c * dy - s * dx) / b;
#endif
  return f;
}
__host__ __device__ __forceinline__ double quad_uv(double u, double v) { return add_rn(mul_rn(u, u), mul_rn(v, v)); }

// Class of cell [i, i+1] x [j, j+1]: SOLID when its four corners lie in the
// closed ellipse, FLUID when the least value of the quadratic form over the
// cell (each edge's convex quadratic at its clamped vertex) is >= 1.
__host__ __device__ __forceinline__ int ellipse_cell_class(int i, int j, double X, double Y, double a, double b,
                                                           double c, double s) {
  double cu[4], cv[4];
  const double xs[4] = {double(i), double(i + 1), double(i + 1), double(i)};
  const double ys[4] = {double(j), double(j), double(j + 1), double(j + 1)};
  double qmax = 0.0, qmin = 0.0;
  for (int k = 0; k < 4; ++k) {
    const EllFrame f = ellipse_frame(xs[k], ys[k], X, Y, a, b, c, s);
    cu[k] = f.u; cv[k] = f.v;
    const double q = quad_uv(f.u, f.v);
    qmax = k == 0 ? q : (q > qmax ? q : qmax);
    qmin = k == 0 ? q : (q < qmin ? q : qmin);
  }
  if (qmax <= 1.0) return CELL_SOLID;
  if (double(i) <= X && X <= double(i + 1) && double(j) <= Y && Y <= double(j + 1)) return CELL_INTERFACE;
  for (int k = 0; k < 4; ++k) {
    const int k1 = (k + 1) & 3;
    const double du = add_rn(cu[k1], -cu[k]), dv = add_rn(cv[k1], -cv[k]);
    const double A = quad_uv(du, dv);
#ifdef __CUDA_ARCH__
    double t = __ddiv_rn(-add_rn(mul_rn(cu[k], du), mul_rn(cv[k], dv)), A);
#else
    double t = -(cu[k] * du + cv[k] * dv) / A;
#endif
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    const double q = quad_uv(add_rn(cu[k], mul_rn(t, du)), add_rn(cv[k], mul_rn(t, dv)));
    qmin = q < qmin ? q : qmin;
  }
  return qmin >= 1.0 ? CELL_FLUID : CELL_INTERFACE;
}

// Area of the unit disk within the convex quadrilateral (us, vs) (counter-
// clockwise), by Green's theorem on the intersection's boundary: inside
// parts of the edges contribute (u_a v_b - u_b v_a) / 2, the arcs between
// leaving the disk on one edge and entering it on a later one half their
// counter-clockwise angle; a vertex on the circle (exit and entry at the same
// point of consecutive edges) adds no arc.
__host__ __device__ __forceinline__ double quad_unit_disk_area(const double (&us)[4], const double (&vs)[4]) {
  double pa_u[4], pa_v[4], pb_u[4], pb_v[4];
  int edge[4];
  int m = 0;
  for (int k = 0; k < 4; ++k) {
    const int k1 = (k + 1) & 3;
    const double u0 = us[k], v0 = vs[k];
    const double du = us[k1] - u0, dv = vs[k1] - v0;
    const double A = du * du + dv * dv, B = u0 * du + v0 * dv, C = u0 * u0 + v0 * v0 - 1.0;
    const double disc = B * B - A * C;
    if (A == 0.0 || disc <= 0.0) continue;
    const double r = sqrt(disc);
    double t0 = (-B - r) / A, t1 = (-B + r) / A;
    t0 = t0 > 0.0 ? t0 : 0.0;
    t1 = t1 < 1.0 ? t1 : 1.0;
    if (t1 <= t0) continue;
    pa_u[m] = u0 + t0 * du; pa_v[m] = v0 + t0 * dv;
    pb_u[m] = u0 + t1 * du; pb_v[m] = v0 + t1 * dv;
    edge[m] = k;
    ++m;
  }
  if (m == 0) {
    bool inside = true;  // the disk's centre inside the polygon (then the whole disk is)
    for (int k = 0; k < 4; ++k) {
      const int k1 = (k + 1) & 3;
      inside = inside && ((us[k1] - us[k]) * (0.0 - vs[k]) - (vs[k1] - vs[k]) * (0.0 - us[k]) >= 0.0);
    }
    return inside ? 3.14159265358979323846 : 0.0;
  }
  double area = 0.0;
  for (int q = 0; q < m; ++q) {
    area += 0.5 * (pa_u[q] * pb_v[q] - pb_u[q] * pa_v[q]);
    const int n1 = q + 1 < m ? q + 1 : 0;
    const double qu = pa_u[n1], qv = pa_v[n1];
    const double gu = qu - pb_u[q], gv = qv - pb_v[q];
    if (edge[n1] == ((edge[q] + 1) & 3) && gu * gu + gv * gv < 1e-24) continue;
    double ang = atan2(pb_u[q] * qv - pb_v[q] * qu, pb_u[q] * qu + pb_v[q] * qv);
    if (ang < 0.0) ang += 2.0 * 3.14159265358979323846;
    area += 0.5 * ang;
  }
  return area;
}

// Exact area of the ellipse in cell [i, i+1] x [j, j+1] (the cell is a
// parallelogram in the unit-disk frame; areas scale by a b).
__host__ __device__ __forceinline__ double ellipse_cell_area(int i, int j, double X, double Y, double a, double b,
                                                             double c, double s) {
  const double xs[4] = {double(i), double(i + 1), double(i + 1), double(i)};
  const double ys[4] = {double(j), double(j), double(j + 1), double(j + 1)};
  double us[4], vs[4];
  for (int k = 0; k < 4; ++k) {
    const EllFrame f = ellipse_frame(xs[k], ys[k], X, Y, a, b, c, s);
    us[k] = f.u; vs[k] = f.v;
  }
  return a * b * quad_unit_disk_area(us, vs);
}

// Class and fraction of cell (gi, gj) of the lattice for an ellipse; the
// quick test on the circumscribed and inscribed circles first (its SOLID and
// FLUID answers are exact), the FP64 class and area for the band cells.
template <class C>
__host__ __device__ __forceinline__ int ellipse_cell_fraction(int il, int jl, int gi, int gj, const PartTile<C>& p,
                                                              C& fsp) {
  const int qc = quick_class(il, jl, p);
  if (qc == CELL_FLUID) { fsp = C(0); return CELL_FLUID; }
  if (qc == CELL_SOLID) { fsp = C(1); return CELL_SOLID; }
  const int cls = ellipse_cell_class(gi, gj, p.ex, p.ey, p.ea, p.eb, p.ec, p.es);
  if (cls == CELL_SOLID) { fsp = C(1); return cls; }
  if (cls == CELL_FLUID) { fsp = C(0); return cls; }
  const double ar = ellipse_cell_area(gi, gj, p.ex, p.ey, p.ea, p.eb, p.ec, p.es);
  fsp = C(ar < 0.0 ? 0.0 : (ar > 1.0 ? 1.0 : ar));
  return cls;
}

// Class and solid fraction of tile cell (il, jl) for one particle.
template <class C>
__host__ __device__ __forceinline__ int cell_fraction(int il, int jl, const PartTile<C>& p, C& fsp) {
  const int qc = quick_class(il, jl, p);
  if (qc == CELL_FLUID) { fsp = C(0); return CELL_FLUID; }
  if (qc == CELL_SOLID) { fsp = C(1); return CELL_SOLID; }
  const int cls = cell_class_exact(il, jl, p);
  if (cls == CELL_SOLID) { fsp = C(1); return cls; }
  if (cls == CELL_FLUID) { fsp = C(0); return cls; }
  const C cx = (p.xh - C(il)) + p.xl;  // disk centre in cell-local coordinates
  const C cy = (p.yh - C(jl)) + p.yl;
  fsp = disk_unit_cell_area(cx, cy, p.r);
  return cls;
}

// The geometry fields of a particle's raster record as seen from the tile with
// origin (x0, y0) (FP32, no FP64 arithmetic): everything cell_fraction reads.
__host__ __device__ __forceinline__ void tile_geometry(const RasterRec& rc, int x0, int y0, PartTile<float>& q) {
  const long long Q = 1ll << QBITS;
  q.xq = (long long)(rc.xi - x0) * Q + rc.qfx;
  q.yq = (long long)(rc.yi - y0) * Q + rc.qfy;
  q.rq2 = rc.rq2;
  const float fx = float(rc.xi - x0), fy = float(rc.yi - y0);  // exact small integers
  q.xh = add_rn(fx, rc.xfh);
  q.xl = add_rn(add_rn(add_rn(fx, -q.xh), rc.xfh), rc.xfl);
  q.yh = add_rn(fy, rc.yfh);
  q.yl = add_rn(add_rn(add_rn(fy, -q.yh), rc.yfh), rc.yfl);
  q.r = rc.r; q.far2 = rc.far2; q.near2 = rc.near2;
  q.ci = rc.xi; q.cj = rc.yi;
}

}  // namespace vlb
