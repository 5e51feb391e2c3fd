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

// One particle as seen from one tile (shared memory).  Coordinates are
// relative to the tile's lower-left corner.
template <class C>
struct PartTile {
  long long xq, yq, rq2;  // fixed-point centre and R^2 (2^-20 grid)
  C xh, xl, yh, yl;       // centre as an unevaluated sum hi + lo
  C r, far2, near2;       // radius, quick-reject bounds on the centre distance^2
  C ux, uy, om;           // rigid-body motion (Eq. 27)
  C uxl, uyl;             // low parts of U (U = ux + uxl to FP64 accuracy)
  C lam_s, T0;
  int id;                 // particle id
  int ci, cj;             // cell of the centre (band table origin)
  int fixed;              // held at its temperature T0 (reading R11)
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
