// Device code of the particle step (Sec. 2.3), shared by the single-case
// kernels (vlb_particles.cu) and the batched ones (vlb_batch.cu).
//
// Particle kernels (Sec. 2.3).
//
//   particle_step (one launch per time step): for each particle
//     advance (one lane, FP64): F_MES, T_MES of Eq. 28 from the integer
//       accumulators the lattice kernel filled (then cleared); the
//       inside-fluid force and torque of Eq. 29 with backward differences;
//       the short-range contact force; Eqs. 26 and 30 by forward Euler; the
//       raster record and the tile range of the new position;
//     band pass (one warp): appends the particle to the tile lists of its
//       range (the lattice kernel ranks each list by id and finds the
//       contact partners of the level) and fills its band table (FP32 for a
//       disk, FP64 for an ellipse).
//   particle_range, particle_band: the same for the initial state.
#pragma once

#include <math.h>

#include "vlb_common.cuh"
#include "vlb_kernels.h"
#include "vlb_raster.cuh"

namespace vlb {

// Tiles covered by [X - R - m, X + R + m] (clipped to the domain), in FP32: the
// margin m >= 2 cells absorbs the rounding, and the range is computed once per
// step and stored, so every use of it agrees.
__device__ __forceinline__ int4 tile_range(const ParticleConst& c, double Xd, double Yd, double Rd) {
  const float X = float(Xd), Y = float(Yd), e = float(Rd) + float(c.margin);
  int cx0 = (int)floorf(X - e), cx1 = (int)floorf(X + e);
  int cy0 = (int)floorf(Y - e), cy1 = (int)floorf(Y + e);
  cx0 = max(cx0, 0); cy0 = max(cy0, 0);
  cx1 = min(cx1, c.nx - 1); cy1 = min(cy1, c.ny - 1);
  if (cx1 < cx0 || cy1 < cy0) return make_int4(0, 0, 0, 0);
  const int tx0 = cx0 / TILE_X, tx1 = cx1 / TILE_X;
  const int ty0 = cy0 / TILE_Y, ty1 = cy1 / TILE_Y;
  return make_int4(tx0, ty0, tx1 - tx0 + 1, ty1 - ty0 + 1);
}

__device__ __forceinline__ void check_domain(const ParticleConst& c, double X, double Y, double R,
                                             unsigned* err) {
  bool bad = !(X >= 0.0 && X <= double(c.nx) && Y >= 0.0 && Y <= double(c.ny));
  if (c.per_x) bad |= (X - R - 1.0 < 0.0) || (X + R + 1.0 > double(c.nx));
  if (c.per_y) bad |= (Y - R - 1.0 < 0.0) || (Y + R + 1.0 > double(c.ny));
  if (bad) atomicOr(err, ERR_OUT_OF_DOMAIN);
}

// Raster record of particle p at centre (X, Y) with velocity (ux, uy, om);
// R its radius (an ellipse's semi-major axis), Rb its semi-minor axis: the
// quick test's bounds are the circumscribed and inscribed circles.
__device__ __forceinline__ void write_record(const ParticleArrays& P, int p, double X, double Y, double R, double Rb,
                                             double ux, double uy, double om, float lam_s, float T0) {
  RasterRec q;
  const double Q = double(1 << QBITS);
  q.xi = (int)floor(X);
  q.yi = (int)floor(Y);
  q.qfx = (int)(__double2ll_rn(X * Q) - (long long)q.xi * (1ll << QBITS));
  q.qfy = (int)(__double2ll_rn(Y * Q) - (long long)q.yi * (1ll << QBITS));
  const long long rq = __double2ll_rn(R * Q);
  q.rq2 = rq * rq;
  const double fx = X - double(q.xi), fy = Y - double(q.yi);
  q.xfh = float(fx); q.xfl = float(fx - double(q.xfh));
  q.yfh = float(fy); q.yfl = float(fy - double(q.yfh));
  q.r = float(R);
  q.far2 = float((R + 0.75) * (R + 0.75));
  q.near2 = Rb > 0.75 ? float((Rb - 0.75) * (Rb - 0.75)) : -1.0f;
  q.ux = float(ux); q.uxl = float(ux - double(q.ux));
  q.uy = float(uy); q.uyl = float(uy - double(q.uy));
  q.om = float(om);
  q.lam_s = lam_s;
  q.T0 = T0;
  P.rec[p] = q;
}


// Particle p's update (one thread).
__device__ __forceinline__ void advance_one(const ParticleConst& c, const ParticleArrays& P, int p, unsigned* err) {
  const double X = P.x[p], Y = P.y[p], R = P.r[p], Rb = P.rb[p];
  const double ux = P.ux[p], uy = P.uy[p], om = P.om[p];
  const double* kp = P.pk + 8 * p;  // 1/M, 1/I, M_in, I_in, body factor, wall factor
  double k[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) k[i] = kp[i];
  const double ux_prev = P.ux_prev[p], uy_prev = P.uy_prev[p], om_prev = P.om_prev[p];
  const double theta = P.theta[p];
  const float lam_s = float(P.lam_s[p]), T0 = float(P.T0[p]);
  // momentum-exchange force and torque of the current level (Eq. 28) plus the
  // particle-particle contact forces of that level: the lattice kernel's
  // integer accumulators, read and cleared for the next level
  // (read and cleared at the L2 with atomic exchanges, so that a particle
  // step inside a lattice launch never reads an L1 line this SM loaded
  // before other SMs added to the words)
  unsigned long long* acc = P.mes + 6 * (long long)p;
  unsigned long long a[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) a[i] = atomicExch(acc + i, 0ull);
  const double Fm_x = mes_value(a[0], a[1]), Fm_y = mes_value(a[2], a[3]), Tm = mes_value(a[4], a[5]);
  P.nbr_count[p] = 0;  // the lattice kernel of this step lists the next partners
  // wall contact forces: walls x-, x+, y-, y+ (none on open sides); an
  // ellipse meets a wall with its extent along the wall's normal (reading R13)
  double Fc_x = 0.0, Fc_y = 0.0;
  {
    const double dist[4] = {X, double(c.nx) - X, Y, double(c.ny) - Y};
    const double nxw[4] = {1.0, -1.0, 0.0, 0.0}, nyw[4] = {0.0, 0.0, 1.0, -1.0};
    double ext_x = R, ext_y = R;
    if (Rb != R) {
      double sn, cs;
      sincos(theta, &sn, &cs);
      ext_x = sqrt(R * R * cs * cs + Rb * Rb * sn * sn);
      ext_y = sqrt(R * R * sn * sn + Rb * Rb * cs * cs);
    }
    for (int w = 0; w < 4; ++w) {
      if ((w < 2 && c.per_x) || (w >= 2 && c.per_y) || c.outflow[w]) continue;
      const double gap = 2.0 * (w < 2 ? ext_x : ext_y) + c.zeta - 2.0 * dist[w];
      if (gap <= 0.0) continue;
      const double gz = gap * c.inv_zeta;
      const double mag = k[5] * gz * gz;
      Fc_x += mag * nxw[w];
      Fc_y += mag * nyw[w];
    }
  }
  // Eqs. 26, 29, 30: F_c = F_MES - F_in + (rho_s - rho_f) V g + F_contact
  // (Fm_x, Fm_y carry the particle-particle part of F_contact)
  const double Fin_x = -k[2] * (ux - ux_prev);
  const double Fin_y = -k[2] * (uy - uy_prev);
  const double Tin = -k[3] * (om - om_prev);
  const double Fx = Fm_x - Fin_x + k[4] * c.gx + Fc_x;
  const double Fy = Fm_y - Fin_y + k[4] * c.gy + Fc_y;
  const double Tc = Tm - Tin;
  P.fcx[p] = Fx;
  P.fcy[p] = Fy;
  P.tc[p] = Tc;
  const double Xn = X + ux, Yn = Y + uy;
  P.x[p] = Xn;
  P.y[p] = Yn;
  P.theta[p] = theta + om;
  P.ux_prev[p] = ux;
  P.uy_prev[p] = uy;
  P.om_prev[p] = om;
  const double uxn = ux + Fx * k[0], uyn = uy + Fy * k[0];
  const double omn = om + Tc * k[1];
  P.ux[p] = uxn;
  P.uy[p] = uyn;
  P.om[p] = omn;
  if (!(uxn * uxn + uyn * uyn <= 0.25)) atomicOr(err, ERR_TOO_FAST);
  check_domain(c, Xn, Yn, R, err);
  write_record(P, p, Xn, Yn, R, Rb, uxn, uyn, omn, lam_s, T0);
  const int4 nr = tile_range(c, Xn, Yn, R);
  P.prange[p] = nr;
  // (the band kernel that follows appends the particle to the tile lists)
}

// Exact classes and areas (Sec. 2) of the cells whose centre lies in the band
// |d - R| < 0.75 of a disk, i.e. the cells the lattice kernel's quick test
// leaves open.  Results go to the particle's band table with the level's
// stamp; the geometry (tile_geometry) and the tests are the ones the lattice
// kernel itself uses, so the results are the ones it would compute.
constexpr int BAND_WARPS = 4;    // particles per CTA
constexpr int BAND_QUEUE = 256;  // queued band cells per warp before an evaluation pass
constexpr int STEP_WARPS = 16;   // particles per CTA of the particle step

// ELL: the band pass of an ellipse (its exact classes and areas in FP64),
// compiled into a kernel of its own so that the disk path keeps its
// register budget.
template <bool ELL>
__device__ __forceinline__ void band_evaluate(const ParticleConst& c, const ParticleArrays& P, int p, int stamp,
                                              const RasterRec& rc, int bw, const int* queue, int nq, int lane) {
  // an ellipse: its exact classes and areas in FP64 at the level's position
  // and angle (reading R13); a disk: the FP32 geometry of the lattice kernel
  double ea = 0.0, eb = 0.0, ex = 0.0, ey = 0.0, ec = 1.0, es = 0.0;
  if (ELL && nq > 0) {
    ea = P.r[p];
    eb = P.rb[p];
    ex = P.x[p];
    ey = P.y[p];
    sincos(P.theta[p], &es, &ec);
  }
  for (int j = lane; j < nq; j += 32) {
    const int k = queue[j];
    const int by = k / bw, bx = k - by * bw;
    const int x = rc.xi - c.band_off + bx, y = rc.yi - c.band_off + by;
    float f;
    int cls;
    if constexpr (ELL) {
      cls = ellipse_cell_class(x, y, ex, ey, ea, eb, ec, es);
      const double ar = cls == CELL_SOLID ? 1.0 : (cls == CELL_FLUID ? 0.0 : ellipse_cell_area(x, y, ex, ey, ea, eb, ec, es));
      f = float(ar < 0.0 ? 0.0 : (ar > 1.0 ? 1.0 : ar));
    } else {
      const int x0 = x - x % TILE_X, y0 = y - y % TILE_Y;
      PartTile<float> q;
      tile_geometry(rc, x0, y0, q);
      cls = cell_fraction(x - x0, y - y0, q, f);
    }
    P.band[(long long)p * bw * bw + k] = make_int2(cls | (stamp << 2), __float_as_int(f));
  }
}

// Particle p's lists and band table (one warp; queue: BAND_QUEUE ints of
// shared memory of this warp).
template <bool ELL>
__device__ __forceinline__ void band_one(const ParticleConst& c, const ParticleArrays& P, const TileLists& TL,
                                         unsigned* err, int p, int stamp, int* queue, int lane) {
  const RasterRec rc = P.rec[p];
  const int bw = 2 * c.band_off + 1;
  // append the particle to the lists of the tiles of its range, one lane per tile
  {
    const int4 rg = P.prange[p];
    const int n = rg.z * rg.w;
    for (int t = lane; t < n; t += 32) {
      const int ty = t / rg.z, tx = t - ty * rg.z;
      const int tile = (rg.y + ty) * c.ntx + (rg.x + tx);
      const int slot = atomicAdd(&TL.count[tile], 1);
      if (slot < TILE_CAP) TL.ids[(long long)tile * TILE_CAP + slot] = p;
      else atomicOr(err, ERR_TILE_OVERFLOW);
    }
  }
  // Lane r takes row r of the box and only the cells of that row that can be
  // in the band: |x - X| between sqrt((R - 0.75)^2 - dy^2) and
  // sqrt((R + 0.75)^2 - dy^2), widened by half a cell on either side (far
  // more than the FP32 error of these bounds).  The quick test then decides
  // each of these candidates exactly as the lattice kernel does.
  const float cx = float(c.band_off) + rc.xfh, cy = float(c.band_off) + rc.yfh;  // centre in box coordinates
  // the band lies between the inscribed and circumscribed circles' bounds
  // of the quick test (an ellipse: semi-minor and semi-major axis; a disk: R)
  const float ro = rc.r + 0.75f, ri = rc.near2 > 0.0f ? sqrtf(rc.near2) : 0.0f;
  int nq = 0;
  for (int by0 = 0; by0 < bw; by0 += 32) {
    const int by = by0 + lane;
    const int y = rc.yi - c.band_off + by;
    int a0 = 0, a1 = -1, b0 = 0, b1 = -1;  // candidate runs [a0, a1], [b0, b1] of bx
    if (by < bw && y >= 0 && y < c.ny) {
      const float dy = (float(by) + 0.5f) - cy;
      const float oa = ro * ro - dy * dy;
      if (oa > -1.0f) {  // the row meets the widened outer circle
        const float wa = sqrtf(fmaxf(oa, 0.0f)) + 0.5f;
        const float ib = ri * ri - dy * dy;
        const float wb = (ri > 0.0f && ib > 0.0f) ? sqrtf(ib) - 0.5f : 0.0f;
        // cell bx is a candidate when |bx + 0.5 - cx| lies in [wb, wa]
        a0 = max(0, (int)ceilf(cx - wa - 0.5f));
        b1 = min(bw - 1, (int)floorf(cx + wa - 0.5f));
        if (wb > 0.0f) {
          a1 = (int)floorf(cx - wb - 0.5f);
          b0 = (int)ceilf(cx + wb - 0.5f);
        } else {  // one run through the middle
          a1 = b1;
          b0 = 0;
          b1 = -1;
        }
        a1 = min(a1, bw - 1);
        b0 = max(b0, 0);
      }
    }
    const int na = max(a1 - a0 + 1, 0), nb = max(b1 - b0 + 1, 0);
    int nmax = na + nb;
    for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    for (int j = 0; j < nmax; ++j) {
      bool in_band = false;
      int k = 0;
      if (j < na + nb) {
        const int bx = j < na ? a0 + j : b0 + (j - na);
        const int x = rc.xi - c.band_off + bx;
        k = by * bw + bx;
        if (x >= 0 && x < c.nx) {
          const int x0 = x - x % TILE_X, y0 = y - y % TILE_Y;
          PartTile<float> q;
          tile_geometry(rc, x0, y0, q);
          in_band = quick_class(x - x0, y - y0, q) == CELL_BAND;
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, in_band);
      if (in_band) queue[nq + __popc(m & ((1u << lane) - 1u))] = k;
      nq += __popc(m);
      if (nq > BAND_QUEUE - 32) {  // evaluate what is queued before it can overflow
        __syncwarp();
        band_evaluate<ELL>(c, P, p, stamp, rc, bw, queue, nq, lane);
        __syncwarp();
        nq = 0;
      }
    }
  }
  __syncwarp();
  band_evaluate<ELL>(c, P, p, stamp, rc, bw, queue, nq, lane);
}

}  // namespace vlb
