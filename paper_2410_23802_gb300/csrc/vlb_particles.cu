// Particle kernels (Sec. 2.3).
//
//   particle_advance (thread per particle, FP64): F_MES, T_MES of Eq. 28 from
//     the integer accumulators the lattice kernel filled (then cleared); the
//     inside-fluid force and torque of Eq. 29 with backward differences; the
//     short-range contact force; Eqs. 26 and 30 by forward Euler; the raster
//     record and the tile range of the new position;
//   particle_band_cta (CTA per particle, FP32): appends the particle to the
//     tile lists of its range (the lattice kernel ranks each list by id and
//     finds the contact partners of the level) and fills its band table.
//   particle_range, then particle_band_cta: the same for the initial state.
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

// Raster record of particle p at centre (X, Y) with velocity (ux, uy, om).
__device__ __forceinline__ void write_record(const ParticleArrays& P, int p, double X, double Y, double R,
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
  q.near2 = R > 0.75 ? float((R - 0.75) * (R - 0.75)) : -1.0f;
  q.ux = float(ux); q.uxl = float(ux - double(q.ux));
  q.uy = float(uy); q.uyl = float(uy - double(q.uy));
  q.om = float(om);
  q.lam_s = lam_s;
  q.T0 = T0;
  P.rec[p] = q;
}

__global__ void particle_range_kernel(const ParticleConst c, const ParticleArrays P, unsigned* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= c.np) return;
  const int4 rg = tile_range(c, P.x[p], P.y[p], P.r[p]);
  P.prange[p] = rg;
  write_record(P, p, P.x[p], P.y[p], P.r[p], P.ux[p], P.uy[p], P.om[p], float(P.lam_s[p]), float(P.T0[p]));
}

// Particle p's update (one thread).
__device__ __forceinline__ void advance_one(const ParticleConst& c, const ParticleArrays& P, int p, unsigned* err) {
  const double X = P.x[p], Y = P.y[p], R = P.r[p];
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
  unsigned long long* acc = P.mes + 6 * (long long)p;
  const ulonglong2 a0 = reinterpret_cast<const ulonglong2*>(acc)[0];
  const ulonglong2 a1 = reinterpret_cast<const ulonglong2*>(acc)[1];
  const ulonglong2 a2 = reinterpret_cast<const ulonglong2*>(acc)[2];
  const double Fm_x = mes_value(a0.x, a0.y), Fm_y = mes_value(a1.x, a1.y), Tm = mes_value(a2.x, a2.y);
  reinterpret_cast<ulonglong2*>(acc)[0] = make_ulonglong2(0ull, 0ull);
  reinterpret_cast<ulonglong2*>(acc)[1] = make_ulonglong2(0ull, 0ull);
  reinterpret_cast<ulonglong2*>(acc)[2] = make_ulonglong2(0ull, 0ull);
  P.nbr_count[p] = 0;  // the lattice kernel of this step lists the next partners
  // wall contact forces: walls x-, x+, y-, y+
  double Fc_x = 0.0, Fc_y = 0.0;
  {
    const double dist[4] = {X, double(c.nx) - X, Y, double(c.ny) - Y};
    const double nxw[4] = {1.0, -1.0, 0.0, 0.0}, nyw[4] = {0.0, 0.0, 1.0, -1.0};
    for (int w = 0; w < 4; ++w) {
      if ((w < 2 && c.per_x) || (w >= 2 && c.per_y)) continue;
      const double gap = 2.0 * R + c.zeta - 2.0 * dist[w];
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
  write_record(P, p, Xn, Yn, R, uxn, uyn, omn, lam_s, T0);
  const int4 nr = tile_range(c, Xn, Yn, R);
  P.prange[p] = nr;
  // (the band kernel that follows appends the particle to the tile lists)
}

// Exact classes and areas (Sec. 2) of the cells whose centre lies in the band
// |d - R| < 0.75 of a disk, i.e. the cells the lattice kernel's quick test
// leaves open.  Results go to the particle's band table with the level's
// stamp; the geometry (tile_geometry) and the tests are the ones the lattice
// kernel itself uses, so the results are the ones it would compute.
// The band pass of one particle by a whole CTA (BAND_CTA threads), the form
// the time step uses: the particle's tile-list appends one thread per tile,
// the quick test of every cell of its box spread over the threads, the band
// cells queued in shared memory, then their exact class and area one thread
// per cell.  The box is taken in chunks of BAND_CHUNK cells per thread, so
// the queue (at most BAND_CTA * BAND_CHUNK cells) never overflows.  Same
// geometry and tests as band_one, so the same table entries.
constexpr int BAND_CTA = 128;
constexpr int BAND_CHUNK = 8;

__device__ __forceinline__ void band_cta(const ParticleConst& c, const ParticleArrays& P, const TileLists& TL,
                                         unsigned* err, int p, int stamp) {
  __shared__ int s_queue[BAND_CTA * BAND_CHUNK];
  __shared__ int s_nq;
  const int tid = threadIdx.x;
  const RasterRec rc = P.rec[p];
  const int bw = 2 * c.band_off + 1;
  {
    const int4 rg = P.prange[p];
    const int n = rg.z * rg.w;
    for (int t = tid; t < n; t += BAND_CTA) {
      const int ty = t / rg.z, tx = t - ty * rg.z;
      const int tile = (rg.y + ty) * c.ntx + (rg.x + tx);
      const int slot = atomicAdd(&TL.count[tile], 1);
      if (slot < TILE_CAP) TL.ids[(long long)tile * TILE_CAP + slot] = p;
      else atomicOr(err, ERR_TILE_OVERFLOW);
    }
  }
  const int ncell = bw * bw;
  int2* table = P.band + (long long)p * bw * bw;
  for (int base = 0; base < ncell; base += BAND_CTA * BAND_CHUNK) {
    if (tid == 0) s_nq = 0;
    __syncthreads();
#pragma unroll 1
    for (int j = 0; j < BAND_CHUNK; ++j) {
      const int k = base + j * BAND_CTA + tid;
      if (k >= ncell) break;
      const int by = k / bw, bx = k - by * bw;
      const int x = rc.xi - c.band_off + bx, y = rc.yi - c.band_off + by;
      if (x < 0 || x >= c.nx || y < 0 || y >= c.ny) continue;
      const int x0 = x - x % TILE_X, y0 = y - y % TILE_Y;
      PartTile<float> q;
      tile_geometry(rc, x0, y0, q);
      if (quick_class(x - x0, y - y0, q) == CELL_BAND) s_queue[atomicAdd(&s_nq, 1)] = k;
    }
    __syncthreads();
    const int nq = s_nq;
    for (int j = tid; j < nq; j += BAND_CTA) {
      const int k = s_queue[j];
      const int by = k / bw, bx = k - by * bw;
      const int x = rc.xi - c.band_off + bx, y = rc.yi - c.band_off + by;
      const int x0 = x - x % TILE_X, y0 = y - y % TILE_Y;
      PartTile<float> q;
      tile_geometry(rc, x0, y0, q);
      float f;
      const int cls = cell_fraction(x - x0, y - y0, q, f);
      table[k] = make_int2(cls | (stamp << 2), __float_as_int(f));
    }
    __syncthreads();  // s_nq and the queue are reused by the next chunk
  }
}

// Advance of every particle, one thread each.
__global__ void __launch_bounds__(128) particle_advance_kernel(const ParticleConst c, const ParticleArrays P,
                                                               unsigned* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < c.np) advance_one(c, P, p, err);
}

// Lists and band table of every particle, one CTA each.
__global__ void __launch_bounds__(BAND_CTA) particle_band_cta_kernel(const ParticleConst c, const ParticleArrays P,
                                                                     const TileLists TL, unsigned* err) {
  band_cta(c, P, TL, err, blockIdx.x, c.band_stamp);
}

// The same over the particles of many cases, step k of a batch call.
__global__ void __launch_bounds__(128) particle_advance_batch_kernel(const BatchParticles* __restrict__ cases,
                                                                     const int2* __restrict__ items, int nitems) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nitems) return;
  const int2 it = items[i];
  const BatchParticles& d = cases[it.x];
  advance_one(d.c, d.P, it.y, d.err);
}
__global__ void __launch_bounds__(BAND_CTA) particle_band_cta_batch_kernel(const BatchParticles* __restrict__ cases,
                                                                           const int2* __restrict__ items, int k) {
  const int2 it = items[blockIdx.x];
  const BatchParticles& d = cases[it.x];
  const int nl = 1 - (d.tl ^ (k & 1));
  band_cta(d.c, d.P, d.TL[nl], d.err, it.y, band_stamp_after(d.stamp, k + 1));
}

static inline dim3 pgrid(int n) { return dim3((unsigned)((n + 127) / 128)); }

cudaError_t launch_particle_range(const ParticleConst& c, const ParticleArrays& P, unsigned* err,
                                  cudaStream_t st) {
  if (c.np == 0) return cudaSuccess;
  particle_range_kernel<<<pgrid(c.np), 128, 0, st>>>(c, P, err);
  return cudaGetLastError();
}
cudaError_t launch_particle_band(const ParticleConst& c, const ParticleArrays& P, const TileLists& TL, unsigned* err,
                                 cudaStream_t st) {
  if (c.np == 0) return cudaSuccess;
  particle_band_cta_kernel<<<(unsigned)c.np, BAND_CTA, 0, st>>>(c, P, TL, err);
  return cudaGetLastError();
}
// The time step's particle part: the advance (thread per particle), then the
// band pass (CTA per particle).
cudaError_t launch_particle_step(const ParticleConst& c, const ParticleArrays& P, const TileLists& TL, unsigned* err,
                                 cudaStream_t st) {
  if (c.np == 0) return cudaSuccess;
  particle_advance_kernel<<<pgrid(c.np), 128, 0, st>>>(c, P, err);
  particle_band_cta_kernel<<<(unsigned)c.np, BAND_CTA, 0, st>>>(c, P, TL, err);
  return cudaGetLastError();
}
cudaError_t launch_particle_step_batch(const BatchParticles* cases, const int2* items, int nitems, int k,
                                       cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  particle_advance_batch_kernel<<<pgrid(nitems), 128, 0, st>>>(cases, items, nitems);
  particle_band_cta_batch_kernel<<<(unsigned)nitems, BAND_CTA, 0, st>>>(cases, items, k);
  return cudaGetLastError();
}
}  // namespace vlb
