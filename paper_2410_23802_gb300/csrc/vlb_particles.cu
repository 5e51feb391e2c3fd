// Particle kernels (Sec. 2.3), one thread per particle, FP64 throughout.
//
//   particle_advance: F_MES, T_MES as the ordered sum of the per-tile partials
//     of Eq. 28; the inside-fluid force and torque of Eq. 29 with backward
//     differences; the short-range contact force; Eqs. 26 and 30 by forward
//     Euler; the tile range of the new position.
//     The same thread then appends the particle to the tile lists of its new
//     range (the lattice kernel sorts each list by id and finds the contact
//     partners of the next level).
//   particle_bin: the appending alone (initial state).
#include <math.h>

#include "vlb_common.cuh"
#include "vlb_kernels.h"

namespace vlb {

__device__ __forceinline__ int4 tile_range(const ParticleConst& c, double X, double Y, double R) {
  const double m = c.margin;
  int cx0 = (int)floor(X - R - m), cx1 = (int)floor(X + R + m);
  int cy0 = (int)floor(Y - R - m), cy1 = (int)floor(Y + R + m);
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

__global__ void particle_range_kernel(const ParticleConst c, const ParticleArrays P, unsigned* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= c.np) return;
  const int4 rg = tile_range(c, P.x[p], P.y[p], P.r[p]);
  if (rg.z * rg.w > c.kt) atomicOr(err, ERR_PARTIAL_OVERFLOW);
  P.prange[p] = rg;
}

__device__ __forceinline__ void bin_particle(const ParticleConst& c, const TileLists& TL, int p, int4 rg,
                                             unsigned* err) {
  for (int b = 0; b < rg.w; ++b)
    for (int a = 0; a < rg.z; ++a) {
      const int t = (rg.y + b) * c.ntx + (rg.x + a);
      const int slot = atomicAdd(&TL.count[t], 1);
      if (slot < TILE_CAP) TL.ids[(long long)t * TILE_CAP + slot] = p;
      else atomicOr(err, ERR_TILE_OVERFLOW);
    }
}

__global__ void particle_advance_kernel(const ParticleConst c, const ParticleArrays P, const TileLists TL,
                                        unsigned* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= c.np) return;
  const double X = P.x[p], Y = P.y[p], R = P.r[p];
  // momentum-exchange force and torque of the current level (Eq. 28)
  const int4 rg = P.prange[p];
  int nk = rg.z * rg.w;
  if (nk > c.kt) nk = c.kt;
  double Fm_x = 0.0, Fm_y = 0.0, Tm = 0.0;
  const double* part = P.partial + (long long)p * c.kt * 3;
  for (int k = 0; k < nk; ++k) {
    Fm_x += part[3 * k + 0];
    Fm_y += part[3 * k + 1];
    Tm += part[3 * k + 2];
  }
  // contact force: partner forces (computed at this level by the lattice
  // kernel) summed in ascending partner id, then walls x-, x+, y-, y+
  double Fc_x = 0.0, Fc_y = 0.0;
  const int nn = min(P.nbr_count[p], NBR_CAP);
  int nb[NBR_CAP];
  double nfx[NBR_CAP], nfy[NBR_CAP];
  for (int a = 0; a < nn; ++a) {
    const int j = P.nbr[p * NBR_CAP + a];
    const double fx = P.nbr_f[2 * (p * NBR_CAP + a)], fy = P.nbr_f[2 * (p * NBR_CAP + a) + 1];
    int k = a;
    while (k > 0 && nb[k - 1] > j) { nb[k] = nb[k - 1]; nfx[k] = nfx[k - 1]; nfy[k] = nfy[k - 1]; --k; }
    nb[k] = j; nfx[k] = fx; nfy[k] = fy;
  }
  P.nbr_count[p] = 0;  // the lattice kernel of this step lists the next partners
  for (int a = 0; a < nn; ++a) {
    Fc_x += nfx[a];
    Fc_y += nfy[a];
  }
  {
    const double cw = c.contact_scale * R * R / c.eps_w;
    const double dist[4] = {X, double(c.nx) - X, Y, double(c.ny) - Y};
    const double nxw[4] = {1.0, -1.0, 0.0, 0.0}, nyw[4] = {0.0, 0.0, 1.0, -1.0};
    for (int w = 0; w < 4; ++w) {
      if ((w < 2 && c.per_x) || (w >= 2 && c.per_y)) continue;
      const double gap = 2.0 * R + c.zeta - 2.0 * dist[w];
      if (gap <= 0.0) continue;
      const double mag = cw * (gap / c.zeta) * (gap / c.zeta);
      Fc_x += mag * nxw[w];
      Fc_y += mag * nyw[w];
    }
  }
  // Eqs. 26, 29, 30: F_c = F_MES - F_in + (rho_s - rho_f) V g + F_contact
  const double pi = 3.141592653589793;
  const double area = pi * R * R;
  const double M = c.rho_ratio * area, I = 0.5 * M * R * R;
  const double Min = area, Iin = 0.5 * Min * R * R;
  const double ux = P.ux[p], uy = P.uy[p], om = P.om[p];
  const double Fin_x = -Min * (ux - P.ux_prev[p]);
  const double Fin_y = -Min * (uy - P.uy_prev[p]);
  const double Tin = -Iin * (om - P.om_prev[p]);
  const double body = (c.rho_ratio - 1.0) * area;
  const double Fx = Fm_x - Fin_x + body * c.gx + Fc_x;
  const double Fy = Fm_y - Fin_y + body * c.gy + Fc_y;
  const double Tc = Tm - Tin;
  P.fcx[p] = Fx;
  P.fcy[p] = Fy;
  P.tc[p] = Tc;
  const double Xn = X + ux, Yn = Y + uy;
  P.x[p] = Xn;
  P.y[p] = Yn;
  P.theta[p] = P.theta[p] + om;
  P.ux_prev[p] = ux;
  P.uy_prev[p] = uy;
  P.om_prev[p] = om;
  const double uxn = ux + Fx / M, uyn = uy + Fy / M;
  P.ux[p] = uxn;
  P.uy[p] = uyn;
  P.om[p] = om + Tc / I;
  if (!(uxn * uxn + uyn * uyn <= 0.25)) atomicOr(err, ERR_TOO_FAST);
  check_domain(c, Xn, Yn, R, err);
  const int4 nr = tile_range(c, Xn, Yn, R);
  if (nr.z * nr.w > c.kt) atomicOr(err, ERR_PARTIAL_OVERFLOW);
  P.prange[p] = nr;
  bin_particle(c, TL, p, nr, err);
}

__global__ void particle_bin_kernel(const ParticleConst c, const ParticleArrays P, const TileLists TL,
                                    unsigned* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= c.np) return;
  bin_particle(c, TL, p, P.prange[p], err);
}

static inline dim3 pgrid(int n) { return dim3((unsigned)((n + 127) / 128)); }

cudaError_t launch_particle_range(const ParticleConst& c, const ParticleArrays& P, unsigned* err,
                                  cudaStream_t st) {
  if (c.np == 0) return cudaSuccess;
  particle_range_kernel<<<pgrid(c.np), 128, 0, st>>>(c, P, err);
  return cudaGetLastError();
}
cudaError_t launch_particle_advance(const ParticleConst& c, const ParticleArrays& P, const TileLists& TL,
                                    unsigned* err, cudaStream_t st) {
  if (c.np == 0) return cudaSuccess;
  particle_advance_kernel<<<pgrid(c.np), 128, 0, st>>>(c, P, TL, err);
  return cudaGetLastError();
}
cudaError_t launch_particle_bin(const ParticleConst& c, const ParticleArrays& P, const TileLists& TL,
                                unsigned* err, cudaStream_t st) {
  if (c.np == 0) return cudaSuccess;
  particle_bin_kernel<<<pgrid(c.np), 128, 0, st>>>(c, P, TL, err);
  return cudaGetLastError();
}
}  // namespace vlb
