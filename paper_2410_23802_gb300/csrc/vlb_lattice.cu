// The fused lattice kernel: one pass over the lattice per time step.
//
// Per cell, in registers:  pull f-bar and g-bar from the neighbours (Eqs. 3b,
// 17b) with wall rules; f_s^{n+1} from the tile's particle list (Sec. 2);
// volumetric correction of f (Eq. 8) and the momentum-exchange partials of
// Eq. 28; df_s/dt (Eq. 24), c_v and lambda (Eq. 11), grad T (Eq. 23), T
// jointly with u and the buoyancy force (Eqs. 9, 25), eps and q_c (Eqs. 16,
// 21); both MRT collisions (Eqs. 3a, 17a); stores of f-bar, g-bar and
// S = 2 f_s + df_s/dt at level n+1.
//
// Layout in HBM: structure of arrays, one plane per direction, x fastest,
// rows padded to 128 B.  f is stored as the deviation from the rest
// equilibrium w_i, g as the deviation from g^eq(T_fluid) (g_off), S in the
// arithmetic type.  Populations ping-pong between two buffers.
#include "vlb_common.cuh"
#include "vlb_raster.cuh"
#include "vlb_kernels.h"

namespace vlb {

template <class C, class S>
__device__ __forceinline__ C load_pop(const S* p) { return C(__ldg(p)); }

template <class C, class S>
__device__ __forceinline__ void store_pop(S* p, C v) { __stcs(p, S(v)); }

template <class C>
__device__ __forceinline__ C warp_sum(C v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Particle list of one tile, sorted by id (rank sort; ids are unique), with
// each particle's geometry relative to the tile origin.  Returns the count.
template <class C>
__device__ int load_tile_particles(const LatticeConst<C>& K, const ParticleArrays& P, const TileLists& TL,
                                   int tile_x, int tile_y, int* s_n, int* s_raw, PartTile<C>* s_p) {
  const int tid = threadIdx.y * TILE_X + threadIdx.x;
  const int tile = tile_y * K.ntx + tile_x;
  const int x0 = tile_x * TILE_X, y0 = tile_y * TILE_Y;
  if (tid == 0) {
    const int c = TL.count[tile];
    *s_n = c < TILE_CAP ? c : TILE_CAP;
  }
  __syncthreads();
  const int np = *s_n;
  if (tid < np) s_raw[tid] = TL.ids[(long long)tile * TILE_CAP + tid];
  __syncthreads();
  if (tid < np) {
    const int id = s_raw[tid];
    int rank = 0;
    for (int k = 0; k < np; ++k) rank += s_raw[k] < id;
    PartTile<C> q;
    const double X = P.x[id] - double(x0), Y = P.y[id] - double(y0), R = P.r[id];
    const long long Q = 1ll << QBITS;
    q.xq = __double2ll_rn(P.x[id] * double(Q)) - (long long)x0 * Q;
    q.yq = __double2ll_rn(P.y[id] * double(Q)) - (long long)y0 * Q;
    const long long rq = __double2ll_rn(R * double(Q));
    q.rq2 = rq * rq;
    q.xh = C(X); q.xl = C(X - double(q.xh));
    q.yh = C(Y); q.yl = C(Y - double(q.yh));
    q.r = C(R);
    q.far2 = C((R + 0.75) * (R + 0.75));
    q.near2 = R > 0.75 ? C((R - 0.75) * (R - 0.75)) : C(-1);
    q.ux = C(P.ux[id]); q.uy = C(P.uy[id]); q.om = C(P.om[id]);
    q.lam_s = C(P.lam_s[id]); q.T0 = C(P.T0[id]);
    q.id = id;
    const int4 rg = P.prange[id];
    const int kx = tile_x - rg.x, ky = tile_y - rg.y;
    q.k = (kx >= 0 && ky >= 0 && kx < rg.z && ky < rg.w && ky * rg.z + kx < K.kt) ? ky * rg.z + kx : -1;
    s_p[rank] = q;
  }
  __syncthreads();
  return np;
}

// Owners of cell (tx, ty) of the tile: ascending particle order, at most
// MAX_OWNERS, fractions scaled to sum 1 when they exceed it (overlap).
template <class C>
__device__ __forceinline__ C raster_cell(int tx, int ty, int np, const PartTile<C>* s_p, int& nown,
                                         int (&own)[MAX_OWNERS], int (&cls)[MAX_OWNERS],
                                         C (&ofs)[MAX_OWNERS], unsigned* err) {
  nown = 0;
#pragma unroll
  for (int k = 0; k < MAX_OWNERS; ++k) { own[k] = -1; cls[k] = 0; ofs[k] = C(0); }
  for (int s = 0; s < np; ++s) {
    C f;
    const int c = cell_fraction(tx, ty, s_p[s], f);
    if (c == CELL_FLUID) continue;
    if (nown == MAX_OWNERS) { atomicOr(err, ERR_OWNER_OVERFLOW); break; }
#pragma unroll
    for (int k = 0; k < MAX_OWNERS; ++k)
      if (k == nown) { own[k] = s; cls[k] = c; ofs[k] = f; }
    ++nown;
  }
  C fs = C(0);
#pragma unroll
  for (int k = 0; k < MAX_OWNERS; ++k) fs += ofs[k];
  if (fs > C(1)) {
    const C inv = C(1) / fs;
    fs = C(0);
#pragma unroll
    for (int k = 0; k < MAX_OWNERS; ++k) { ofs[k] *= inv; fs += ofs[k]; }
  }
  return fs;
}

template <class S, class C, int MODE>
__global__ void __launch_bounds__(TILE_X * TILE_Y)
lattice_kernel(const LatticeConst<C> K, const StepBuffers B, const ParticleArrays P, const TileLists TL) {
  __shared__ int s_n;
  __shared__ int s_raw[TILE_CAP];
  __shared__ PartTile<C> s_p[TILE_CAP];
  __shared__ C s_red[TILE_Y][3];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TILE_X + tx;
  const int tile_x = blockIdx.x, tile_y = blockIdx.y;
  const int x = tile_x * TILE_X + tx, y = tile_y * TILE_Y + ty;

  const int np = load_tile_particles<C>(K, P, TL, tile_x, tile_y, &s_n, s_raw, s_p);

  const bool active = (x < K.nx) && (y < K.ny);
  const long long cell = (long long)y * K.pitch + x;
  const S* __restrict__ src = static_cast<const S*>(B.src);

  // ---- solid fraction and owners (Sec. 2) -----------------------------------
  int nown = 0;
  int own[MAX_OWNERS], ocls[MAX_OWNERS];
  C ofs[MAX_OWNERS];
  C fs = C(0);
  if (active) fs = raster_cell<C>(tx, ty, np, s_p, nown, own, ocls, ofs, B.err);
  else {
#pragma unroll
    for (int k = 0; k < MAX_OWNERS; ++k) { own[k] = -1; ocls[k] = 0; ofs[k] = C(0); }
  }

  // ---- streaming (pull) with wall rules --------------------------------------
  C f[9], g[9];
  if (MODE == MODE_INIT) {
#pragma unroll
    for (int i = 0; i < 9; ++i) { f[i] = C(0); g[i] = C(0); }
  } else if (active) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      int sx = x - ex(i), sy = y - ey(i);
      bool outx = false, outy = false;
      if (K.per_x) sx = sx < 0 ? sx + K.nx : (sx >= K.nx ? sx - K.nx : sx);
      else outx = sx < 0 || sx >= K.nx;
      if (K.per_y) sy = sy < 0 ? sy + K.ny : (sy >= K.ny ? sy - K.ny : sy);
      else outy = sy < 0 || sy >= K.ny;
      if (!(outx || outy)) {
        const long long sc = (long long)sy * K.pitch + sx;
        f[i] = load_pop<C>(src + (long long)i * K.plane + sc);
        g[i] = load_pop<C>(src + (long long)(9 + i) * K.plane + sc) + K.g_off[i];
      } else {
        // halfway bounce-back of f; g bounces back (adiabatic) or anti-bounces
        // back to the wall temperature; corners go to the y wall
        f[i] = load_pop<C>(src + (long long)opp(i) * K.plane + cell);
        const C gb = load_pop<C>(src + (long long)(9 + opp(i)) * K.plane + cell) + K.g_off[opp(i)];
        const int wall = outy ? (sy < 0 ? 2 : 3) : (sx < 0 ? 0 : 1);
        g[i] = K.wall_dirichlet[wall] ? (C(2) * wgt<C>(i) * K.cref * K.wall_T[wall] - gb) : gb;
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) { f[i] = C(0); g[i] = C(0); }
  }

  // ---- flow: volumetric correction (Eq. 8) and exchange partials (Eq. 28) ---
  // f holds deviations from w_i; rho = 1 + drho.
  C drho = C(0), jx = C(0), jy = C(0);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    drho += f[i];
    jx += C(ex(i)) * f[i];
    jy += C(ey(i)) * f[i];
  }
  const C rho = C(1) + drho;
  C mesF[MAX_OWNERS][3];
#pragma unroll
  for (int k = 0; k < MAX_OWNERS; ++k) { mesF[k][0] = mesF[k][1] = mesF[k][2] = C(0); }
  C lam = (C(1) - fs) * K.lam_f;
  C Tinit_mix = (C(1) - fs) * K.cv_f * K.T_fluid;
  if (nown > 0) {
    const C one_m = C(1) - fs;
    C pf[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) pf[i] = C(0);
    C cjx = one_m * jx, cjy = one_m * jy;
    const C xc = C(tx) + C(0.5), yc = C(ty) + C(0.5);
#pragma unroll
    for (int k = 0; k < MAX_OWNERS; ++k) {
      if (k >= nown) break;
      const PartTile<C>& q = s_p[own[k]];
      const C rx = (xc - q.xh) - q.xl, ry = (yc - q.yh) - q.yl;
      const C usx = q.ux - q.om * ry, usy = q.uy + q.om * rx;  // Eq. 27
      const C w = ofs[k];
      const C u2 = usx * usx + usy * usy;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const C eu = C(ex(i)) * usx + C(ey(i)) * usy;
        pf[i] += w * (C(3) * eu + C(4.5) * eu * eu - C(1.5) * u2);
      }
      // sum_i e_i f_i^eq(rho, u_s) = rho u_s; Delta F = -f_s,p (rho u_s - j*)
      const C dFx = -w * (rho * usx - jx), dFy = -w * (rho * usy - jy);
      mesF[k][0] = dFx;
      mesF[k][1] = dFy;
      mesF[k][2] = rx * dFy - ry * dFx;
      cjx += w * rho * usx;
      cjy += w * rho * usy;
      lam += w * q.lam_s;
      Tinit_mix += w * K.cv_s * q.T0;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = one_m * f[i] + wgt<C>(i) * (fs * drho + rho * pf[i]);
    jx = cjx;
    jy = cjy;
  }

  // ---- thermal macroscopics at n+1 (Eqs. 11, 16, 21-25) ----------------------
  const C cv = (C(1) - fs) * K.cv_f + fs * K.cv_s;
  const C tau_g = C(0.5) + C(3) * lam / K.cref;  // Eq. 22 with alpha_1 = -2
  C T, eps, qc, dfs, ux, uy, Fx, Fy, G;
  const C ax = (C(1) - fs) * K.bx / (C(2) * rho), ay = (C(1) - fs) * K.by / (C(2) * rho);
  if (MODE == MODE_INIT) {
    eps = Tinit_mix;
    G = eps;
    T = eps / cv;
    qc = C(0);
    dfs = C(0);
    // g = g^eq(eps, T) (Eq. 19 with alpha_1 = -2, alpha_2 = 1)
    g[0] = eps - C(5) / C(9) * K.cref * T;
#pragma unroll
    for (int i = 1; i < 9; ++i) g[i] = wgt<C>(i) * K.cref * T;
    ux = jx / rho + ax * (T - K.T_ref);
    uy = jy / rho + ay * (T - K.T_ref);
  } else {
    const C s_old = active ? C(static_cast<const C*>(B.s_src)[cell]) : C(0);
    dfs = C(2) * fs - s_old;  // Eq. 24: 2 (f_s^{n+1} - f_s^n) - [df_s/dt]^n
    G = C(0);
    C qx = C(0), qy = C(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      G += g[i];
      qx += C(ex(i)) * g[i];
      qy += C(ey(i)) * g[i];
    }
    const C gk = C(-3) / (K.cref * tau_g);  // Eq. 23: -6/(4 + alpha_1) = -3
    const C gTx = gk * qx, gTy = gk * qy;
    const C D = cv - C(0.5) * (K.cv_s - K.cv_f) * dfs;
    const C u0x = jx / rho, u0y = jy / rho;
    const C num = G - C(0.5) * cv * ((u0x - ax * K.T_ref) * gTx + (u0y - ay * K.T_ref) * gTy);
    const C den = D + C(0.5) * cv * (ax * gTx + ay * gTy);
    T = num / den;
    ux = u0x + ax * (T - K.T_ref);
    uy = u0y + ay * (T - K.T_ref);
    eps = cv * T;
    qc = -cv * (ux * gTx + uy * gTy) + (K.cv_s - K.cv_f) * T * dfs;
  }
  Fx = (C(1) - fs) * K.bx * (T - K.T_ref);
  Fy = (C(1) - fs) * K.by * (T - K.T_ref);

  if (MODE == MODE_MACROS || MODE == MODE_INIT) {
    if (active && B.macro != nullptr) {
      C* m = static_cast<C*>(B.macro);
      m[0 * K.plane + cell] = rho;
      m[1 * K.plane + cell] = ux;
      m[2 * K.plane + cell] = uy;
      m[3 * K.plane + cell] = T;
      m[4 * K.plane + cell] = fs;
      m[5 * K.plane + cell] = eps;
      m[6 * K.plane + cell] = G;
    }
  }

  if (MODE != MODE_MACROS) {
    // ---- momentum-exchange partial sums per (tile, particle) -----------------
    for (int s = 0; s < np; ++s) {
      C v0 = C(0), v1 = C(0), v2 = C(0);
      bool mine = false;
#pragma unroll
      for (int k = 0; k < MAX_OWNERS; ++k)
        if (own[k] == s) { v0 = mesF[k][0]; v1 = mesF[k][1]; v2 = mesF[k][2]; mine = true; }
      if (!__syncthreads_or(mine)) {
        if (tid < 3) {
          const PartTile<C>& q = s_p[s];
          if (q.k >= 0) P.partial[((long long)q.id * K.kt + q.k) * 3 + tid] = 0.0;
        }
        continue;
      }
      v0 = warp_sum(v0); v1 = warp_sum(v1); v2 = warp_sum(v2);
      if (tx == 0) { s_red[ty][0] = v0; s_red[ty][1] = v1; s_red[ty][2] = v2; }
      __syncthreads();
      if (tid < 3) {
        C acc = C(0);
#pragma unroll
        for (int w = 0; w < TILE_Y; ++w) acc += s_red[w][tid];
        const PartTile<C>& q = s_p[s];
        if (q.k >= 0) P.partial[((long long)q.id * K.kt + q.k) * 3 + tid] = double(acc);
        else atomicOr(B.err, ERR_PARTIAL_OVERFLOW);
      }
      __syncthreads();
    }

    if (!active) return;

    // ---- MRT collision of f in moment space (Eqs. 3a, 4-7) ------------------
    {
      const C m1 = -C(4) * f[0] - (f[1] + f[2] + f[3] + f[4]) + C(2) * (f[5] + f[6] + f[7] + f[8]);
      const C m2 = C(4) * f[0] - C(2) * (f[1] + f[2] + f[3] + f[4]) + (f[5] + f[6] + f[7] + f[8]);
      const C m3 = jx;
      const C m4 = -C(2) * f[1] + C(2) * f[3] + f[5] - f[6] - f[7] + f[8];
      const C m5 = jy;
      const C m6 = -C(2) * f[2] + C(2) * f[4] + f[5] + f[6] - f[7] - f[8];
      const C m7 = f[1] - f[2] + f[3] - f[4];
      const C m8 = f[5] - f[6] + f[7] - f[8];
      // deviations of m^eq(rho, u) from m^eq(1, 0) (Eq. 6)
      const C u2 = ux * ux + uy * uy;
      const C e1 = -C(2) * drho + C(3) * rho * u2;
      const C e2 = drho - C(3) * rho * u2;
      const C e3 = rho * ux, e5 = rho * uy;
      const C e7 = rho * (ux * ux - uy * uy), e8 = rho * ux * uy;
      // forcing moments (Eq. 7)
      const C Fu = Fx * ux + Fy * uy;
      const C F7 = C(2) * (Fx * ux - Fy * uy), F8 = Fx * uy + Fy * ux;
      const C b0 = drho;
      const C b1 = m1 - K.s_e * (m1 - e1) + (C(1) - C(0.5) * K.s_e) * (C(6) * Fu);
      const C b2 = m2 - K.s_eps * (m2 - e2) + (C(1) - C(0.5) * K.s_eps) * (-C(6) * Fu);
      const C b3 = m3 - K.s_j * (m3 - e3) + (C(1) - C(0.5) * K.s_j) * Fx;
      const C b4 = m4 - K.s_q * (m4 + e3) + (C(1) - C(0.5) * K.s_q) * (-Fx);
      const C b5 = m5 - K.s_j * (m5 - e5) + (C(1) - C(0.5) * K.s_j) * Fy;
      const C b6 = m6 - K.s_q * (m6 + e5) + (C(1) - C(0.5) * K.s_q) * (-Fy);
      const C b7 = m7 - K.s_p * (m7 - e7) + (C(1) - C(0.5) * K.s_p) * F7;
      const C b8 = m8 - K.s_p * (m8 - e8) + (C(1) - C(0.5) * K.s_p) * F8;
      // f = M^-1 m = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) m
      const C a0 = b0 / C(9), a1 = b1 / C(36), a2 = b2 / C(36), a3 = b3 / C(6), a4 = b4 / C(12);
      const C a5 = b5 / C(6), a6 = b6 / C(12), a7 = b7 / C(4), a8 = b8 / C(4);
      S* dst = static_cast<S*>(B.dst);
      const C c14 = a0 - a1 - C(2) * a2;
      const C c58 = a0 + C(2) * a1 + a2;
      store_pop<C>(dst + 0 * K.plane + cell, a0 - C(4) * a1 + C(4) * a2);
      store_pop<C>(dst + 1 * K.plane + cell, c14 + a3 - C(2) * a4 + a7);
      store_pop<C>(dst + 2 * K.plane + cell, c14 + a5 - C(2) * a6 - a7);
      store_pop<C>(dst + 3 * K.plane + cell, c14 - a3 + C(2) * a4 + a7);
      store_pop<C>(dst + 4 * K.plane + cell, c14 - a5 + C(2) * a6 - a7);
      store_pop<C>(dst + 5 * K.plane + cell, c58 + a3 + a4 + a5 + a6 + a8);
      store_pop<C>(dst + 6 * K.plane + cell, c58 - a3 - a4 + a5 + a6 - a8);
      store_pop<C>(dst + 7 * K.plane + cell, c58 - a3 - a4 - a5 - a6 + a8);
      store_pop<C>(dst + 8 * K.plane + cell, c58 + a3 + a4 - a5 - a6 - a8);
    }

    // ---- MRT collision of g with the source term (Eqs. 17a, 18-20) ----------
    {
      const C n0 = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6] + g[7] + g[8];
      const C n1 = -C(4) * g[0] - (g[1] + g[2] + g[3] + g[4]) + C(2) * (g[5] + g[6] + g[7] + g[8]);
      const C n2 = C(4) * g[0] - C(2) * (g[1] + g[2] + g[3] + g[4]) + (g[5] + g[6] + g[7] + g[8]);
      const C n3 = g[1] - g[3] + g[5] - g[6] - g[7] + g[8];
      const C n4 = -C(2) * g[1] + C(2) * g[3] + g[5] - g[6] - g[7] + g[8];
      const C n5 = g[2] - g[4] + g[5] + g[6] - g[7] - g[8];
      const C n6 = -C(2) * g[2] + C(2) * g[4] + g[5] + g[6] - g[7] - g[8];
      const C n7 = g[1] - g[2] + g[3] - g[4];
      const C n8 = g[5] - g[6] + g[7] - g[8];
      const C sj = C(1) / tau_g;
      const C se = (K.rates_mode == C(0)) ? C(1) / (C(0.5) + C(0.25) / (tau_g - C(0.5))) : C(1);
      // n^eq = [eps, -4 eps + 2 c_ref T, 4 eps - 3 c_ref T, 0, ...]; q_m = [q, -4q, 4q, 0, ...]
      const C ct = K.cref * T;
      const C b0 = n0 - (n0 - eps) + C(0.5) * qc;  // sigma_0 = 1
      const C b1 = n1 - se * (n1 - (-C(4) * eps + C(2) * ct)) + (C(1) - C(0.5) * se) * (-C(4) * qc);
      const C b2 = n2 - se * (n2 - (C(4) * eps - C(3) * ct)) + (C(1) - C(0.5) * se) * (C(4) * qc);
      const C b3 = (C(1) - sj) * n3, b4 = (C(1) - sj) * n4;
      const C b5 = (C(1) - sj) * n5, b6 = (C(1) - sj) * n6;
      const C b7 = (C(1) - se) * n7, b8 = (C(1) - se) * n8;
      const C a0 = b0 / C(9), a1 = b1 / C(36), a2 = b2 / C(36), a3 = b3 / C(6), a4 = b4 / C(12);
      const C a5 = b5 / C(6), a6 = b6 / C(12), a7 = b7 / C(4), a8 = b8 / C(4);
      S* dst = static_cast<S*>(B.dst) + 9 * K.plane;
      const C c14 = a0 - a1 - C(2) * a2;
      const C c58 = a0 + C(2) * a1 + a2;
      store_pop<C>(dst + 0 * K.plane + cell, a0 - C(4) * a1 + C(4) * a2 - K.g_off[0]);
      store_pop<C>(dst + 1 * K.plane + cell, c14 + a3 - C(2) * a4 + a7 - K.g_off[1]);
      store_pop<C>(dst + 2 * K.plane + cell, c14 + a5 - C(2) * a6 - a7 - K.g_off[2]);
      store_pop<C>(dst + 3 * K.plane + cell, c14 - a3 + C(2) * a4 + a7 - K.g_off[3]);
      store_pop<C>(dst + 4 * K.plane + cell, c14 - a5 + C(2) * a6 - a7 - K.g_off[4]);
      store_pop<C>(dst + 5 * K.plane + cell, c58 + a3 + a4 + a5 + a6 + a8 - K.g_off[5]);
      store_pop<C>(dst + 6 * K.plane + cell, c58 - a3 - a4 + a5 + a6 - a8 - K.g_off[6]);
      store_pop<C>(dst + 7 * K.plane + cell, c58 - a3 - a4 - a5 - a6 + a8 - K.g_off[7]);
      store_pop<C>(dst + 8 * K.plane + cell, c58 + a3 + a4 - a5 - a6 - a8 - K.g_off[8]);
    }
    static_cast<C*>(B.s_dst)[cell] = C(2) * fs + dfs;
  }
}

// Ownership of every cell at the current level, from the same raster code as
// the lattice kernel (inspection of the integer part of Sec. 2's f_s).
template <class C>
__global__ void __launch_bounds__(TILE_X * TILE_Y)
raster_dump_kernel(const LatticeConst<C> K, const ParticleArrays P, const TileLists TL, unsigned char* count,
                   int* owner, unsigned char* flag, double* fsp, unsigned* err) {
  __shared__ int s_n;
  __shared__ int s_raw[TILE_CAP];
  __shared__ PartTile<C> s_p[TILE_CAP];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int np = load_tile_particles<C>(K, P, TL, blockIdx.x, blockIdx.y, &s_n, s_raw, s_p);
  const int x = blockIdx.x * TILE_X + tx, y = blockIdx.y * TILE_Y + ty;
  if (x >= K.nx || y >= K.ny) return;
  int nown, own[MAX_OWNERS], cls[MAX_OWNERS];
  C ofs[MAX_OWNERS];
  raster_cell<C>(tx, ty, np, s_p, nown, own, cls, ofs, err);
  const long long c = (long long)y * K.nx + x;
  count[c] = (unsigned char)nown;
#pragma unroll
  for (int k = 0; k < MAX_OWNERS; ++k) {
    owner[4 * c + k] = k < nown ? s_p[own[k]].id : -1;
    flag[4 * c + k] = (unsigned char)(k < nown ? cls[k] : 0);
    fsp[4 * c + k] = k < nown ? double(ofs[k]) : 0.0;
  }
}

// FP64 audit of the stored state: per-block sums of f (populations are
// deviations from w_i, so each cell adds 1), eps and g (macro planes 5, 6),
// then one ordered pass over the block sums.
template <class S, class C>
__global__ void audit_blocks_kernel(const LatticeConst<C> K, const S* pop, const C* macro, double* scratch,
                                    unsigned* err) {
  __shared__ double red[3][256];
  double sf = 0.0, se = 0.0, sg = 0.0;
  bool bad = false;
  const long long ncell = (long long)K.nx * K.ny;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const long long x = c % K.nx, y = c / K.nx;
    const long long cell = y * K.pitch + x;
    double cf = 1.0;
    for (int i = 0; i < 9; ++i) {
      const double v = double(pop[(long long)i * K.plane + cell]);
      const double w = double(pop[(long long)(9 + i) * K.plane + cell]);
      bad |= !(v == v) || !(w == w);
      cf += v;
    }
    sf += cf;
    se += double(macro[5 * K.plane + cell]);
    sg += double(macro[6 * K.plane + cell]);
  }
  if (bad) atomicOr(err, ERR_NAN);
  red[0][threadIdx.x] = sf;
  red[1][threadIdx.x] = se;
  red[2][threadIdx.x] = sg;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 3) scratch[3 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void audit_final_kernel(const double* scratch, int nblocks, double* out) {
  if (threadIdx.x >= 3) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += scratch[3 * b + threadIdx.x];
  out[threadIdx.x] = s;
}

template <class S, class C>
static cudaError_t launch_mode(int mode, const LatticeConst<C>& K, const StepBuffers& B,
                               const ParticleArrays& P, const TileLists& TL, cudaStream_t st) {
  dim3 grid(K.ntx, K.nty), block(TILE_X, TILE_Y);
  if (mode == MODE_INIT) lattice_kernel<S, C, MODE_INIT><<<grid, block, 0, st>>>(K, B, P, TL);
  else if (mode == MODE_STEP) lattice_kernel<S, C, MODE_STEP><<<grid, block, 0, st>>>(K, B, P, TL);
  else lattice_kernel<S, C, MODE_MACROS><<<grid, block, 0, st>>>(K, B, P, TL);
  return cudaGetLastError();
}

cudaError_t launch_lattice_f32(int mode, const LatticeConst<float>& K, const StepBuffers& B,
                               const ParticleArrays& P, const TileLists& TL, cudaStream_t st) {
  return launch_mode<float, float>(mode, K, B, P, TL, st);
}
cudaError_t launch_lattice_f64(int mode, const LatticeConst<double>& K, const StepBuffers& B,
                               const ParticleArrays& P, const TileLists& TL, cudaStream_t st) {
  return launch_mode<double, double>(mode, K, B, P, TL, st);
}

}  // namespace vlb

namespace vlb {

cudaError_t launch_raster_dump_f32(const LatticeConst<float>& K, const ParticleArrays& P,
                                   const TileLists& TL, unsigned char* count, int* owner,
                                   unsigned char* flag, double* fsp, unsigned* err, cudaStream_t st) {
  raster_dump_kernel<float><<<dim3(K.ntx, K.nty), dim3(TILE_X, TILE_Y), 0, st>>>(K, P, TL, count, owner, flag,
                                                                                 fsp, err);
  return cudaGetLastError();
}
cudaError_t launch_raster_dump_f64(const LatticeConst<double>& K, const ParticleArrays& P,
                                   const TileLists& TL, unsigned char* count, int* owner,
                                   unsigned char* flag, double* fsp, unsigned* err, cudaStream_t st) {
  raster_dump_kernel<double><<<dim3(K.ntx, K.nty), dim3(TILE_X, TILE_Y), 0, st>>>(K, P, TL, count, owner, flag,
                                                                                  fsp, err);
  return cudaGetLastError();
}

template <class S, class C>
static cudaError_t audit(const LatticeConst<C>& K, const void* pop, const void* macro, double* scratch,
                         int nblocks, double* out, unsigned* err, cudaStream_t st) {
  audit_blocks_kernel<S, C><<<nblocks, 256, 0, st>>>(K, static_cast<const S*>(pop),
                                                     static_cast<const C*>(macro), scratch, err);
  audit_final_kernel<<<1, 32, 0, st>>>(scratch, nblocks, out);
  return cudaGetLastError();
}
cudaError_t launch_audit_f32(const LatticeConst<float>& K, const void* pop, const void* macro, double* scratch,
                             int nblocks, double* out, unsigned* err, cudaStream_t st) {
  return audit<float, float>(K, pop, macro, scratch, nblocks, out, err, st);
}
cudaError_t launch_audit_f64(const LatticeConst<double>& K, const void* pop, const void* macro,
                             double* scratch, int nblocks, double* out, unsigned* err, cudaStream_t st) {
  return audit<double, double>(K, pop, macro, scratch, nblocks, out, err, st);
}

}  // namespace vlb
