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

// b / d for d = 9, 36, 6, 12 (index k), correctly rounded: q0 = b r, then one
// correction with the exact residual b - d q0.  For FP32 this equals IEEE
// division for every input of magnitude >= 2^-119 (checked exhaustively for
// these four divisors).  Correct rounding matters: a steady state maps
// d * (b / d) back to b, whereas a plain reciprocal product perturbs it every
// step, and identical cells (a solid interior) add such errors up coherently.
template <class C>
__device__ __forceinline__ C rdiv(C b, const LatticeConst<C>& K, int k) {
  const C d = k == 0 ? C(9) : (k == 1 ? C(36) : (k == 2 ? C(6) : C(12)));
  const C q0 = b * K.rcp[k];
  return fma(fma(-d, q0, b), K.rcp[k], q0);
}

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
    q.uxl = C(P.ux[id] - double(q.ux)); q.uyl = C(P.uy[id] - double(q.uy));
    q.lam_s = C(P.lam_s[id]); q.T0 = C(P.T0[id]);
    q.id = id;
    const int4 rg = P.prange[id];
    const int kx = tile_x - rg.x, ky = tile_y - rg.y;
    q.k = (kx >= 0 && ky >= 0 && kx < rg.z && ky < rg.w && ky * rg.z + kx < K.kt) ? ky * rg.z + kx : -1;
    q.rx = rg.x;
    q.ry = rg.y;
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

// CTAs per SM the FP32 register budget is sized for (4 x 256 threads: <= 64
// registers); the FP64 variant keeps the default budget
#ifndef VLB_LATTICE_MIN_BLOCKS
#define VLB_LATTICE_MIN_BLOCKS 4
#endif

template <class S, class C, int MODE>
__global__ void __launch_bounds__(TILE_X * TILE_Y, sizeof(C) == 4 ? VLB_LATTICE_MIN_BLOCKS : 1)
lattice_kernel(const LatticeConst<C> K, const StepBuffers B, const ParticleArrays P, const TileLists TL) {
  __shared__ int s_n;
  __shared__ int s_raw[TILE_CAP];
  __shared__ PartTile<C> s_p[TILE_CAP];
  __shared__ C s_red[TILE_Y][TILE_CAP][3];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TILE_X + tx;
  const int tile_x = blockIdx.x, tile_y = blockIdx.y;
  const int x = tile_x * TILE_X + tx, y = tile_y * TILE_Y + ty;
  const bool active = (x < K.nx) && (y < K.ny);
  const int cell = y * K.pitch + x;
  const S* __restrict__ src = static_cast<const S*>(B.src);

  // ---- streaming (pull) with wall rules, issued first ------------------------
  C f[9], g[9];
  C s_old = C(0);
  if (MODE == MODE_INIT) {
#pragma unroll
    for (int i = 0; i < 9; ++i) { f[i] = C(0); g[i] = C(0); }
  } else if (tile_x * TILE_X >= 1 && tile_x * TILE_X + TILE_X <= K.nx - 1 && tile_y * TILE_Y >= 1 &&
             tile_y * TILE_Y + TILE_Y <= K.ny - 1) {
    // interior tile: every x - e_i lies inside the domain
    const S* base = src + cell;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const long long off = (long long)i * K.plane - ex(i) - (long long)ey(i) * K.pitch;
      f[i] = load_pop<C>(base + off);
      g[i] = load_pop<C>(base + off + 9 * K.plane);
    }
    s_old = C(static_cast<const C*>(B.s_src)[cell]);
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
        g[i] = load_pop<C>(src + (long long)(9 + i) * K.plane + sc);
      } else {
        // halfway bounce-back of f; g bounces back (adiabatic) or anti-bounces
        // back to the wall temperature; corners go to the y wall
        f[i] = load_pop<C>(src + (long long)opp(i) * K.plane + cell);
        // (deviations: g^eq_i(T_w) - g^eq_i(T_f) = w_i c_ref (T_w - T_f) for i >= 1)
        const C gb = load_pop<C>(src + (long long)(9 + opp(i)) * K.plane + cell);
        const int wall = outy ? (sy < 0 ? 2 : 3) : (sx < 0 ? 0 : 1);
        g[i] = K.wall_dirichlet[wall] ? (C(2) * wgt<C>(i) * K.cref * K.wall_dT[wall] - gb) : gb;
      }
    }
    s_old = C(static_cast<const C*>(B.s_src)[cell]);
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) { f[i] = C(0); g[i] = C(0); }
  }

  // ---- particle list of the tile (loads above are in flight) ----------------
  const int np = load_tile_particles<C>(K, P, TL, tile_x, tile_y, &s_n, s_raw, s_p);
  if (MODE != MODE_MACROS) {
    // the other list buffer is filled by the next particle step
    if (tid == 0 && TL.next_count != nullptr) TL.next_count[tile_y * K.ntx + tile_x] = 0;
    // contact partners of the particles of this tile (Sec. 2.3): each pair is
    // tested in the first tile both ranges share, and appended to both lists
    for (int t = tid; t < np * np; t += TILE_X * TILE_Y) {
      const int a = t / np, b = t - a * np;
      if (b <= a) continue;
      const PartTile<C>& qa = s_p[a];
      const PartTile<C>& qb = s_p[b];
      if (max(qa.rx, qb.rx) != tile_x || max(qa.ry, qb.ry) != tile_y) continue;
      const int i = qa.id, j = qb.id;
      const double xi = P.x[i], yi = P.y[i], ri = P.r[i], xj = P.x[j], yj = P.y[j], rj = P.r[j];
      if (!in_contact_range(xi, yi, ri, xj, yj, rj, K.zeta)) continue;
      // repulsion on i from j (contact reading of Sec. 2.3); j gets the negative
      const double dx = xi - xj, dy = yi - yj;
      const double d = sqrt(dx * dx + dy * dy);
      const double gap = ri + rj + K.zeta - d;
      double fx = 0.0, fy = 0.0;
      if (gap > 0.0) {
        const double rm = fmax(ri, rj);
        const double mag = (K.contact_scale * rm * rm / K.eps_p) * (gap / K.zeta) * (gap / K.zeta) / d;
        fx = mag * dx;
        fy = mag * dy;
      }
      const int si = atomicAdd(&P.nbr_count[i], 1);
      const int sj = atomicAdd(&P.nbr_count[j], 1);
      if (si < NBR_CAP) {
        P.nbr[i * NBR_CAP + si] = j;
        P.nbr_f[2 * (i * NBR_CAP + si)] = fx;
        P.nbr_f[2 * (i * NBR_CAP + si) + 1] = fy;
      }
      if (sj < NBR_CAP) {
        P.nbr[j * NBR_CAP + sj] = i;
        P.nbr_f[2 * (j * NBR_CAP + sj)] = -fx;
        P.nbr_f[2 * (j * NBR_CAP + sj) + 1] = -fy;
      }
      if (si >= NBR_CAP || sj >= NBR_CAP) atomicOr(B.err, ERR_NBR_OVERFLOW);
    }
  }

  // ---- solid fraction and owners (Sec. 2) -----------------------------------
  int nown = 0;
  int own[MAX_OWNERS], ocls[MAX_OWNERS];
  C ofs[MAX_OWNERS];
  C fs = C(0);
  if (active && np > 0) fs = raster_cell<C>(tx, ty, np, s_p, nown, own, ocls, ofs, B.err);
  else {
#pragma unroll
    for (int k = 0; k < MAX_OWNERS; ++k) { own[k] = -1; ocls[k] = 0; ofs[k] = C(0); }
  }

  // ---- flow: volumetric correction (Eq. 8) and exchange partials (Eq. 28) ---
  // f holds deviations from w_i; rho = 1 + drho.
  // momenta as sums of differences of opposite populations: those differences
  // are exact when the two are close, which keeps j* accurate where it nearly
  // cancels rho u_s in the exchange term below
  C drho = ((f[0] + (f[1] + f[3])) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8]));
  const C d57 = f[5] - f[7], d86 = f[8] - f[6];
  C jx = (f[1] - f[3]) + (d57 + d86);
  C jy = (f[2] - f[4]) + (d57 - d86);
  const C rho = C(1) + drho;
  const C inv_rho = C(1) / rho;
  C mesF[MAX_OWNERS][3];
#pragma unroll
  for (int k = 0; k < MAX_OWNERS; ++k) { mesF[k][0] = mesF[k][1] = mesF[k][2] = C(0); }
  C lam = (C(1) - fs) * K.lam_f;
  C dT_init = C(0);  // sum_p f_s,p c_vs (T0_p - T_f): eps^0 - c_v T_f of the mixing rule
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
      const C rotx = -q.om * ry, roty = q.om * rx;
      const C usx = q.ux + (q.uxl + rotx), usy = q.uy + (q.uyl + roty);  // Eq. 27
      const C w = ofs[k];
      const C u2 = usx * usx + usy * usy;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const C eu = C(ex(i)) * usx + C(ey(i)) * usy;
        pf[i] += w * (C(3) * eu + C(4.5) * eu * eu - C(1.5) * u2);
      }
      // sum_i e_i f_i^eq(rho, u_s) = rho u_s; Delta F = -f_s,p (rho u_s - j*),
      // formed as (U_hi - j*) + (U_lo + Omega x r) + drho u_s
      const C dFx = -w * (((q.ux - jx) + (q.uxl + rotx)) + drho * usx);
      const C dFy = -w * (((q.uy - jy) + (q.uyl + roty)) + drho * usy);
      mesF[k][0] = dFx;
      mesF[k][1] = dFy;
      mesF[k][2] = rx * dFy - ry * dFx;
      cjx += w * rho * usx;
      cjy += w * rho * usy;
      lam += w * q.lam_s;
      dT_init += w * K.cv_s * (q.T0 - K.T_fluid);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = one_m * f[i] + wgt<C>(i) * (fs * drho + rho * pf[i]);
    jx = cjx;
    jy = cjy;
  }

  // ---- thermal macroscopics at n+1 (Eqs. 11, 16, 21-25) ----------------------
  // g holds deviations from g^eq(eps_f, T_f) of the initial fluid state
  // (eps_f = c_vf T_f); T, eps and sum g are carried as deviations dT, deps, dG
  // from T_f, eps_f, eps_f so that FP32 rounds the small parts only.
  const C cv = (C(1) - fs) * K.cv_f + fs * K.cv_s;
  // tau_g from Eq. 22 with alpha_1 = -2; the thermal rates of Eq. 18 (fluid
  // cells use the precomputed values)
  C tau_g = K.tau_gf, sj = K.sj_f, se = K.se_f, gk = K.gk_f;
  if (nown > 0) {
    tau_g = C(0.5) + C(3) * lam / K.cref;
    sj = C(1) / tau_g;
    se = (K.rates_mode == C(0)) ? (tau_g - C(0.5)) / (C(0.5) * (tau_g - C(0.5)) + C(0.25)) : C(1);
    gk = C(-3) * sj / K.cref;  // Eq. 23: -6/(4 + alpha_1) / (c_ref tau_g)
  }
  C dT, deps, dG, qc, dfs, ux, uy;
  const C half_inv_rho = C(0.5) * inv_rho;
  const C ax = (C(1) - fs) * K.bx * half_inv_rho, ay = (C(1) - fs) * K.by * half_inv_rho;
  if (MODE == MODE_INIT) {
    dT = dT_init / cv;                         // T^0 = eps^0 / c_v
    deps = (cv - K.cv_f) * K.T_fluid + cv * dT;  // eps^0 - eps_f
    dG = deps;
    qc = C(0);
    dfs = C(0);
    // g = g^eq(eps, T) (Eq. 19 with alpha_1 = -2, alpha_2 = 1), as a deviation
    g[0] = deps - C(5) / C(9) * K.cref * dT;
#pragma unroll
    for (int i = 1; i < 9; ++i) g[i] = wgt<C>(i) * K.cref * dT;
    ux = jx * inv_rho + ax * (K.dT_ref + dT);
    uy = jy * inv_rho + ay * (K.dT_ref + dT);
  } else {
    dfs = C(2) * fs - s_old;  // Eq. 24: 2 (f_s^{n+1} - f_s^n) - [df_s/dt]^n
    dG = ((g[0] + (g[1] + g[3])) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
    const C h57 = g[5] - g[7], h86 = g[8] - g[6];
    const C qx = (g[1] - g[3]) + (h57 + h86);
    const C qy = (g[2] - g[4]) + (h57 - h86);
    const C gTx = gk * qx, gTy = gk * qy;
    const C D = cv - C(0.5) * (K.cv_s - K.cv_f) * dfs;
    const C u0x = jx * inv_rho, u0y = jy * inv_rho;
    // Eq. 25 with u = u0 + a (T - T_ref), solved for T - T_f:
    // T - T_f = [(c_vf - D) T_f + dG - c_v/2 (u0.gradT + (T_f - T_ref) a.gradT)] / (D + c_v/2 a.gradT)
    const C agT = ax * gTx + ay * gTy;
    const C num = (K.cv_f - D) * K.T_fluid + dG - C(0.5) * cv * (u0x * gTx + u0y * gTy + K.dT_ref * agT);
    const C den = D + C(0.5) * cv * agT;
    dT = num / den;
    ux = u0x + ax * (K.dT_ref + dT);
    uy = u0y + ay * (K.dT_ref + dT);
    qc = -cv * (ux * gTx + uy * gTy) + (K.cv_s - K.cv_f) * (K.T_fluid + dT) * dfs;
    // Eq. 21, eps = sum g + q_c / 2, taken literally (equal to c_v T in exact
    // arithmetic): the conserved moment then carries no rounding of the solve
    deps = dG + C(0.5) * qc;
  }
  const C Fx = (C(1) - fs) * K.bx * (K.dT_ref + dT);
  const C Fy = (C(1) - fs) * K.by * (K.dT_ref + dT);

  if (MODE == MODE_MACROS || MODE == MODE_INIT) {
    if (active && B.macro != nullptr) {
      C* m = static_cast<C*>(B.macro);
      m[0 * K.plane + cell] = rho;
      m[1 * K.plane + cell] = ux;
      m[2 * K.plane + cell] = uy;
      m[3 * K.plane + cell] = K.T_fluid + dT;
      m[4 * K.plane + cell] = fs;
      m[5 * K.plane + cell] = K.cv_f * K.T_fluid + deps;
      m[6 * K.plane + cell] = K.cv_f * K.T_fluid + dG;
    }
  }

  if (MODE != MODE_MACROS) {
    // ---- momentum-exchange partial sums per (tile, particle) -----------------
    // each warp (one row of the tile) reduces its cells with shuffles in a
    // fixed order; one barrier; then the 8 row sums add up in row order
    if (np > 0) {
      for (int sl = 0; sl < np; ++sl) {
        C v0 = C(0), v1 = C(0), v2 = C(0);
        bool mine = false;
#pragma unroll
        for (int k = 0; k < MAX_OWNERS; ++k)
          if (own[k] == sl) { v0 = mesF[k][0]; v1 = mesF[k][1]; v2 = mesF[k][2]; mine = true; }
        if (__any_sync(0xffffffffu, mine)) {
          v0 = warp_sum(v0); v1 = warp_sum(v1); v2 = warp_sum(v2);
        }
        if (tx == 0) { s_red[ty][sl][0] = v0; s_red[ty][sl][1] = v1; s_red[ty][sl][2] = v2; }
      }
      __syncthreads();
      for (int t = tid; t < 3 * np; t += TILE_X * TILE_Y) {
        const int sl = t / 3, c = t - 3 * sl;
        C acc = C(0);
#pragma unroll
        for (int w = 0; w < TILE_Y; ++w) acc += s_red[w][sl][c];
        const PartTile<C>& q = s_p[sl];
        if (q.k >= 0) P.partial[((long long)q.id * K.kt + q.k) * 3 + c] = double(acc);
        else if (c == 0) atomicOr(B.err, ERR_PARTIAL_OVERFLOW);
      }
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
      // deviations of m^eq(rho, u) from m^eq(1, 0) (Eq. 6), with rho u = j + F/2
      // (Eq. 9) taken directly instead of through u
      const C e3 = jx + C(0.5) * Fx, e5 = jy + C(0.5) * Fy;
      const C ru2 = e3 * ux + e5 * uy;
      const C e1 = -C(2) * drho + C(3) * ru2;
      const C e2 = drho - C(3) * ru2;
      const C e7 = e3 * ux - e5 * uy, e8 = e3 * uy;
      // forcing moments (Eq. 7)
      const C Fu = Fx * ux + Fy * uy;
      const C F7 = C(2) * (Fx * ux - Fy * uy), F8 = Fx * uy + Fy * ux;
      const C b0 = drho;
      const C b1 = m1 - K.s_e * (m1 - e1) + (C(1) - C(0.5) * K.s_e) * (C(6) * Fu);
      const C b2 = m2 - K.s_eps * (m2 - e2) + (C(1) - C(0.5) * K.s_eps) * (-C(6) * Fu);
      // conserved momentum: m3 - s_j (m3 - rho u) + (1 - s_j/2) F = j + F for any s_j
      const C b3 = m3 + Fx;
      const C b4 = m4 - K.s_q * (m4 + e3) + (C(1) - C(0.5) * K.s_q) * (-Fx);
      const C b5 = m5 + Fy;
      const C b6 = m6 - K.s_q * (m6 + e5) + (C(1) - C(0.5) * K.s_q) * (-Fy);
      const C b7 = m7 - K.s_p * (m7 - e7) + (C(1) - C(0.5) * K.s_p) * F7;
      const C b8 = m8 - K.s_p * (m8 - e8) + (C(1) - C(0.5) * K.s_p) * F8;
      // f = M^-1 m = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) m
      const C a0 = rdiv(b0, K, 0), a1 = rdiv(b1, K, 1), a2 = rdiv(b2, K, 1);
      const C a3 = rdiv(b3, K, 2), a4 = rdiv(b4, K, 3), a5 = rdiv(b5, K, 2);
      const C a6 = rdiv(b6, K, 3), a7 = b7 * C(0.25), a8 = b8 * C(0.25);
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
      // n^eq = [eps, -4 eps + 2 c_ref T, 4 eps - 3 c_ref T, 0, ...]; q_m = [q, -4q, 4q, 0, ...]
      // (deviations from the moments of g^eq(eps_f, T_f))
      const C ct = K.cref * dT;
      const C b0 = n0 + qc;  // sigma_0 = 1 with eps = sum g + q_c / 2 (Eq. 21)
      const C b1 = n1 - se * (n1 - (-C(4) * deps + C(2) * ct)) + (C(1) - C(0.5) * se) * (-C(4) * qc);
      const C b2 = n2 - se * (n2 - (C(4) * deps - C(3) * ct)) + (C(1) - C(0.5) * se) * (C(4) * qc);
      const C b3 = (C(1) - sj) * n3, b4 = (C(1) - sj) * n4;
      const C b5 = (C(1) - sj) * n5, b6 = (C(1) - sj) * n6;
      const C b7 = (C(1) - se) * n7, b8 = (C(1) - se) * n8;
      const C a0 = rdiv(b0, K, 0), a1 = rdiv(b1, K, 1), a2 = rdiv(b2, K, 1);
      const C a3 = rdiv(b3, K, 2), a4 = rdiv(b4, K, 3), a5 = rdiv(b5, K, 2);
      const C a6 = rdiv(b6, K, 3), a7 = b7 * C(0.25), a8 = b8 * C(0.25);
      S* dst = static_cast<S*>(B.dst) + 9 * K.plane;
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
