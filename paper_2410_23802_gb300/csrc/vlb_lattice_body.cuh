// Device code of one lattice time step at one cell, shared by the
// single-case kernels (vlb_lattice.cu) and the batched ones (vlb_batch.cu).
//
// The fused lattice kernel: one pass over the lattice per time step.
//
// Per cell, in registers:  pull f-bar and g-bar from the neighbours (Eqs. 3b,
// 17b) with wall rules; f_s^{n+1} from the tile's particle list (Sec. 2);
// volumetric correction of f (Eq. 8) and the momentum-exchange sums of
// Eq. 28 (per row of the tile, added to per-particle integer accumulators); df_s/dt (Eq. 24), c_v and lambda (Eq. 11), grad T (Eq. 23), T
// jointly with u and the buoyancy force (Eqs. 9, 25), eps and q_c (Eqs. 16,
// 21); both MRT collisions (Eqs. 3a, 17a); stores of f-bar, g-bar and
// S = 2 f_s + df_s/dt at level n+1.
//
// Layout in HBM: structure of arrays, one plane per direction, x fastest,
// rows padded to 32 B.  f is stored as the deviation from the rest
// equilibrium w_i, g as the deviation from g^eq(T_fluid) (g_off), S in the
// arithmetic type.  Populations ping-pong between two buffers.
#pragma once

#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "vlb_common.cuh"
#include "vlb_raster.cuh"
#include "vlb_kernels.h"

namespace vlb {

// Population loads and streaming stores for FP64, FP32, FP16 and BF16 storage.
// FP16 holds the deviation times 2^12: the deviations of a slow flow (of order
// w_i 3 |u| ~ 1e-5 at |u| ~ 1e-4) lie below FP16's smallest normal number
// (6.1e-5), where its spacing is a fixed 6e-8 and the relative precision
// drops to 1e-2 .. 1e-3; scaled, they keep the full 11 bits down to 1.5e-8,
// and deviations up to 16 stay below FP16's largest value.  The power of two
// scales exactly.  BF16 has FP32's exponent range and needs no scale.
constexpr float FP16_SCALE = 4096.0f;
constexpr float FP16_UNSCALE = 1.0f / 4096.0f;
template <class C, class S>
__device__ __forceinline__ C stored_value(S v) { return C(v); }
template <>
__device__ __forceinline__ float stored_value<float, __half>(__half v) { return __half2float(v) * FP16_UNSCALE; }
template <>
__device__ __forceinline__ float stored_value<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <class C, class S>
__device__ __forceinline__ C load_pop(const S* p) { return stored_value<C, S>(__ldg(p)); }

// Stores of the nine post-collision populations o[i] of one distribution
// into planes i of dst.  FP32 and FP64 storage keep the value.  16-bit
// storage rounds stochastically: a value between two neighbouring 16-bit
// numbers goes up with probability equal to its distance from the lower one,
// so the rounding error has zero mean and does not repeat from step to step.
// Round-to-nearest makes the same error every step wherever the flow is
// steady (the inside of a translating disk, say), and those errors add up
// coherently in the exchange force of Eq. 28: on the settling-disk channel
// that bias, not the noise, took FP16 to 1.2e-3 and BF16 to 2.9e-2 relative
// L2 in u over 1000 steps.  The rounding is the hardware conversion with
// random bits (cvt.rs); the bits come from a counter-based hash of the cell's
// index in its lattice and the level stamp, so a case draws the same bits
// alone, in a batch or after a checkpoint.
template <class C, class S>
__device__ __forceinline__ void store_pop(S* p, C v) { __stcs(p, S(v)); }

// The "lowbias32" integer hash (C. Wellons, hash-prospector, 2018).
__device__ __forceinline__ unsigned lowbias32(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}
// Random key of one cell at one level.
__device__ __forceinline__ unsigned sr_key(int cell_index, int stamp) {
  return lowbias32((unsigned)cell_index ^ lowbias32((unsigned)stamp));
}
// Odd multipliers that spread one key into independent-looking words, one
// per packed conversion (five for f, five for g).
__device__ __forceinline__ unsigned sr_word(unsigned key, int k) {
  constexpr unsigned m[10] = {0x9E3779B1u, 0x85EBCA77u, 0xC2B2AE3Du, 0x27D4EB2Fu, 0x165667B1u,
                              0xD3A2646Cu | 1u, 0xFD7046C5u, 0xB55A4F09u, 0x2545F491u, 0x4F1BBCDDu};
  return key * m[k];
}
template <class S>
__device__ __forceinline__ unsigned cvt_rs2(float hi, float lo, unsigned rbits);
template <>
__device__ __forceinline__ unsigned cvt_rs2<__half>(float hi, float lo, unsigned rbits) {
  unsigned d;
  asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}
template <>
__device__ __forceinline__ unsigned cvt_rs2<__nv_bfloat16>(float hi, float lo, unsigned rbits) {
  unsigned d;
  asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}
template <class S>
__device__ __forceinline__ void store_half_bits(S* p, unsigned short b);
template <>
__device__ __forceinline__ void store_half_bits<__half>(__half* p, unsigned short b) { __stcs(p, __ushort_as_half(b)); }
template <>
__device__ __forceinline__ void store_half_bits<__nv_bfloat16>(__nv_bfloat16* p, unsigned short b) {
  __stcs(p, __ushort_as_bfloat16(b));
}

// word0: index of the first of the five random words of this distribution
template <class S, class C>
__device__ __forceinline__ void store_pops(S* dst, long long plane, int cell, const C (&o)[9], unsigned key,
                                           int word0) {
  if constexpr (sizeof(S) == 2) {
    constexpr float sc = std::is_same<S, __half>::value ? FP16_SCALE : 1.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned d = cvt_rs2<S>(sc * o[2 * k + 1], sc * o[2 * k], sr_word(key, word0 + k));
      store_half_bits<S>(dst + (2 * k) * plane + cell, (unsigned short)(d & 0xffffu));
      store_half_bits<S>(dst + (2 * k + 1) * plane + cell, (unsigned short)(d >> 16));
    }
    const unsigned d = cvt_rs2<S>(0.0f, sc * o[8], sr_word(key, word0 + 4));
    store_half_bits<S>(dst + 8 * plane + cell, (unsigned short)(d & 0xffffu));
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) store_pop<C>(dst + i * plane + cell, o[i]);
  }
}

template <class C>
__device__ __forceinline__ C warp_sum(C v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared memory of one tile: its particles.
template <class C>
struct TileShared {
  PartTile<C> p[TILE_CAP];
};

// Particle list of one tile, sorted by id (rank sort; ids are unique), with
// each particle's geometry relative to the tile origin.  Returns the count.
// Every thread reads the count itself, so a tile without particles passes no
// barrier; otherwise one barrier publishes the records.
template <class C>
__device__ int load_tile_particles(const LatticeConst<C>& K, const ParticleArrays& P, const TileLists& TL,
                                   int tile_x, int tile_y, TileShared<C>& sh) {
  PartTile<C>* s_p = sh.p;
  const int tid = threadIdx.y * TILE_X + threadIdx.x;
  const int tile = tile_y * K.ntx + tile_x;
  const int x0 = tile_x * TILE_X, y0 = tile_y * TILE_Y;
  // warp 0 reads the list's slots together with the count (slots beyond the
  // count hold stale ids and are ignored), so the records wait on one load
  int sid = 0;
  if (tid < TILE_CAP) sid = TL.ids[(long long)tile * TILE_CAP + tid];
  const int c = TL.count[tile];
  const int np = c < TILE_CAP ? c : TILE_CAP;
  if (np == 0) return 0;
  if (tid < 32) {  // warp 0 (TILE_CAP = 32): rank the ids with shuffles
    const int id = tid < np ? sid : 0x7fffffff;
    int rank = 0;  // ids are unique: rank = number of smaller ids
    for (int k = 0; k < np; ++k) rank += __shfl_sync(0xffffffffu, id, k) < id;
    if (tid < np) {
    PartTile<C> q;
    if constexpr (sizeof(C) == 4) {
      // FP32 kernel: the particle kernel's raster record, no FP64 arithmetic
      // (the geometry the band kernel used for this tile)
      const RasterRec rc = P.rec[id];
      tile_geometry(rc, x0, y0, q);
      q.ux = rc.ux; q.uxl = rc.uxl; q.uy = rc.uy; q.uyl = rc.uyl; q.om = rc.om;
      q.lam_s = rc.lam_s; q.T0 = rc.T0;
      q.fixed = P.fixed_T[id];
    } else {
      const double X = P.x[id] - double(x0), Y = P.y[id] - double(y0), R = P.r[id];
      const long long Q = 1ll << QBITS;
      q.xq = __double2ll_rn(P.x[id] * double(Q)) - (long long)x0 * Q;
      q.yq = __double2ll_rn(P.y[id] * double(Q)) - (long long)y0 * Q;
      const long long rq = __double2ll_rn(R * double(Q));
      q.rq2 = rq * rq;
      q.xh = C(X); q.xl = C(X - double(q.xh));
      q.yh = C(Y); q.yl = C(Y - double(q.yh));
      const double Rb = P.rb[id];
      q.r = C(R);
      q.far2 = C((R + 0.75) * (R + 0.75));
      q.near2 = Rb > 0.75 ? C((Rb - 0.75) * (Rb - 0.75)) : C(-1);
      q.ell = Rb != R;  // an ellipse: semi-axes R >= Rb (reading R13)
      q.ex = P.x[id]; q.ey = P.y[id]; q.ea = R; q.eb = Rb;
      q.ec = 1.0; q.es = 0.0;
      if (q.ell) sincos(P.theta[id], &q.es, &q.ec);
      q.ux = C(P.ux[id]); q.uy = C(P.uy[id]); q.om = C(P.om[id]);
      q.uxl = C(P.ux[id] - double(q.ux)); q.uyl = C(P.uy[id] - double(q.uy));
      q.lam_s = C(P.lam_s[id]); q.T0 = C(P.T0[id]);
      q.ci = 0; q.cj = 0;
      q.fixed = P.fixed_T[id];
    }
    q.id = id;
    const int4 rg = P.prange[id];
    q.rx = rg.x;
    q.ry = rg.y;
    s_p[rank] = q;
    }
  }
  __syncthreads();
  return np;
}

// Owners of cell (tx, ty) of the tile: ascending particle order, at most
// MAX_OWNERS, fractions scaled to sum 1 when they exceed it (overlap).  The
// FP32 kernel reads the exact class and area of band cells from the band
// tables (gx, gy: the cell's lattice coordinates), which must carry the
// level's stamp; the FP64 kernel computes them here.
template <class C>
__device__ __forceinline__ C raster_cell(int tx, int ty, int gx, int gy, int np, const PartTile<C>* s_p,
                                         const int2* __restrict__ band, int band_off, int band_stamp,
                                         int& nown, int (&own)[MAX_OWNERS], int (&cls)[MAX_OWNERS],
                                         C (&ofs)[MAX_OWNERS], unsigned* err) {
  nown = 0;
#pragma unroll
  for (int k = 0; k < MAX_OWNERS; ++k) { own[k] = -1; cls[k] = 0; ofs[k] = C(0); }
  for (int s = 0; s < np; ++s) {
    C f;
    int c;
    if constexpr (sizeof(C) == 4) {
      const PartTile<C>& q = s_p[s];
      c = quick_class(tx, ty, q);
      if (c == CELL_FLUID) continue;
      if (c == CELL_SOLID) {
        f = C(1);
      } else {
        const int bw = 2 * band_off + 1;
        const int bx = gx - q.ci + band_off, by = gy - q.cj + band_off;
        int2 e = make_int2(0, 0);
        if ((unsigned)bx < (unsigned)bw && (unsigned)by < (unsigned)bw)
          e = band[((long long)q.id * bw + by) * bw + bx];
        if ((e.x >> 2) != band_stamp) {  // not written for this level (cannot happen)
          atomicOr(err, ERR_BAND);
          continue;
        }
        c = e.x & 3;
        f = __int_as_float(e.y);
        if (c == CELL_FLUID) continue;
      }
    } else {
      c = s_p[s].ell ? ellipse_cell_fraction(tx, ty, gx, gy, s_p[s], f) : cell_fraction(tx, ty, s_p[s], f);
      if (c == CELL_FLUID) continue;
    }
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

// CTAs per SM the FP32 register budget is sized for (1024 threads per SM:
// <= 64 registers); the FP64 variant keeps the default budget
#ifndef VLB_LATTICE_MIN_BLOCKS
#define VLB_LATTICE_MIN_BLOCKS (1024 / (TILE_X * TILE_Y))
#endif

// Pull streaming of one cell (Eqs. 3b, 17b) with the wall rules: f-bar and
// g-bar of x - e_i, or the bounced value at a wall; S of level n.
template <class S, class C, int MODE>
__device__ __forceinline__ void pull_direct(const LatticeConst<C>& K, const StepBuffers& B, int tile_x, int tile_y,
                                            C (&f)[9], C (&g)[9], C& s_old) {
  const int x = tile_x * TILE_X + threadIdx.x, y = tile_y * TILE_Y + threadIdx.y;
  const bool active = (x < K.nx) && (y < K.ny);
  const int cell = y * K.pitch + x;
  const S* __restrict__ src = static_cast<const S*>(B.src);
  s_old = C(0);
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
      // an open side (reading R14): the population takes the value of the
      // same population one cell further in, i.e. the source moved back
      // across the side(s) it crossed; a corner under a closed side bounces
      // off that side
      if (outx && (sx < 0 ? K.outflow[0] : K.outflow[1])) { sx = x; outx = false; }
      if (outy && (sy < 0 ? K.outflow[2] : K.outflow[3])) { sy = y; outy = false; }
      if (!(outx || outy)) {
        const long long sc = (long long)sy * K.pitch + sx;
        f[i] = load_pop<C>(src + (long long)i * K.plane + sc);
        g[i] = load_pop<C>(src + (long long)(9 + i) * K.plane + sc);
      } else {
        // halfway bounce-back of f; g bounces back (adiabatic) or anti-bounces
        // back to the wall temperature; corners between closed sides go to
        // the y wall
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

}

// Everything of one time step at one cell after the pull: the tile's particle
// list, f_s and owners, correction, thermal macroscopics, exchange sums,
// both collisions and the stores.  Called by every thread of the CTA (it has
// barriers); returns the tile's particle count.
template <class S, class C, int MODE, bool HOLD>
__device__ __forceinline__ int cell_body(const LatticeConst<C>& K, const StepBuffers& B, const ParticleArrays& P,
                                         const TileLists& TL, int tile_x, int tile_y, C (&f)[9], C (&g)[9],
                                         const C s_old, TileShared<C>& sh, int band_stamp) {
  const PartTile<C>* s_p = sh.p;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TILE_X + tx;
  const int x = tile_x * TILE_X + tx, y = tile_y * TILE_Y + ty;
  const bool active = (x < K.nx) && (y < K.ny);
  const int cell = y * K.pitch + x;

  // ---- particle list of the tile (loads above are in flight) ----------------
  const int np = load_tile_particles<C>(K, P, TL, tile_x, tile_y, sh);
  if (MODE != MODE_MACROS) {
    // the other list buffer is filled by the next particle step
    if (tid == 0 && TL.next_count != nullptr) TL.next_count[tile_y * K.ntx + tile_x] = 0;
    // contact partners of the particles of this tile (Sec. 2.3): each pair is
    // tested in the first tile both ranges share, and appended to both lists
    for (int t = tid; t < np * np; t += TILE_X * TILE_Y) {
      const int a = t / max(np, 1), b = t - a * np;
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
      // the force goes into both particles' integer force accumulators (+F on
      // i, -F on j: exact negation, so F_ji = -F_ij and the sum over all
      // pairs does not depend on the order); the partner lists are kept for
      // inspection
      if (fx != 0.0 || fy != 0.0) {
        mes_add(P.mes + 6 * (long long)i, fx, B.err);
        mes_add(P.mes + 6 * (long long)i + 2, fy, B.err);
        mes_add(P.mes + 6 * (long long)j, -fx, B.err);
        mes_add(P.mes + 6 * (long long)j + 2, -fy, B.err);
      }
      const int si = atomicAdd(&P.nbr_count[i], 1);
      const int sj = atomicAdd(&P.nbr_count[j], 1);
      if (si < NBR_CAP) P.nbr[i * NBR_CAP + si] = j;
      if (sj < NBR_CAP) P.nbr[j * NBR_CAP + sj] = i;
      if (si >= NBR_CAP || sj >= NBR_CAP) atomicOr(B.err, ERR_NBR_OVERFLOW);
    }

  }

  // ---- solid fraction and owners (Sec. 2) -----------------------------------
  int nown = 0;
  int own[MAX_OWNERS], ocls[MAX_OWNERS];
  C ofs[MAX_OWNERS];
  C fs = C(0);
  if (active && np > 0)
    fs = raster_cell<C>(tx, ty, x, y, np, s_p, P.band, K.band_off, band_stamp, nown, own, ocls, ofs, B.err);
  else {
#pragma unroll
    for (int k = 0; k < MAX_OWNERS; ++k) { own[k] = -1; ocls[k] = 0; ofs[k] = C(0); }
  }

  // ---- flow: volumetric correction (Eq. 8) and the exchange terms (Eq. 28) ---
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
  const C jxs = jx, jys = jy;  // j* before the correction (for the exchange term)
  C lam = (C(1) - fs) * K.lam_f;
  C dT_init = C(0);  // sum_p f_s,p c_vs (T0_p - T_f): eps^0 - c_v T_f of the mixing rule
  if (nown > 0) {
    const C one_m = C(1) - fs;
    C pf[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) pf[i] = C(0);
    C cjx = one_m * jx, cjy = one_m * jy;
    C hfix = C(0), h0 = C(0), hr = C(0);  // held owners: covered fraction, g^eq deviations
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
      cjx += w * rho * usx;
      cjy += w * rho * usy;
      lam += w * q.lam_s;
      if (HOLD && q.fixed) {
        // held at T_p = T0: its part of the cell (reading R11), or the whole
        // cell (fixed == 2, reading R11b), takes g^eq(c_vs T_p, T_p), here as
        // the deviation from g^eq(eps_f, T_f)
        const C dTp = q.T0 - K.T_fluid;
        const C wh = q.fixed == 2 ? C(1) : w;
        hfix += wh;
        h0 += wh * ((K.cv_s * q.T0 - K.cv_f * K.T_fluid) - C(5.0 / 9.0) * K.cref * dTp);
        hr += wh * K.cref * dTp;
      }
      dT_init += w * K.cv_s * (q.T0 - K.T_fluid);
      if (MODE != MODE_MACROS) {
        // momentum exchange (Eq. 28), added to the particle's integer
        // accumulators (no reduction, no barrier; a total independent of the
        // order): sum_i e_i f_i^eq(rho, u_s) = rho u_s, so Delta F =
        // -f_s,p (rho u_s - j*), formed as (U_hi - j*) + (U_lo + Omega x r) + drho u_s
        const C v0 = -w * (((q.ux - jxs) + (q.uxl + rotx)) + drho * usx);
        const C v1 = -w * (((q.uy - jys) + (q.uyl + roty)) + drho * usy);
        const C v2 = rx * v1 - ry * v0;
        unsigned long long* acc = P.mes + 6 * (long long)q.id;
        mes_add(acc, v0, B.err);
        mes_add(acc + 2, v1, B.err);
        mes_add(acc + 4, v2, B.err);
      }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = one_m * f[i] + wgt<C>(i) * (fs * drho + rho * pf[i]);
    jx = cjx;
    jy = cjy;
    if (HOLD && hfix > C(0)) {  // g = (1 - f_fix) g + sum over held owners of f_s,p g^eq(c_vs T_p, T_p)
      if (hfix > C(1)) {  // whole-cell holds of several owners: their mean
        const C inv = C(1) / hfix;
        h0 *= inv;
        hr *= inv;
        hfix = C(1);
      }
      const C keep = C(1) - hfix;
      g[0] = keep * g[0] + h0;
#pragma unroll
      for (int i = 1; i < 9; ++i) g[i] = keep * g[i] + wgt<C>(i) * hr;
    }
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
    tau_g = C(0.5) + lam * K.k3_cref;  // 3 / c_ref
    sj = C(1) / tau_g;
    se = (K.rates_mode == C(0)) ? (tau_g - C(0.5)) / (C(0.5) * (tau_g - C(0.5)) + C(0.25)) : C(1);
    gk = -sj * K.k3_cref;  // Eq. 23: -6/(4 + alpha_1) / (c_ref tau_g)
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
    if (!active) return np;
    // random key of stochastic rounding (16-bit storage only)
    const unsigned skey = sizeof(S) == 2 ? sr_key(y * K.nx + x, band_stamp) : 0u;

    // ---- MRT collision of f in moment space (Eqs. 3a, 4-7) ------------------
    // Written as f-bar = f + M^-1 (m-bar - m): only the relaxed moments and the
    // forcing change, and M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6,
    // 1/12, 1/4, 1/4).  The conserved moments get exactly rho and j + F
    // (Eq. 9: rho u = j + F/2); in cells the correction touched, whose f carries
    // FP32-rounded weights, the difference to those targets is put back here
    // so that no rounding bias repeats step after step.
    {
      const C m1 = -C(4) * f[0] - (f[1] + f[2] + f[3] + f[4]) + C(2) * (f[5] + f[6] + f[7] + f[8]);
      const C m2 = C(4) * f[0] - C(2) * (f[1] + f[2] + f[3] + f[4]) + (f[5] + f[6] + f[7] + f[8]);
      const C m4 = -C(2) * f[1] + C(2) * f[3] + f[5] - f[6] - f[7] + f[8];
      const C m6 = -C(2) * f[2] + C(2) * f[4] + f[5] + f[6] - f[7] - f[8];
      const C m7 = f[1] - f[2] + f[3] - f[4];
      const C m8 = f[5] - f[6] + f[7] - f[8];
      // deviations of m^eq(rho, u) from m^eq(1, 0) (Eq. 6), with rho u = j + F/2
      const C e3 = jx + C(0.5) * Fx, e5 = jy + C(0.5) * Fy;
      const C ru2 = e3 * ux + e5 * uy;
      const C e1 = -C(2) * drho + C(3) * ru2;
      const C e2 = drho - C(3) * ru2;
      const C e7 = e3 * ux - e5 * uy, e8 = e3 * uy;
      // forcing moments (Eq. 7)
      const C Fu = Fx * ux + Fy * uy;
      const C F7 = C(2) * (Fx * ux - Fy * uy), F8 = Fx * uy + Fy * ux;
      const C d1 = -K.s_e * (m1 - e1) + (C(1) - C(0.5) * K.s_e) * (C(6) * Fu);
      const C d2 = -K.s_eps * (m2 - e2) + (C(1) - C(0.5) * K.s_eps) * (-C(6) * Fu);
      const C d4 = -K.s_q * (m4 + e3) + (C(1) - C(0.5) * K.s_q) * (-Fx);
      const C d6 = -K.s_q * (m6 + e5) + (C(1) - C(0.5) * K.s_q) * (-Fy);
      const C d7 = -K.s_p * (m7 - e7) + (C(1) - C(0.5) * K.s_p) * F7;
      const C d8 = -K.s_p * (m8 - e8) + (C(1) - C(0.5) * K.s_p) * F8;
      // conserved moments: m-bar_0 = rho, m-bar_3 = j_x + F_x, m-bar_5 = j_y + F_y
      C d0 = C(0), d3 = Fx, d5 = Fy;
      if (nown > 0) {
        const C n0 = ((f[0] + (f[1] + f[3])) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8]));
        const C q57 = f[5] - f[7], q86 = f[8] - f[6];
        d0 = drho - n0;
        d3 = (jx - ((f[1] - f[3]) + (q57 + q86))) + Fx;
        d5 = (jy - ((f[2] - f[4]) + (q57 - q86))) + Fy;
      }
      const C a0 = d0 * C(1.0 / 9.0), a1 = d1 * C(1.0 / 36.0), a2 = d2 * C(1.0 / 36.0);
      const C a3 = d3 * C(1.0 / 6.0), a4 = d4 * C(1.0 / 12.0), a5 = d5 * C(1.0 / 6.0);
      const C a6 = d6 * C(1.0 / 12.0), a7 = d7 * C(0.25), a8 = d8 * C(0.25);
      S* dst = static_cast<S*>(B.dst);
      const C c14 = a0 - a1 - C(2) * a2;
      const C c58 = a0 + C(2) * a1 + a2;
      const C o[9] = {f[0] + (a0 - C(4) * a1 + C(4) * a2), f[1] + (c14 + a3 - C(2) * a4 + a7),
                      f[2] + (c14 + a5 - C(2) * a6 - a7),  f[3] + (c14 - a3 + C(2) * a4 + a7),
                      f[4] + (c14 - a5 + C(2) * a6 - a7),  f[5] + (c58 + a3 + a4 + a5 + a6 + a8),
                      f[6] + (c58 - a3 - a4 + a5 + a6 - a8), f[7] + (c58 - a3 - a4 - a5 - a6 + a8),
                      f[8] + (c58 + a3 + a4 - a5 - a6 - a8)};
      store_pops<S, C>(dst, K.plane, cell, o, skey, 0);
    }

    // ---- MRT collision of g with the source term (Eqs. 17a, 18-20) ----------
    // The same delta form: n-bar - n for the relaxed moments and the source;
    // the conserved moment gets sum g + q_c exactly (sigma_0 = 1 with
    // eps = sum g + q_c / 2, Eq. 21).
    {
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
      const C d1 = -se * (n1 - (-C(4) * deps + C(2) * ct)) + (C(1) - C(0.5) * se) * (-C(4) * qc);
      const C d2 = -se * (n2 - (C(4) * deps - C(3) * ct)) + (C(1) - C(0.5) * se) * (C(4) * qc);
      const C a0 = qc * C(1.0 / 9.0), a1 = d1 * C(1.0 / 36.0), a2 = d2 * C(1.0 / 36.0);
      const C a3 = -sj * n3 * C(1.0 / 6.0), a4 = -sj * n4 * C(1.0 / 12.0);
      const C a5 = -sj * n5 * C(1.0 / 6.0), a6 = -sj * n6 * C(1.0 / 12.0);
      const C a7 = -se * n7 * C(0.25), a8 = -se * n8 * C(0.25);
      S* dst = static_cast<S*>(B.dst) + 9 * K.plane;
      const C c14 = a0 - a1 - C(2) * a2;
      const C c58 = a0 + C(2) * a1 + a2;
      const C o[9] = {g[0] + (a0 - C(4) * a1 + C(4) * a2), g[1] + (c14 + a3 - C(2) * a4 + a7),
                      g[2] + (c14 + a5 - C(2) * a6 - a7),  g[3] + (c14 - a3 + C(2) * a4 + a7),
                      g[4] + (c14 - a5 + C(2) * a6 - a7),  g[5] + (c58 + a3 + a4 + a5 + a6 + a8),
                      g[6] + (c58 - a3 - a4 + a5 + a6 - a8), g[7] + (c58 - a3 - a4 - a5 - a6 + a8),
                      g[8] + (c58 + a3 + a4 - a5 - a6 - a8)};
      store_pops<S, C>(dst, K.plane, cell, o, skey, 5);
    }
    static_cast<C*>(B.s_dst)[cell] = C(2) * fs + dfs;
  }
  return np;
}

}  // namespace vlb
