// Shared definitions of the sm_103a kernels: lattice constants, the data
// layout in HBM, kernel argument blocks and device-side error bits.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vlb {

// ---------------------------------------------------------------------------
// D2Q9 velocity set of Eq. 2 (c = 1) and opposite directions.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ex(int i) {
  return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int ey(int i) {
  return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "opp");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "opp");

// D2Q9 weights: f^eq(1, 0) = M^-1 m^eq(1, 0) of Eqs. 4 and 6.
template <class C>
__host__ __device__ constexpr C wgt(int i) {
  return i == 0 ? C(4) / C(9) : (i <= 4 ? C(1) / C(9) : C(1) / C(36));
}

// Tiles of the lattice kernel: one CTA of 32 x TILE_Y threads per 32 x TILE_Y
// cells (one warp per row of the tile).  TILE_Y is a build-time choice.
#ifndef VLB_TILE_Y
#define VLB_TILE_Y 4
#endif
constexpr int TILE_X = 32;
constexpr int TILE_Y = VLB_TILE_Y;
static_assert(TILE_Y == 1 || TILE_Y == 2 || TILE_Y == 4 || TILE_Y == 8, "TILE_Y: 1, 2, 4 or 8 rows");
constexpr int TILE_CAP = 32;   // particles listed per tile
static_assert(TILE_CAP == 32, "a tile list is ranked by one warp");
constexpr int MAX_OWNERS = 4;  // particles owning one cell
constexpr int NBR_CAP = 16;    // contact partners per particle
constexpr int QBITS = 20;      // fixed-point grid of the integer cell tests

// Device error bits (mapped host word).
enum : unsigned {
  ERR_TILE_OVERFLOW = 1u,
  ERR_OWNER_OVERFLOW = 2u,
  ERR_NBR_OVERFLOW = 4u,
  ERR_MES_RANGE = 8u,  // an exchange row sum beyond the fixed-point range
  ERR_OUT_OF_DOMAIN = 16u,
  ERR_TOO_FAST = 32u,
  ERR_NAN = 64u,
  ERR_BAND = 128u,  // a band cell whose table entry is not of the current level
  ERR_TIMEOUT = 256u,  // a bounded device-side wait of a persistent launch ran out
};

// Band-table stamps run 1 .. 2^29 - 1 and then start again at 1 (0: none
// yet); the stamp k >= 1 levels after stamp s.
constexpr int BAND_STAMP_CYCLE = (1 << 29) - 1;
__host__ __device__ __forceinline__ int band_stamp_after(int s, long long k) {
  return 1 + (int)(((long long)s - 1 + k) % BAND_STAMP_CYCLE);
}

// Kernel modes of the lattice kernel.
enum : int { MODE_INIT = 0, MODE_STEP = 1, MODE_MACROS = 2 };

// ---------------------------------------------------------------------------
// Particle arrays (SoA, FP64) -- Sec. 2.3.
// ---------------------------------------------------------------------------
// What the FP32 lattice kernel needs of one particle, prepared once per step
// by the particle kernel so that the lattice kernel does no FP64 arithmetic.
// Centre: cell index (xi, yi) plus the fraction X - xi as an unevaluated FP32
// sum xfh + xfl and as a 2^-20 fixed-point offset qfx.
struct alignas(16) RasterRec {
  int xi, yi, qfx, qfy;
  long long rq2;               // (R rounded to 2^-20)^2, fixed point
  float xfh, xfl, yfh, yfl;
  float r, far2, near2;        // radius; quick-reject bounds on the centre distance^2
  float ux, uxl, uy, uyl, om;  // U as hi + lo, Omega
  float lam_s, T0;
};

struct ParticleArrays {
  double *x, *y, *theta, *ux, *uy, *om;
  double *ux_prev, *uy_prev, *om_prev;
  double *fcx, *fcy, *tc;  // F_c, T_c of the last update
  double *r, *lam_s, *T0;  // radius (an ellipse's semi-major axis), lambda_s, initial temperature
  double* rb;              // semi-minor axis (equal to r for a disk; reading R13)
  int4* prange;            // tile range (tx0, ty0, ntx, nty) at the current level
  unsigned long long* mes; // [n][3][2] F_MES,x + contact x, F_MES,y + contact y, T_MES as fixed point (mes_add)
  int* nbr_count;          // contact partners per particle
  int* nbr;                // [n][NBR_CAP], unordered (sorted where used)
  int* fixed_T;            // [n] held at T0: 1 over the covered part (reading R11), 2 whole cells (R11b)
  double* pk;              // [n][8] constants: 1/M, 1/I, M_in, I_in, body force factor, wall factor
  RasterRec* rec;          // [n] raster records of the current level
  int2* band;              // [n][bw][bw] band tables: (class | stamp << 2, area bits) of the cells of
                           // each disk's box, bw = 2 band_off + 1, centred on the record's cell
};

struct TileLists {
  int* count;       // [ntiles]
  int* ids;         // [ntiles][TILE_CAP], unordered
  int* next_count;  // counts of the other list buffer, cleared by the lattice kernel (may be null)
};

// Contact decision d_ij^2 < (R_i + R_j + zeta)^2 in FP64 without contraction,
// so that every device and the reference arithmetic take it identically.
__device__ __forceinline__ bool in_contact_range(double xi, double yi, double ri, double xj, double yj,
                                                 double rj, double zeta) {
  const double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj);
  const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
  const double thr = __dadd_rn(__dadd_rn(ri, rj), zeta);
  return d2 < __dmul_rn(thr, thr);
}

// Momentum-exchange sums (Eq. 28) are accumulated as integers, so that their
// totals do not depend on the order in which cells add them: word 0 (signed,
// two's complement) counts units of 2^-40, word 1 (unsigned) units of 2^-104
// with its carries moved into word 0.  The FP32 kernel fills word 0 only: a
// cell's term v becomes round(v 2^40), exact for |v| >= 2^-17 and within 2^-41
// below (over a disk's few hundred cells the rounding stays near 1e-11, far
// under the FP32 terms' own rounding); the FP64 kernel keeps 104 fraction bits.
// |v| < 2^21 is required (|f_s (rho u_s - j*)| <= 1 times an arm of at most
// 10^4 stays far below); larger values set ERR_MES_RANGE and are dropped.
constexpr double MES_SCALE_HI = 1099511627776.0;         // 2^40
constexpr double MES_SCALE_LO = 18446744073709551616.0;  // 2^64
__device__ __forceinline__ void mes_add(unsigned long long* w, float v, unsigned* err) {
  const float t = v * 1099511627776.0f;  // exact (power of two)
  if (!(fabsf(t) < 2.305843e18f)) { atomicOr(err, ERR_MES_RANGE); return; }  // 2^61
  const long long q = __float2ll_rn(t);
  if (q != 0) atomicAdd(w, (unsigned long long)q);
}
__device__ __forceinline__ void mes_add(unsigned long long* w, double v, unsigned* err) {
  const double t = v * MES_SCALE_HI;
  if (!(fabs(t) < 2.305843009213694e18)) { atomicOr(err, ERR_MES_RANGE); return; }
  const double fl = floor(t);
  const long long hi = (long long)fl;
  const unsigned long long lo = (unsigned long long)((t - fl) * MES_SCALE_LO);
  if (lo != 0ull) {
    const unsigned long long old = atomicAdd(w + 1, lo);
    if (old + lo < old) atomicAdd(w, 1ull);  // carry
  }
  if (hi != 0) atomicAdd(w, (unsigned long long)hi);
}
// The total of one accumulator pair as a double.
__host__ __device__ __forceinline__ double mes_value(unsigned long long hi, unsigned long long lo) {
  return (double)(long long)hi / MES_SCALE_HI + (double)lo / (MES_SCALE_HI * MES_SCALE_LO);
}

// Problem constants in the arithmetic type C of the lattice kernel.
template <class C>
struct LatticeConst {
  int nx, ny, pitch, ntx, nty;
  long long plane;         // elements per population plane
  int per_x, per_y;        // periodic axes
  int band_off;            // half-width of the band tables (cells)
  int band_stamp;          // level stamp the band tables must carry
  int any_held;            // some particle is held at its temperature (reading R11)
  int wall_dirichlet[4];   // x-, x+, y-, y+
  int outflow[4];          // open sides (zero normal gradient; reading R14)
  int np;
  double zeta;             // contact range
  double contact_scale;    // |rho_r - 1| rho_f |g| pi
  double eps_p;            // particle-particle stiffness parameter
  // flow rates (Eq. 5)
  C s_e, s_eps, s_j, s_q, s_p;
  // thermal (Eqs. 11, 18-22)
  C cv_f, cv_s, cref, lam_f, rates_mode;
  C bx, by, T_ref, T_fluid;  // buoyancy b = -rho_f beta g; T_f = initial fluid temperature
  C dT_ref;                  // T_f - T_ref
  C tau_gf, sj_f, se_f, gk_f;  // thermal rates of a fluid cell (Eqs. 18, 22, 23)
  C wall_dT[4];              // T_w - T_f per side
  C k3_cref;                 // 3 / c_ref
};

struct StepBuffers {
  void* src;     // populations at level n (18 planes of the storage type)
  void* dst;     // populations at level n+1
  void* s_src;   // S = 2 f_s + df_s/dt at level n (one plane, arithmetic type)
  void* s_dst;
  void* macro;   // rho, ux, uy, T, fs planes (arithmetic type); may be null
  unsigned* err;
};

}  // namespace vlb
