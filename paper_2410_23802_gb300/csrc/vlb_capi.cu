// C ABI of the library (include/vlb.h): handle life cycle, device memory,
// the order of the kernels within a time step, and the copies to the host.
//
// One time step n -> n+1 on the handle's stream:
//   particle_step      F_c^n from the exchange sums and contact forces of level
//                      n (clearing the sums), forward Euler to X^{n+1}, U^{n+1};
//                      writes the raster records, appends each particle to
//                      the tile lists of X^{n+1} (list buffer b) and fills the
//                      band tables of level n+1
//   lattice (STEP)     fused pull / correction / thermal / collision pass that
//                      writes level n+1, adds the exchange sums of level n+1,
//                      lists the contact partners of level n+1, and clears list
//                      buffer 1 - b for the next step
// The first step is preceded by the initial state (lattice INIT mode).
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/vlb.h"
#include "vlb_common.cuh"
#include "vlb_internal.h"
#include "vlb_kernels.h"

using namespace vlb;

struct vlb_handle {
  vlb_params p{};
  std::string err;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;  // the device current at vlb_create, which holds every buffer
  cudaMemPool_t pool = nullptr;  // when set (served cases), buffers come from this stream-ordered pool
  int nx = 0, ny = 0, pitch = 0, ntx = 0, nty = 0;
  long long plane = 0;
  size_t ssize = 0;          // bytes per stored population
  size_t esize = 0;          // bytes per arithmetic value (S and macroscopic planes)
  int storage = 0;           // STORE_* of the FP32-arithmetic kernels
  void* pop[2] = {nullptr, nullptr};
  void* spl[2] = {nullptr, nullptr};
  void* macro = nullptr;
  int cur = 0;
  bool initialized = false;
  bool macros_valid = false;
  long long step = 0;
  // particles
  int np = 0, cap = 0;
  std::vector<double> hx, hy, hr, hT0, hk, hux, huy, hom;
  std::vector<double> hrb, hth;  // semi-minor axes (= hr for disks) and initial angles (reading R13)
  std::vector<int> hfix;  // particles held at their temperature
  ParticleArrays P{};
  TileLists TL[2] = {};
  int tl = 0;  // list buffer of the current level
  void* pbase = nullptr;
  size_t pbytes = 0;  // bytes of the particle block at pbase
  // device error word and its pinned host copy (refreshed in stream order)
  unsigned* err_host = nullptr;
  bool err_host_external = false;  // the served mode's arena owns it
  unsigned* err_dev = nullptr;
  double* audit_scratch = nullptr;
  double* audit_out = nullptr;
  int audit_blocks = 0;
  LatticeConst<float> K32{};
  LatticeConst<double> K64{};
  ParticleConst PC{};
  // profiling
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  int ev_used = 0, ev_cap = 0;
  double* pstage = nullptr;    // pinned staging of particle-state read-backs [12][cap]
  // queued particle-state copies (vlb_particle_state_async): a ring of two
  double* aring[2] = {nullptr, nullptr};
  cudaEvent_t aev[2] = {nullptr, nullptr};
  int an[2] = {0, 0};
  long long astep[2] = {0, 0};
  int ahead = 0, acount = 0;
  cudaEvent_t join = nullptr;  // orders this handle's stream with a batch call's
  // pinned staging of the descriptors of batch calls led by this handle, and
  // the event after their last copy
  unsigned char* bhost = nullptr;
  size_t bhost_cap = 0;
  cudaEvent_t bcopied = nullptr;
};

static thread_local std::string g_create_error;

// Device buffers of a handle: cudaMalloc, or for a handle made in a memory
// pool (the served mode's) stream-ordered allocation from it, whose frees do
// not synchronise the device.
static cudaError_t dev_alloc(vlb_handle* h, void** p, size_t bytes) {
  if (h->pool) return cudaMallocFromPoolAsync(p, bytes, h->pool, h->stream);
  return cudaMalloc(p, bytes);
}
static void dev_free(vlb_handle* h, void* p) {
  if (!p) return;
  if (h->pool) cudaFreeAsync(p, h->stream);
  else cudaFree(p);
}

static vlb_status fail(vlb_handle* h, vlb_status s, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return s;
}

static vlb_status cuda_fail(vlb_handle* h, cudaError_t e, const char* where) {
  return fail(h, VLB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                         \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
  } while (0)

// Queue a copy of the device error word into pinned host memory.
static cudaError_t pull_flags(vlb_handle* h) {
  return cudaMemcpyAsync(h->err_host, h->err_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
}

static vlb_status device_flags(vlb_handle* h) {
  const unsigned e = *(volatile unsigned*)h->err_host;
  if (e == 0) return VLB_OK;
  std::string m = "device reported:";
  if (e & ERR_TILE_OVERFLOW) m += " tile list overflow;";
  if (e & ERR_OWNER_OVERFLOW) m += " more than 4 owners in a cell;";
  if (e & ERR_NBR_OVERFLOW) m += " contact partner overflow;";
  if (e & ERR_BAND) m += " band table entry of another level;";
  if (e & ERR_MES_RANGE) m += " momentum-exchange sum out of fixed-point range;";
  if (e & ERR_OUT_OF_DOMAIN) m += " particle out of the domain;";
  if (e & ERR_TOO_FAST) m += " particle faster than 0.5 lu/step;";
  if (e & ERR_NAN) m += " NaN population;";
  if (e & ERR_TIMEOUT) m += " a device-side wait of the persistent batched step ran out;";
  if (e & ERR_TIMEOUT) return fail(h, VLB_ETIMEOUT, m);
  const bool unstable = e & (ERR_OUT_OF_DOMAIN | ERR_TOO_FAST | ERR_NAN);
  return fail(h, unstable ? VLB_EUNSTABLE : VLB_EOVERFLOW, m);
}

extern "C" {

size_t vlb_params_size(void) { return sizeof(vlb_params); }

vlb_status vlb_params_default(vlb_params* p) {
  if (!p) return VLB_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->abi_version = VLB_ABI_VERSION;
  p->nx = 64;
  p->ny = 64;
  p->precision = VLB_FP32;
  p->max_particles = 1024;
  p->tau_f = 0.8;
  p->lambda_q_flow = 1.0 / 12.0;
  p->s_e = 1.25;
  p->prandtl = 0.7;
  p->rho_ratio = 1.5;
  p->cv_ratio = 1.0;
  p->k_ratio_default = 1.0;
  p->T_ref = 1.0;
  p->T_fluid_init = 1.0;
  p->contact_range = 2.0;
  p->contact_eps_p = 0.01;
  p->contact_eps_w = 0.005;
  return VLB_OK;
}

const char* vlb_last_error(const vlb_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

template <class C>
static void fill_const(vlb_handle* h, LatticeConst<C>& K) {
  const vlb_params& p = h->p;
  K.nx = h->nx; K.ny = h->ny; K.pitch = h->pitch; K.ntx = h->ntx; K.nty = h->nty;
  K.plane = h->plane;
  K.per_x = p.periodic[0]; K.per_y = p.periodic[1];
  for (int w = 0; w < 4; ++w) K.outflow[w] = (p.outflow_mask >> w) & 1;
  for (int w = 0; w < 4; ++w) {
    K.wall_dirichlet[w] = p.thermal_wall[w] == VLB_WALL_DIRICHLET;
    K.wall_dT[w] = C(p.wall_T[w] - p.T_fluid_init);
  }
  K.np = h->np;
  // Eq. 5 with the rules of Sec. 3
  const double sp = 1.0 / p.tau_f;
  const double sq = 1.0 / (0.5 + p.lambda_q_flow / (p.tau_f - 0.5));
  K.s_e = C(p.s_e); K.s_eps = C(p.s_e); K.s_j = C(1); K.s_q = C(sq); K.s_p = C(sp);
  // Eqs. 11, 22 with rho_f = c_vf = 1; lambda_f = nu / Pr
  const double cvf = 1.0, cvs = p.cv_ratio;
  const double cref = 2.0 * cvf * cvs / (cvf + cvs);
  const double nu = (p.tau_f - 0.5) / 3.0;
  K.cv_f = C(cvf); K.cv_s = C(cvs); K.cref = C(cref); K.lam_f = C(nu / p.prandtl);
  K.rates_mode = C(p.thermal_rates_mode);
  K.bx = C(-p.beta * p.gravity[0]); K.by = C(-p.beta * p.gravity[1]);
  K.T_ref = C(p.T_ref); K.T_fluid = C(p.T_fluid_init);
  K.dT_ref = C(p.T_fluid_init - p.T_ref);
  const double tgf = 0.5 + 3.0 * (nu / p.prandtl) / cref;
  K.tau_gf = C(tgf);
  K.sj_f = C(1.0 / tgf);
  K.se_f = C(p.thermal_rates_mode == 0 ? 1.0 / (0.5 + 0.25 / (tgf - 0.5)) : 1.0);
  K.k3_cref = C(3.0 / cref);
  K.gk_f = C(-3.0 / (cref * tgf));
}

extern "C" {

static void free_all(vlb_handle* h) {
  for (int b = 0; b < 2; ++b) {
    dev_free(h, h->pop[b]);
    dev_free(h, h->spl[b]);
  }
  dev_free(h, h->macro);
  dev_free(h, h->pbase);
  for (int b = 0; b < 2; ++b) {
    dev_free(h, h->TL[b].count);
    dev_free(h, h->TL[b].ids);
  }
  dev_free(h, h->P.mes);
  dev_free(h, h->P.band);
  dev_free(h, h->audit_scratch);
  if (h->err_host && !h->err_host_external) cudaFreeHost(h->err_host);
  dev_free(h, h->err_dev);
  for (auto& e : h->ev) cudaEventDestroy(e);
  if (h->join) cudaEventDestroy(h->join);
  if (h->pstage) cudaFreeHost(h->pstage);
  for (int b = 0; b < 2; ++b) {
    if (h->aring[b]) cudaFreeHost(h->aring[b]);
    if (h->aev[b]) cudaEventDestroy(h->aev[b]);
  }
  if (h->bcopied) cudaEventDestroy(h->bcopied);
  if (h->bhost) cudaFreeHost(h->bhost);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

}  // extern "C"

// The first inconsistency of a parameter block, or nullptr.
static const char* params_error(const vlb_params& p) {
  if (p.abi_version != VLB_ABI_VERSION) return "abi_version mismatch";
  if (p.nx < 2 || p.ny < 2 || p.nx > (1 << 16) || p.ny > (1 << 16))
    return "nx, ny must be in [2, 65536]";
  if (!(p.tau_f > 0.5)) return "tau_f must exceed 1/2";
  if (!(p.lambda_q_flow > 0.0) || !(p.s_e > 0.0 && p.s_e < 2.0) || !(p.prandtl > 0.0))
    return "lambda_q_flow, s_e or prandtl out of range";
  if (!(p.rho_ratio > 0.0) || !(p.cv_ratio > 0.0) || !(p.k_ratio_default > 0.0))
    return "rho_ratio, cv_ratio, k_ratio_default must be positive";
  if (!(p.contact_range > 0.0) || !(p.contact_eps_p > 0.0) || !(p.contact_eps_w > 0.0))
    return "contact parameters must be positive";
  if (p.precision < VLB_FP64 || p.precision > VLB_BF16_STORE)
    return "precision must be a vlb_precision value";
  if (p.max_particles < 0 || p.max_particles > (1 << 24)) return "max_particles";
  if (p.thermal_rates_mode != 0 && p.thermal_rates_mode != 1)
    return "thermal_rates_mode must be 0 or 1";
  for (int k = 0; k < 2; ++k)
    if (p.periodic[k] != 0 && p.periodic[k] != 1) return "periodic must be 0/1";
  for (int w = 0; w < 4; ++w)
    if (p.thermal_wall[w] != 0 && p.thermal_wall[w] != 1) return "thermal_wall";
  if (p.outflow_mask & ~0xF) return "outflow_mask has bits beyond the four sides";
  for (int w = 0; w < 4; ++w)
    if (((p.outflow_mask >> w) & 1) && p.periodic[w / 2]) return "an open (outflow) side on a periodic axis";
  return nullptr;
}

// Sizes and layout every handle of parameters p uses.  Rows are padded to a
// 32-byte sector, not to a 128-byte line: the L2 fetches whole lines from
// DRAM, so the pad of a row padded to a line came in with its last cells
// (about 9 B per cell update over 256 channels of widths 64..256, measured),
// while with sector padding that line carries the next row's first cells,
// which the tile at the start of the row has just used.
struct Layout {
  int pitch, ntx, nty;
  long long plane;
  size_t ssize, esize;
};
static Layout layout_of(const vlb_params& p) {
  Layout L;
  L.esize = p.precision == VLB_FP64 ? 8 : 4;
  L.ssize = p.precision == VLB_FP64 ? 8 : (p.precision == VLB_FP32 ? 4 : 2);
  const int align = 32 / (int)L.ssize;
  L.pitch = (p.nx + align - 1) / align * align;
  L.plane = (long long)L.pitch * p.ny;
  L.ntx = (p.nx + TILE_X - 1) / TILE_X;
  L.nty = (p.ny + TILE_Y - 1) / TILE_Y;
  return L;
}
static size_t a256(size_t b) { return (b + 255) / 256 * 256; }
// Separation d of two centres along an axis of length L: on a periodic axis
// the nearest image, so that disks meeting across the boundary count as close.
static double min_image(double d, int L, int periodic) {
  if (!periodic) return d;
  if (d > 0.5 * L) return d - L;
  if (d < -0.5 * L) return d + L;
  return d;
}
// The particle block: 16 doubles, one int4, NBR_CAP + 2 ints, 8 doubles and
// one raster record per particle, every sub-array on a 256-byte boundary.
static size_t particle_block_bytes(size_t capn) {
  return 16 * a256(capn * sizeof(double)) + a256(capn * sizeof(int4)) + a256(capn * sizeof(int)) +
         a256(capn * NBR_CAP * sizeof(int)) + a256(capn * sizeof(int)) + a256(capn * 8 * sizeof(double)) +
         a256(capn * sizeof(RasterRec));
}
static int band_offset(double rmax) { return (int)std::ceil(rmax) + 2; }
constexpr int AUDIT_BLOCKS = 608;  // 4 x 152 SMs

extern "C" {

vlb_status vlb_device_bytes(const vlb_params* pp, int32_t n, const double* radius, uint64_t* bytes) {
  if (!pp || !bytes || n < 0 || (n > 0 && !radius)) return fail(nullptr, VLB_EINVAL, "vlb_device_bytes: arguments");
  if (const char* m = params_error(*pp)) return fail(nullptr, VLB_EINVAL, m);
  const vlb_params& p = *pp;
  const Layout L = layout_of(p);
  double rmax = 0.0;
  for (int k = 0; k < n; ++k) rmax = std::max(rmax, radius[k]);
  const size_t ntiles = (size_t)L.ntx * L.nty;
  const size_t bw = 2 * (size_t)band_offset(rmax) + 1;
  uint64_t b = 0;
  b += 2 * (18 * (uint64_t)L.plane * L.ssize + (uint64_t)L.plane * L.esize);  // populations, S
  b += 7 * (uint64_t)L.plane * L.esize;                                       // macroscopic planes
  b += 2 * ntiles * (sizeof(int) + TILE_CAP * sizeof(int));                   // tile lists
  b += particle_block_bytes((size_t)std::max(std::max(p.max_particles, n), 1));
  // exchange sums and band tables, sized for max_particles
  b += (uint64_t)std::max(p.max_particles, n) * (6 * sizeof(unsigned long long) + bw * bw * sizeof(int2));
  b += (3 * AUDIT_BLOCKS + 3) * sizeof(double) + sizeof(unsigned);
  *bytes = b;
  return VLB_OK;
}

vlb_status vlb_create(const vlb_params* pp, vlb_handle** out) { return vlb_create_in(pp, nullptr, out); }

}  // extern "C"

vlb_status vlb_create_in(const vlb_params* pp, const vlb_handle_alloc* alloc, vlb_handle** out) {
  if (!out) return fail(nullptr, VLB_EINVAL, "out is NULL");
  *out = nullptr;
  if (!pp) return fail(nullptr, VLB_EINVAL, "params is NULL");
  const vlb_params& p = *pp;
  if (const char* m = params_error(p)) return fail(nullptr, VLB_EINVAL, m);

  vlb_handle* h = new (std::nothrow) vlb_handle();
  if (!h) return fail(nullptr, VLB_ENOMEM, "host allocation");
  h->p = p;
  if (alloc) {
    h->pool = alloc->pool;
    h->err_host = alloc->err_host;
    h->err_host_external = alloc->err_host != nullptr;
  }
  h->nx = p.nx;
  h->ny = p.ny;
  const Layout L = layout_of(p);
  h->esize = L.esize;
  h->ssize = L.ssize;
  h->storage = p.precision == VLB_FP16_STORE ? STORE_F16 : (p.precision == VLB_BF16_STORE ? STORE_BF16 : STORE_F32);
  h->pitch = L.pitch;
  h->plane = L.plane;
  if (h->plane >= (1ll << 31)) {
    delete h;
    return fail(nullptr, VLB_EINVAL, "lattice too large for 32-bit cell offsets");
  }
  h->ntx = L.ntx;
  h->nty = L.nty;
  h->cap = p.max_particles;
  auto bail = [&](cudaError_t e, const char* where) {
    g_create_error = std::string(where) + ": " + cudaGetErrorString(e);
    free_all(h);
    delete h;
    return e == cudaErrorMemoryAllocation ? VLB_ENOMEM : VLB_ECUDA;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&h->device)) != cudaSuccess) return bail(e, "device");
  if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail(e, "stream");
  h->own_stream = true;
  const size_t popbytes = (size_t)18 * h->plane * h->ssize;
  for (int b = 0; b < 2; ++b) {
    if ((e = dev_alloc(h, &h->pop[b], popbytes)) != cudaSuccess) return bail(e, "populations");
    if ((e = dev_alloc(h, &h->spl[b], (size_t)h->plane * h->esize)) != cudaSuccess) return bail(e, "S plane");
    cudaMemsetAsync(h->spl[b], 0, (size_t)h->plane * h->esize, h->stream);
  }
  if ((e = dev_alloc(h, &h->macro, (size_t)7 * h->plane * h->esize)) != cudaSuccess) return bail(e, "macros");
  const long long ntiles = (long long)h->ntx * h->nty;
  for (int b = 0; b < 2; ++b) {
    if ((e = dev_alloc(h, reinterpret_cast<void**>(&h->TL[b].count), ntiles * sizeof(int))) != cudaSuccess) return bail(e, "tiles");
    if ((e = dev_alloc(h, reinterpret_cast<void**>(&h->TL[b].ids), ntiles * TILE_CAP * sizeof(int))) != cudaSuccess) return bail(e, "tiles");
    cudaMemsetAsync(h->TL[b].count, 0, ntiles * sizeof(int), h->stream);
  }
  // particle arrays (int4 and record loads need 16-byte alignment)
  const size_t capn = (size_t)std::max(h->cap, 1);
  const size_t pbytes = particle_block_bytes(capn);
  if ((e = dev_alloc(h, &h->pbase, pbytes)) != cudaSuccess) return bail(e, "particles");
  h->pbytes = pbytes;
  {
    char* b = static_cast<char*>(h->pbase);
    double** d[16] = {&h->P.x, &h->P.y, &h->P.theta, &h->P.ux, &h->P.uy, &h->P.om, &h->P.ux_prev,
                      &h->P.uy_prev, &h->P.om_prev, &h->P.fcx, &h->P.fcy, &h->P.tc, &h->P.r,
                      &h->P.lam_s, &h->P.T0, &h->P.rb};
    for (int k = 0; k < 16; ++k) { *d[k] = reinterpret_cast<double*>(b); b += a256(capn * sizeof(double)); }
    h->P.prange = reinterpret_cast<int4*>(b); b += a256(capn * sizeof(int4));
    h->P.nbr_count = reinterpret_cast<int*>(b); b += a256(capn * sizeof(int));
    h->P.nbr = reinterpret_cast<int*>(b); b += a256(capn * NBR_CAP * sizeof(int));
    h->P.fixed_T = reinterpret_cast<int*>(b); b += a256(capn * sizeof(int));
    h->P.pk = reinterpret_cast<double*>(b); b += a256(capn * 8 * sizeof(double));
    h->P.rec = reinterpret_cast<RasterRec*>(b);
  }
  cudaMemsetAsync(h->pbase, 0, pbytes, h->stream);
  h->audit_blocks = AUDIT_BLOCKS;
  if ((e = dev_alloc(h, reinterpret_cast<void**>(&h->audit_scratch), (3 * h->audit_blocks + 3) * sizeof(double))) != cudaSuccess)
    return bail(e, "audit");
  h->audit_out = h->audit_scratch + 3 * h->audit_blocks;
  if (!h->err_host_external && (e = cudaHostAlloc(&h->err_host, sizeof(unsigned), cudaHostAllocDefault)) != cudaSuccess)
    return bail(e, "error word");
  *h->err_host = 0;
  if ((e = dev_alloc(h, reinterpret_cast<void**>(&h->err_dev), sizeof(unsigned))) != cudaSuccess) return bail(e, "error word");
  cudaMemsetAsync(h->err_dev, 0, sizeof(unsigned), h->stream);
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(e, "create sync");
  *out = h;
  return VLB_OK;
}

extern "C" {

vlb_status vlb_set_fixed_temperature(vlb_handle* h, int32_t first, int32_t n, const int32_t* held) {
  if (!h) return VLB_EINVAL;
  if (h->initialized) return fail(h, VLB_ESTATE, "fixed temperatures must be set before the first step");
  if (first < 0 || n < 0 || first + n > h->np || (n > 0 && !held))
    return fail(h, VLB_EINVAL, "vlb_set_fixed_temperature: particle range outside the added particles");
  for (int k = 0; k < n; ++k) h->hfix[first + k] = held[k] == 2 ? 2 : (held[k] != 0 ? 1 : 0);
  return VLB_OK;
}

vlb_status vlb_set_stream(vlb_handle* h, void* s) {
  if (!h) return VLB_EINVAL;
  CK(h, cudaStreamSynchronize(h->stream));
  if (h->own_stream) cudaStreamDestroy(h->stream);
  h->own_stream = false;
  h->stream = static_cast<cudaStream_t>(s);
  return VLB_OK;
}

vlb_status vlb_add_particles(vlb_handle* h, int32_t n, const double* xy, const double* radius,
                             const double* T0, const double* k_ratio, const double* uv, const double* omega) {
  if (!h) return VLB_EINVAL;
  if (h->initialized) return fail(h, VLB_ESTATE, "particles must be added before the first step");
  if (n < 0 || (n > 0 && (!xy || !radius || !T0))) return fail(h, VLB_EINVAL, "bad particle arrays");
  if (h->np + n > h->cap) return fail(h, VLB_EOVERFLOW, "max_particles exceeded");
  const vlb_params& p = h->p;
  for (int k = 0; k < n; ++k) {
    const double X = xy[2 * k], Y = xy[2 * k + 1], R = radius[k];
    if (!(R >= 1.0) || !std::isfinite(X) || !std::isfinite(Y)) return fail(h, VLB_EINVAL, "radius < 1 or bad centre");
    const bool inx = p.periodic[0] ? (X - R - 1.0 >= 0.0 && X + R + 1.0 <= p.nx) : (X - R >= 0.0 && X + R <= p.nx);
    const bool iny = p.periodic[1] ? (Y - R - 1.0 >= 0.0 && Y + R + 1.0 <= p.ny) : (Y - R >= 0.0 && Y + R <= p.ny);
    if (!inx || !iny) return fail(h, VLB_EINVAL, "particle outside the domain or across a periodic boundary");
    if (k_ratio && !(k_ratio[k] > 0.0)) return fail(h, VLB_EINVAL, "k_ratio must be positive");
  }
  // overlap test against existing and new disks (minimum image on periodic axes)
  std::vector<double> X(h->hx), Y(h->hy), Rr(h->hr);
  for (int k = 0; k < n; ++k) { X.push_back(xy[2 * k]); Y.push_back(xy[2 * k + 1]); Rr.push_back(radius[k]); }
  std::vector<int> order(X.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return X[a] < X[b]; });
  double rmax = 0.0;
  for (double r : Rr) rmax = std::max(rmax, r);
  const size_t nold = h->hx.size();
  auto overlap = [&](int i, int j) {
    if ((size_t)i < nold && (size_t)j < nold) return false;
    const double dx = min_image(X[i] - X[j], p.nx, p.periodic[0]);
    const double dy = min_image(Y[i] - Y[j], p.ny, p.periodic[1]);
    return dx * dx + dy * dy < (Rr[i] + Rr[j]) * (Rr[i] + Rr[j]);
  };
  for (size_t a = 0; a < order.size(); ++a)
    for (size_t b = a + 1; b < order.size(); ++b) {
      const int i = order[a], j = order[b];
      if (X[j] - X[i] > 2.0 * rmax) break;
      if (overlap(i, j)) return fail(h, VLB_EINVAL, "particles overlap");
    }
  if (p.periodic[0]) {  // pairs that meet across the periodic x boundary
    for (size_t a = 0; a < order.size() && X[order[a]] < 2.0 * rmax; ++a)
      for (size_t b = order.size(); b-- > a + 1 && X[order[b]] > p.nx - 2.0 * rmax;)
        if (overlap(order[a], order[b])) return fail(h, VLB_EINVAL, "particles overlap");
  }
  for (int k = 0; k < n; ++k) {
    h->hx.push_back(xy[2 * k]);
    h->hy.push_back(xy[2 * k + 1]);
    h->hr.push_back(radius[k]);
    h->hrb.push_back(radius[k]);
    h->hth.push_back(0.0);
    h->hT0.push_back(T0[k]);
    h->hk.push_back(k_ratio ? k_ratio[k] : p.k_ratio_default);
    h->hfix.push_back(0);
    h->hux.push_back(uv ? uv[2 * k] : 0.0);
    h->huy.push_back(uv ? uv[2 * k + 1] : 0.0);
    h->hom.push_back(omega ? omega[k] : 0.0);
  }
  h->np += n;
  return VLB_OK;
}


vlb_status vlb_add_ellipses(vlb_handle* h, int32_t n, const double* xy, const double* semi_a, const double* semi_b,
                            const double* theta, const double* T0, const double* k_ratio, const double* uv,
                            const double* omega) {
  if (!h) return VLB_EINVAL;
  if (n < 0 || (n > 0 && (!semi_a || !semi_b || !theta))) return fail(h, VLB_EINVAL, "bad ellipse arrays");
  for (int k = 0; k < n; ++k)
    if (!(semi_b[k] >= 1.0 && semi_a[k] >= semi_b[k]) || !std::isfinite(theta[k]))
      return fail(h, VLB_EINVAL, "ellipse semi-axes must satisfy semi_a >= semi_b >= 1 and theta be finite");
  const int n0 = h->np;
  // the circumscribed disks go through the disks' checks (domain, overlap)
  const vlb_status st = vlb_add_particles(h, n, xy, semi_a, T0, k_ratio, uv, omega);
  if (st != VLB_OK) return st;
  for (int k = 0; k < n; ++k) {
    h->hrb[n0 + k] = semi_b[k];
    h->hth[n0 + k] = theta[k];
  }
  return VLB_OK;
}

// Lattice pass with list buffer `lists`; STEP and INIT also clear the other
// list buffer for the next particle step.
static vlb_status launch_lattice(vlb_handle* h, int mode, int src_buf, int dst_buf, int lists) {
  StepBuffers B;
  B.src = h->pop[src_buf];
  B.dst = h->pop[dst_buf];
  B.s_src = h->spl[src_buf];
  B.s_dst = h->spl[dst_buf];
  B.macro = h->macro;
  B.err = h->err_dev;
  TileLists TL = h->TL[lists];
  TL.next_count = mode == MODE_MACROS ? nullptr : h->TL[1 - lists].count;
  cudaError_t e = h->p.precision == VLB_FP64 ? launch_lattice_f64(mode, h->K64, B, h->P, TL, h->stream)
                                             : launch_lattice_f32(mode, h->K32, B, h->P, TL, h->stream, h->storage);
  if (e != cudaSuccess) return cuda_fail(h, e, "lattice kernel");
  return VLB_OK;
}

// Each band-kernel pass writes its entries with a new stamp (1 .. 2^29 - 1,
// cycling); the lattice and dump kernels accept only entries with the stamp of
// the tables they are given.
static void advance_band_stamp(vlb_handle* h, long long levels) {
  const int s = band_stamp_after(h->PC.band_stamp, levels);
  h->PC.band_stamp = s;
  h->K32.band_stamp = h->K64.band_stamp = s;
}
static void next_band_stamp(vlb_handle* h) { advance_band_stamp(h, 1); }

// Particles [first, first + count) of the host vectors to the device: state,
// properties and the per-particle constants of Eqs. 26, 29 (disk, rho_f = 1)
// and the wall contact factor.  The update starts from rest of the inside
// fluid terms (previous velocities = current ones).
static vlb_status upload_particles(vlb_handle* h, int first, int count) {
  const vlb_params& p = h->p;
  std::vector<double> lam(count), pk((size_t)8 * count, 0.0);
  const double lam_f = (p.tau_f - 0.5) / 3.0 / p.prandtl;
  const double gmag = std::hypot(p.gravity[0], p.gravity[1]);
  const double cscale = std::fabs(p.rho_ratio - 1.0) * gmag * M_PI;
  for (int k = 0; k < count; ++k) {
    lam[k] = h->hk[first + k] * lam_f;
    // an ellipse of semi-axes a >= b (a disk: a = b = R): area pi a b, polar
    // moment M (a^2 + b^2) / 4 (reading R13)
    const double a = h->hr[first + k], b = h->hrb[first + k], area = M_PI * a * b;
    const double M = p.rho_ratio * area, I = 0.25 * M * (a * a + b * b);
    double* q = pk.data() + 8 * (size_t)k;
    q[0] = 1.0 / M;
    q[1] = 1.0 / I;
    q[2] = area;                            // M_in = rho_f M / rho_s
    q[3] = 0.25 * area * (a * a + b * b);   // I_in
    q[4] = (p.rho_ratio - 1.0) * area;
    q[5] = cscale * a * a / p.contact_eps_w;
  }
  const size_t b = count * sizeof(double);
  auto up = [&](double* dst, const double* src) {
    return cudaMemcpyAsync(dst + first, src, b, cudaMemcpyHostToDevice, h->stream);
  };
  CK(h, up(h->P.x, h->hx.data() + first));
  CK(h, up(h->P.y, h->hy.data() + first));
  CK(h, up(h->P.r, h->hr.data() + first));
  CK(h, up(h->P.rb, h->hrb.data() + first));
  CK(h, up(h->P.theta, h->hth.data() + first));
  CK(h, up(h->P.T0, h->hT0.data() + first));
  CK(h, up(h->P.lam_s, lam.data()));
  CK(h, cudaMemcpyAsync(h->P.fixed_T + first, h->hfix.data() + first, count * sizeof(int), cudaMemcpyHostToDevice,
                        h->stream));
  CK(h, up(h->P.ux, h->hux.data() + first));
  CK(h, up(h->P.uy, h->huy.data() + first));
  CK(h, up(h->P.om, h->hom.data() + first));
  CK(h, up(h->P.ux_prev, h->hux.data() + first));
  CK(h, up(h->P.uy_prev, h->huy.data() + first));
  CK(h, up(h->P.om_prev, h->hom.data() + first));
  CK(h, cudaMemcpyAsync(h->P.pk + 8 * (size_t)first, pk.data(), pk.size() * sizeof(double), cudaMemcpyHostToDevice,
                        h->stream));
  CK(h, cudaStreamSynchronize(h->stream));  // the staging vectors end here
  return VLB_OK;
}

static vlb_status initialize(vlb_handle* h) {
  const vlb_params& p = h->p;
  const int n = h->np;
  const double margin = 0.5 * p.contact_range + 2.0;
  // band tables: a box of 2 band_off + 1 cells around each disk's centre cell
  // holds every cell with |d - R| < 0.75 (the centre lies in [xi, xi + 1))
  double rmax = 0.0;
  for (double r : h->hr) rmax = std::max(rmax, r);
  const int band_off = band_offset(rmax);
  if (h->cap > 0) {
    // exchange accumulators and band tables for max_particles disks (later
    // insertions append to them): zero before the first lattice pass
    const size_t capn = (size_t)h->cap;
    CK(h, dev_alloc(h, reinterpret_cast<void**>(&h->P.mes), capn * 6 * sizeof(unsigned long long)));
    CK(h, cudaMemsetAsync(h->P.mes, 0, capn * 6 * sizeof(unsigned long long), h->stream));
    const size_t bw = 2 * (size_t)band_off + 1;
    CK(h, dev_alloc(h, reinterpret_cast<void**>(&h->P.band), capn * bw * bw * sizeof(int2)));
    CK(h, cudaMemsetAsync(h->P.band, 0, capn * bw * bw * sizeof(int2), h->stream));
  }
  if (n > 0) {
    vlb_status st = upload_particles(h, 0, n);
    if (st != VLB_OK) return st;
  }
  fill_const(h, h->K32);
  fill_const(h, h->K64);

  ParticleConst& c = h->PC;
  c.np = n; c.nx = h->nx; c.ny = h->ny; c.per_x = p.periodic[0]; c.per_y = p.periodic[1];
  for (int w = 0; w < 4; ++w) c.outflow[w] = (p.outflow_mask >> w) & 1;
  c.ntx = h->ntx; c.nty = h->nty;
  c.band_off = band_off;
  h->K32.band_off = h->K64.band_off = band_off;
  int any_held = 0;
  for (int v : h->hfix) any_held |= v;
  h->K32.any_held = h->K64.any_held = any_held;
  c.any_ellipse = 0;
  for (size_t k = 0; k < h->hr.size(); ++k) c.any_ellipse |= h->hrb[k] != h->hr[k];
  c.rho_ratio = p.rho_ratio; c.gx = p.gravity[0]; c.gy = p.gravity[1];
  c.zeta = p.contact_range; c.eps_p = p.contact_eps_p; c.eps_w = p.contact_eps_w;
  c.contact_scale = std::fabs(p.rho_ratio - 1.0) * std::hypot(p.gravity[0], p.gravity[1]) * M_PI;
  c.margin = margin;
  c.inv_zeta = 1.0 / p.contact_range;
  h->K32.zeta = h->K64.zeta = p.contact_range;
  h->K32.contact_scale = h->K64.contact_scale = c.contact_scale;
  h->K32.eps_p = h->K64.eps_p = p.contact_eps_p;
  CK(h, launch_particle_range(c, h->P, h->err_dev, h->stream));
  h->tl = 0;
  next_band_stamp(h);
  CK(h, launch_particle_band(c, h->P, h->TL[0], h->err_dev, h->stream));
  h->cur = 0;
  vlb_status s = launch_lattice(h, MODE_INIT, 0, 0, 0);
  if (s != VLB_OK) return s;
  h->initialized = true;
  h->macros_valid = true;
  h->step = 0;
  return VLB_OK;
}

// One time step of h, queued on its stream.
static vlb_status step_once(vlb_handle* h) {
  vlb_status s;
  const int nl = 1 - h->tl;
  next_band_stamp(h);
  CK(h, launch_particle_step(h->PC, h->P, h->TL[nl], h->err_dev, h->stream));
  const bool rec = h->prof && h->ev_used + 2 <= h->ev_cap;
  if (rec) CK(h, cudaEventRecord(h->ev[h->ev_used], h->stream));
  if ((s = launch_lattice(h, MODE_STEP, h->cur, 1 - h->cur, nl)) != VLB_OK) return s;
  h->tl = nl;
  if (rec) {
    CK(h, cudaEventRecord(h->ev[h->ev_used + 1], h->stream));
    h->ev_used += 2;
  }
  h->cur = 1 - h->cur;
  ++h->step;
  h->macros_valid = false;
  return VLB_OK;
}

vlb_status vlb_insert_particles(vlb_handle* h, int32_t n, const double* xy, const double* radius, const double* T0,
                                const double* k_ratio, const double* uv, const double* omega) {
  if (!h) return VLB_EINVAL;
  if (!h->initialized) return vlb_add_particles(h, n, xy, radius, T0, k_ratio, uv, omega);
  if (n < 0 || (n > 0 && (!xy || !radius || !T0))) return fail(h, VLB_EINVAL, "bad particle arrays");
  if (n == 0) return VLB_OK;
  if (h->np + n > h->cap) return fail(h, VLB_EOVERFLOW, "max_particles exceeded");
  const vlb_params& p = h->p;
  const double rcap = double(h->PC.band_off - 2);  // the band tables hold disks up to this radius
  for (int k = 0; k < n; ++k) {
    const double X = xy[2 * k], Y = xy[2 * k + 1], R = radius[k];
    if (!(R >= 1.0) || !std::isfinite(X) || !std::isfinite(Y)) return fail(h, VLB_EINVAL, "radius < 1 or bad centre");
    if (R > rcap)
      return fail(h, VLB_EINVAL, "radius larger than the largest disk present at the first step (band-table size)");
    const bool inx = p.periodic[0] ? (X - R - 1.0 >= 0.0 && X + R + 1.0 <= p.nx) : (X - R >= 0.0 && X + R <= p.nx);
    const bool iny = p.periodic[1] ? (Y - R - 1.0 >= 0.0 && Y + R + 1.0 <= p.ny) : (Y - R >= 0.0 && Y + R <= p.ny);
    if (!inx || !iny) return fail(h, VLB_EINVAL, "particle outside the domain or across a periodic boundary");
    if (k_ratio && !(k_ratio[k] > 0.0)) return fail(h, VLB_EINVAL, "k_ratio must be positive");
  }
  // overlap against the disks where they are now, and among the new ones
  vlb_status st = vlb_synchronize(h);
  if (st != VLB_OK) return st;
  const int n0 = h->np;
  std::vector<double> X(n0), Y(n0);
  if (n0 > 0) {
    CK(h, cudaMemcpy(X.data(), h->P.x, n0 * sizeof(double), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(Y.data(), h->P.y, n0 * sizeof(double), cudaMemcpyDeviceToHost));
  }
  for (int k = 0; k < n; ++k) {
    const double x = xy[2 * k], y = xy[2 * k + 1], r = radius[k];
    for (int i = 0; i < n0; ++i) {
      const double dx = min_image(x - X[i], p.nx, p.periodic[0]), dy = min_image(y - Y[i], p.ny, p.periodic[1]);
      const double rr = r + h->hr[i];
      if (dx * dx + dy * dy < rr * rr) return fail(h, VLB_EINVAL, "particles overlap");
    }
    for (int j = 0; j < k; ++j) {
      const double dx = min_image(x - xy[2 * j], p.nx, p.periodic[0]);
      const double dy = min_image(y - xy[2 * j + 1], p.ny, p.periodic[1]);
      const double rr = r + radius[j];
      if (dx * dx + dy * dy < rr * rr) return fail(h, VLB_EINVAL, "particles overlap");
    }
  }
  for (int k = 0; k < n; ++k) {
    h->hx.push_back(xy[2 * k]);
    h->hy.push_back(xy[2 * k + 1]);
    h->hr.push_back(radius[k]);
    h->hrb.push_back(radius[k]);
    h->hth.push_back(0.0);
    h->hT0.push_back(T0[k]);
    h->hk.push_back(k_ratio ? k_ratio[k] : p.k_ratio_default);
    h->hfix.push_back(0);
    h->hux.push_back(uv ? uv[2 * k] : 0.0);
    h->huy.push_back(uv ? uv[2 * k + 1] : 0.0);
    h->hom.push_back(omega ? omega[k] : 0.0);
  }
  // the entries beyond the old count are still as created: zero angle, force,
  // partner count and exchange sums, band tables without a valid stamp
  if ((st = upload_particles(h, n0, n)) != VLB_OK) return st;
  h->np = n0 + n;
  h->PC.np = h->np;
  h->K32.np = h->K64.np = h->np;
  return VLB_OK;
}

vlb_status vlb_step(vlb_handle* h, int32_t nsteps) {
  if (!h) return VLB_EINVAL;
  if (nsteps < 0) return fail(h, VLB_EINVAL, "nsteps < 0");
  vlb_status s = device_flags(h);
  if (s != VLB_OK) return s;
  if (!h->initialized && (s = initialize(h)) != VLB_OK) return s;
  for (int k = 0; k < nsteps; ++k)
    if ((s = step_once(h)) != VLB_OK) return s;
  CK(h, pull_flags(h));
  return VLB_OK;
}

}  // extern "C"

// Descriptors of one batch call, packed into one host block and one device
// copy: the particle descriptors, the (case, particle) items, and per group
// of handles that share a lattice kernel (precision, storage, held path) the
// lattice descriptors and the tile-to-case table.
namespace {
struct BatchGroup {
  bool f64 = false, held = false;
  int storage = 0;
  std::vector<int> handles;  // indices into the call's handle array
  size_t desc_off = 0, table_off = 0;
  int ntiles = 0;
  // the persistent form: (case of the group, particle) items, the handle of
  // each case, the work counters and the tiles done per case
  std::vector<int2> pitems;
  size_t pitems_off = 0, chandle_off = 0, ctl_off = 0, done_off = 0;
  int grid = 0;
};

// Test hook of the persistent step's bounded waits (vlb_debug_batch_wait).
std::atomic<long long> g_wait_ns{1000000000ll};  // one second
std::atomic<int> g_stuck_handle{-1};

size_t align16(size_t n) { return (n + 15) & ~size_t(15); }

// The form of the batched step (vlb_set_batch_form): one CTA per tile and a
// particle kernel per level, or the persistent launch.  The build option
// VLB_BATCH_PERSISTENT sets the default (an autotuner candidate).
#ifndef VLB_BATCH_PERSISTENT
#define VLB_BATCH_PERSISTENT 0
#endif
std::atomic<int> g_batch_form{VLB_BATCH_PERSISTENT != 0 ? 1 : 0};
// steps of the persistent form per captured CUDA graph
constexpr int kGraphSteps = 64;

template <class C>
void fill_persistent(PersistentBatch<C>& A, unsigned char* dev, const BatchGroup& g, const BatchParticles* d_part,
                     bool with_particles, int stuck) {
  A.cases = reinterpret_cast<const BatchLattice<C>*>(dev + g.desc_off);
  A.tile_case = reinterpret_cast<const int*>(dev + g.table_off);
  A.pcases = d_part;
  A.case_handle = reinterpret_cast<const int*>(dev + g.chandle_off);
  A.pitems = reinterpret_cast<const int2*>(dev + g.pitems_off);
  A.ctl = reinterpret_cast<BatchCtl*>(dev + g.ctl_off);
  A.done = reinterpret_cast<int*>(dev + g.done_off);
  A.ntiles = g.ntiles;
  A.npitems = (int)g.pitems.size();
  A.ncases = (int)g.handles.size();
  A.with_particles = with_particles ? 1 : 0;
  A.stuck_case = stuck;
  A.wait_ns = g_wait_ns.load();
}

template <class C>
void fill_lattice_desc(vlb_handle* h, const LatticeConst<C>& K, int tile0, BatchLattice<C>& d) {
  d = BatchLattice<C>{};
  d.K = K;
  for (int b = 0; b < 2; ++b) {
    d.B[b].src = h->pop[b];
    d.B[b].dst = h->pop[1 - b];
    d.B[b].s_src = h->spl[b];
    d.B[b].s_dst = h->spl[1 - b];
    d.B[b].macro = h->macro;
    d.B[b].err = h->err_dev;
    d.TL[b] = h->TL[b];
    d.TL[b].next_count = h->TL[1 - b].count;
  }
  d.P = h->P;
  d.tile0 = tile0;
  d.cur = h->cur;
  d.tl = h->tl;
  d.stamp = h->PC.band_stamp;
}
}  // namespace

extern "C" {

}  // extern "C"

// The batched step; the descriptor staging block and its event are the
// caller's when given (stage != nullptr), else those of the leading handle.
static vlb_status step_batch_impl(vlb_handle* const* hs, int32_t n, int32_t nsteps, int32_t* failed,
                                  unsigned char** stage, size_t* stage_cap, cudaEvent_t* stage_copied) {
  if (failed) *failed = -1;
  if (n < 0 || (n > 0 && !hs)) return fail(nullptr, VLB_EINVAL, "vlb_step_batch: n < 0 or no handle array");
  if (nsteps < 0) return fail(nullptr, VLB_EINVAL, "vlb_step_batch: nsteps < 0");
  auto bad = [&](int i, vlb_status s) {
    if (failed) *failed = i;
    return s;
  };
#define BCK(i, call)                                                              \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) return bad((i), cuda_fail(hs[(i)], e_, #call));        \
  } while (0)
  for (int i = 0; i < n; ++i) {
    vlb_handle* h = hs[i];
    if (!h) return bad(i, fail(nullptr, VLB_EINVAL, "vlb_step_batch: NULL handle"));
    for (int j = 0; j < i; ++j)
      if (hs[j] == h) return bad(i, fail(h, VLB_EINVAL, "vlb_step_batch: a handle appears twice"));
    vlb_status s = device_flags(h);
    if (s != VLB_OK) return bad(i, s);
    if (!h->initialized && (s = initialize(h)) != VLB_OK) return bad(i, s);
    if (!h->join) {
      cudaError_t e = cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming);
      if (e != cudaSuccess) return bad(i, cuda_fail(h, e, "event"));
    }
  }
  if (n == 0 || nsteps == 0) {
    for (int i = 0; i < n; ++i) {
      cudaError_t e = pull_flags(hs[i]);
      if (e != cudaSuccess) return bad(i, cuda_fail(hs[i], e, "pull_flags"));
    }
    return VLB_OK;
  }

  // ---- descriptors -----------------------------------------------------------
  const int h0dev = hs[0]->device;
  const bool persistent = g_batch_form.load() == 1;
  std::vector<BatchGroup> groups;
  std::vector<int2> items;
  for (int i = 0; i < n; ++i) {
    vlb_handle* h = hs[i];
    const bool f64 = h->p.precision == VLB_FP64;
    const bool held = f64 ? h->K64.any_held : h->K32.any_held;
    const int storage = f64 ? 0 : h->storage;
    BatchGroup* g = nullptr;
    for (auto& q : groups)
      if (q.f64 == f64 && q.held == held && q.storage == storage) g = &q;
    if (!g) {
      groups.emplace_back();
      g = &groups.back();
      g->f64 = f64;
      g->held = held;
      g->storage = storage;
    }
    g->handles.push_back(i);
    for (int k = 0; k < h->np; ++k) items.push_back(make_int2(i, k));
  }
  size_t bytes = align16(sizeof(BatchParticles) * n);
  const size_t items_off = bytes;
  bytes = align16(bytes + sizeof(int2) * items.size());
  for (auto& g : groups) {
    long long nt = 0;
    for (int i : g.handles) nt += (long long)hs[i]->ntx * hs[i]->nty;
    if (nt > (1ll << 31) - 1) return bad(g.handles[0], fail(hs[g.handles[0]], VLB_EINVAL, "vlb_step_batch: too many tiles"));
    g.ntiles = (int)nt;
    g.desc_off = bytes;
    bytes = align16(bytes + (g.f64 ? sizeof(BatchLattice<double>) : sizeof(BatchLattice<float>)) * g.handles.size());
    g.table_off = bytes;
    bytes = align16(bytes + sizeof(int) * nt);
    if (persistent) {
      for (size_t c = 0; c < g.handles.size(); ++c)
        for (int k = 0; k < hs[g.handles[c]]->np; ++k) g.pitems.push_back(make_int2((int)c, k));
      g.pitems_off = bytes;
      bytes = align16(bytes + sizeof(int2) * g.pitems.size());
      g.chandle_off = bytes;
      bytes = align16(bytes + sizeof(int) * g.handles.size());
      g.ctl_off = bytes;
      bytes = align16(bytes + sizeof(BatchCtl));
      g.done_off = bytes;
      bytes = align16(bytes + sizeof(int) * g.handles.size());
      g.grid = persistent_grid(h0dev, g.f64, g.storage, g.held);
      if (g.grid <= 0) return bad(g.handles[0], fail(hs[g.handles[0]], VLB_ECUDA, "vlb_step_batch: occupancy query"));
    }
  }
  // the staging block of the previous call (led by hs[0], or the caller's)
  // is free once its copy ran
  vlb_handle* h0 = hs[0];
  if (!stage) {
    stage = &h0->bhost;
    stage_cap = &h0->bhost_cap;
    stage_copied = &h0->bcopied;
  }
  if (!*stage_copied) BCK(0, cudaEventCreateWithFlags(stage_copied, cudaEventDisableTiming));
  BCK(0, cudaEventSynchronize(*stage_copied));
  if (*stage_cap < bytes) {
    if (*stage) cudaFreeHost(*stage);
    *stage = nullptr;
    *stage_cap = 0;
    BCK(0, cudaMallocHost(reinterpret_cast<void**>(stage), bytes));
    *stage_cap = bytes;
  }
  unsigned char* hostp = *stage;
  std::memset(hostp, 0, bytes);
  auto* bp = reinterpret_cast<BatchParticles*>(hostp);
  for (int i = 0; i < n; ++i) {
    vlb_handle* h = hs[i];
    BatchParticles d{};
    d.c = h->PC;
    d.P = h->P;
    d.TL[0] = h->TL[0];
    d.TL[1] = h->TL[1];
    d.err = h->err_dev;
    d.tl = h->tl;
    d.stamp = h->PC.band_stamp;
    bp[i] = d;
  }
  if (!items.empty()) std::memcpy(hostp + items_off, items.data(), sizeof(int2) * items.size());
  for (auto& g : groups) {
    int* table = reinterpret_cast<int*>(hostp + g.table_off);
    int tile0 = 0;
    for (size_t c = 0; c < g.handles.size(); ++c) {
      vlb_handle* h = hs[g.handles[c]];
      if (g.f64) fill_lattice_desc(h, h->K64, tile0, reinterpret_cast<BatchLattice<double>*>(hostp + g.desc_off)[c]);
      else fill_lattice_desc(h, h->K32, tile0, reinterpret_cast<BatchLattice<float>*>(hostp + g.desc_off)[c]);
      const int nt = h->ntx * h->nty;
      for (int t = 0; t < nt; ++t) table[tile0 + t] = (int)c;
      tile0 += nt;
    }
    if (persistent) {
      if (!g.pitems.empty()) std::memcpy(hostp + g.pitems_off, g.pitems.data(), sizeof(int2) * g.pitems.size());
      int* ch = reinterpret_cast<int*>(hostp + g.chandle_off);
      for (size_t c = 0; c < g.handles.size(); ++c) ch[c] = g.handles[c];
    }
  }

  // ---- launches on the first handle's stream, joined with the others ---------
  cudaStream_t bs = h0->stream;
  for (int i = 1; i < n; ++i) {
    vlb_handle* h = hs[i];
    if (h->stream == bs) continue;
    BCK(i, cudaEventRecord(h->join, h->stream));
    BCK(0, cudaStreamWaitEvent(bs, h->join, 0));
  }
  unsigned char* dev = nullptr;
  BCK(0, cudaMallocAsync(reinterpret_cast<void**>(&dev), bytes, bs));
  cudaError_t e = cudaMemcpyAsync(dev, hostp, bytes, cudaMemcpyHostToDevice, bs);
  if (e == cudaSuccess) e = cudaEventRecord(*stage_copied, bs);
  const auto* d_part = reinterpret_cast<const BatchParticles*>(dev);
  const auto* d_items = reinterpret_cast<const int2*>(dev + items_off);
  const int nitems = (int)items.size();
  bool any_ellipse = false;
  for (int i = 0; i < n; ++i) any_ellipse |= hs[i]->PC.any_ellipse != 0;
  if (!persistent) {
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
      e = launch_particle_step_batch(d_part, d_items, nitems, k, any_ellipse, bs);
      for (auto& g : groups) {
        if (e != cudaSuccess) break;
        const int* table = reinterpret_cast<const int*>(dev + g.table_off);
        e = g.f64 ? launch_lattice_batch_f64(reinterpret_cast<const BatchLattice<double>*>(dev + g.desc_off), table,
                                             g.ntiles, k, g.held, bs)
                  : launch_lattice_batch_f32(reinterpret_cast<const BatchLattice<float>*>(dev + g.desc_off), table,
                                             g.ntiles, k, g.storage, g.held, bs);
      }
    }
  } else if (e == cudaSuccess) {
    // particle step of level 0; then nsteps - 1 persistent launches per group
    // of tiles of level s and particle steps of level s + 1 (the same launches
    // every level: captured once into a CUDA graph and replayed); then the
    // tiles of the last level
    auto persistent = [&](bool with_particles) -> cudaError_t {
      for (auto& g : groups) {
        int stuck = -1;
        for (size_t c = 0; c < g.handles.size(); ++c)
          if (g.handles[c] == g_stuck_handle.load()) stuck = (int)c;
        cudaError_t el;
        if (g.f64) {
          PersistentBatch<double> A{};
          fill_persistent(A, dev, g, d_part, with_particles, stuck);
          el = launch_lattice_persistent_f64(A, g.grid, g.held, bs);
        } else {
          PersistentBatch<float> A{};
          fill_persistent(A, dev, g, d_part, with_particles, stuck);
          el = launch_lattice_persistent_f32(A, g.grid, g.storage, g.held, bs);
        }
        if (el != cudaSuccess) return el;
      }
      if (with_particles && any_ellipse)
        return launch_particle_band_ellipse_batch(d_part, d_items, nitems, 0,
                                                  &reinterpret_cast<const BatchCtl*>(dev + groups[0].ctl_off)->k, bs);
      return cudaSuccess;
    };
    e = launch_particle_step_batch(d_part, d_items, nitems, 0, any_ellipse, bs);
    // the steps' launches are the same every step (the step index lives on
    // the device): up to kGraphSteps of them are captured into one CUDA graph,
    // replayed as often as it fits, and the rest launched plainly
    const int reps = nsteps - 1;
    const int gsteps = std::min(reps, kGraphSteps);
    bool captured = false;
    if (e == cudaSuccess && reps >= 2) {
      captured = cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (!captured) cudaGetLastError();  // a stream that cannot be captured (the legacy default stream)
    }
    int done_reps = 0;
    if (captured) {
      // the executable graph of the last call is kept (per host thread) and
      // updated with this call's launches when they have the same shape, which
      // costs far less than instantiating one per call; it lives as long as
      // the thread (one per thread that ever ran this form: destroying it at
      // thread exit could run after the CUDA runtime has been unloaded)
      thread_local cudaGraphExec_t cached = nullptr;
      cudaGraph_t graph = nullptr;
      cudaError_t eb = cudaSuccess;
      for (int r = 0; r < gsteps && eb == cudaSuccess; ++r) eb = persistent(true);
      e = cudaStreamEndCapture(bs, &graph);
      if (e == cudaSuccess) e = eb;
      if (e == cudaSuccess) {
        cudaGraphExecUpdateResultInfo info;
        if (!cached || cudaGraphExecUpdate(cached, graph, &info) != cudaSuccess) {
          cudaGetLastError();
          if (cached) cudaGraphExecDestroy(cached);  // (freed once its launches are done)
          cached = nullptr;
          e = cudaGraphInstantiate(&cached, graph, 0);
        }
      }
      for (; done_reps + gsteps <= reps && e == cudaSuccess; done_reps += gsteps) e = cudaGraphLaunch(cached, bs);
      if (graph) cudaGraphDestroy(graph);
    }
    for (; done_reps < reps && e == cudaSuccess; ++done_reps) e = persistent(true);
    if (e == cudaSuccess) e = persistent(false);
  }
  const cudaError_t ef = cudaFreeAsync(dev, bs);
  if (e != cudaSuccess) return bad(0, cuda_fail(h0, e, "batch kernels"));
  if (ef != cudaSuccess) return bad(0, cuda_fail(h0, ef, "batch descriptors"));
  BCK(0, cudaEventRecord(h0->join, bs));
  for (int i = 0; i < n; ++i) {
    vlb_handle* h = hs[i];
    if (h->stream != bs) {
      cudaError_t ew = cudaStreamWaitEvent(h->stream, h0->join, 0);
      if (ew != cudaSuccess) return bad(i, cuda_fail(h, ew, "stream join"));
    }
    // the host's view of the levels, as nsteps single steps would leave it
    h->cur ^= nsteps & 1;
    h->tl ^= nsteps & 1;
    advance_band_stamp(h, nsteps);
    h->step += nsteps;
    h->macros_valid = false;
    cudaError_t ep = pull_flags(h);
    if (ep != cudaSuccess) return bad(i, cuda_fail(h, ep, "pull_flags"));
  }
  return VLB_OK;
#undef BCK
}

vlb_status vlb_step_batch_staged(vlb_handle* const* hs, int32_t n, int32_t nsteps, int32_t* failed,
                                 unsigned char** stage, size_t* stage_cap, cudaEvent_t* stage_copied) {
  return step_batch_impl(hs, n, nsteps, failed, stage, stage_cap, stage_copied);
}

extern "C" {

vlb_status vlb_step_batch(vlb_handle* const* hs, int32_t n, int32_t nsteps, int32_t* failed) {
  return step_batch_impl(hs, n, nsteps, failed, nullptr, nullptr, nullptr);
}

vlb_status vlb_set_batch_form(int32_t form) {
  if (form != 0 && form != 1) return fail(nullptr, VLB_EINVAL, "vlb_set_batch_form: form must be 0 or 1");
  g_batch_form.store(form);
  return VLB_OK;
}

int32_t vlb_get_batch_form(void) { return g_batch_form.load(); }

vlb_status vlb_debug_batch_wait(int64_t wait_ns, int32_t stuck_handle) {
  if (stuck_handle < -1) return fail(nullptr, VLB_EINVAL, "vlb_debug_batch_wait: stuck_handle < -1");
  g_wait_ns = wait_ns > 0 ? (long long)wait_ns : 1000000000ll;
  g_stuck_handle = stuck_handle;
  return VLB_OK;
}

vlb_status vlb_synchronize(vlb_handle* h) {
  if (!h) return VLB_EINVAL;
  CK(h, pull_flags(h));
  CK(h, cudaStreamSynchronize(h->stream));
  return device_flags(h);
}

vlb_status vlb_get_step(vlb_handle* h, int64_t* n) {
  if (!h || !n) return VLB_EINVAL;
  *n = h->step;
  return VLB_OK;
}

static vlb_status ensure_ready(vlb_handle* h) {
  vlb_status s;
  if (!h->initialized && (s = initialize(h)) != VLB_OK) return s;
  if (!h->macros_valid) {
    // re-run the pre-collision part of the last step from the previous buffer
    if ((s = launch_lattice(h, MODE_MACROS, 1 - h->cur, h->cur, h->tl)) != VLB_OK) return s;
    h->macros_valid = true;
  }
  CK(h, pull_flags(h));
  CK(h, cudaStreamSynchronize(h->stream));
  return device_flags(h);
}

vlb_status vlb_get_fields(vlb_handle* h, uint32_t mask, double* rho, double* ux, double* uy, double* T,
                          double* fs) {
  if (!h) return VLB_EINVAL;
  double* outs[5] = {rho, ux, uy, T, fs};
  for (int k = 0; k < 5; ++k)
    if ((mask & (1u << k)) && !outs[k]) return fail(h, VLB_EINVAL, "NULL field array for a selected field");
  vlb_status s = ensure_ready(h);
  if (s != VLB_OK) return s;
  const size_t ncell = (size_t)h->nx * h->ny;
  // (a zero-filled vector: its pages are resident before the copy lands in
  // them, which measured faster than a fresh allocation on the Grace host)
  std::vector<char> tmp(ncell * h->esize);
  for (int k = 0; k < 5; ++k) {
    if (!(mask & (1u << k))) continue;
    const char* src = static_cast<const char*>(h->macro) + (size_t)k * h->plane * h->esize;
    CK(h, cudaMemcpy2D(tmp.data(), h->nx * h->esize, src, h->pitch * h->esize, h->nx * h->esize, h->ny,
                       cudaMemcpyDeviceToHost));
    if (h->esize == 8) std::memcpy(outs[k], tmp.data(), ncell * 8);
    else {
      const float* f = reinterpret_cast<const float*>(tmp.data());
      for (size_t c = 0; c < ncell; ++c) outs[k][c] = f[c];
    }
  }
  return VLB_OK;
}

}  // extern "C"

size_t vlb_value_bytes(const vlb_handle* h) { return h->esize; }

vlb_status vlb_check_flags(vlb_handle* h) { return h ? device_flags(h) : VLB_EINVAL; }

vlb_status vlb_readback_async(vlb_handle* h, void* fields, double* pstate, cudaEvent_t ev) {
  if (!h || !fields || !ev) return VLB_EINVAL;
  vlb_status s = device_flags(h);
  if (s != VLB_OK) return s;
  if (!h->initialized && (s = initialize(h)) != VLB_OK) return s;
  if (!h->macros_valid) {
    if ((s = launch_lattice(h, MODE_MACROS, 1 - h->cur, h->cur, h->tl)) != VLB_OK) return s;
    h->macros_valid = true;
  }
  const size_t row = (size_t)h->nx * h->esize;
  for (int k = 0; k < 5; ++k) {
    const char* src = static_cast<const char*>(h->macro) + (size_t)k * h->plane * h->esize;
    char* dst = static_cast<char*>(fields) + (size_t)k * h->ny * row;
    CK(h, cudaMemcpy2DAsync(dst, row, src, h->pitch * h->esize, row, h->ny, cudaMemcpyDeviceToHost, h->stream));
  }
  if (h->np > 0 && pstate) {
    const size_t cap = (size_t)std::max(h->cap, 1);
    CK(h, cudaMemcpy2DAsync(pstate, h->np * sizeof(double), h->P.x, a256(cap * sizeof(double)), h->np * sizeof(double),
                            12, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(h, pull_flags(h));
  CK(h, cudaEventRecord(ev, h->stream));
  return VLB_OK;
}

extern "C" {

vlb_status vlb_get_particle_count(vlb_handle* h, int32_t* n) {
  if (!h || !n) return VLB_EINVAL;
  *n = h->np;
  return VLB_OK;
}

}  // extern "C"

// The rows x, y, theta, ux, uy, om, (previous velocities), fcx, fcy, tc of a
// staged particle-state copy [12][n] into the caller's arrays.
static void unpack_particle_state(const double* st, int n, double* xy, double* theta, double* uv, double* omega,
                                  double* force, double* torque) {
  const double* row[12];
  for (int r = 0; r < 12; ++r) row[r] = st + (size_t)r * n;
  for (int k = 0; k < n; ++k) {
    if (xy) { xy[2 * k] = row[0][k]; xy[2 * k + 1] = row[1][k]; }
    if (theta) theta[k] = row[2][k];
    if (uv) { uv[2 * k] = row[3][k]; uv[2 * k + 1] = row[4][k]; }
    if (omega) omega[k] = row[5][k];
    if (force) { force[2 * k] = row[9][k]; force[2 * k + 1] = row[10][k]; }
    if (torque) torque[k] = row[11][k];
  }
}

extern "C" {

vlb_status vlb_get_particle_state(vlb_handle* h, int32_t n, double* xy, double* theta, double* uv,
                                  double* omega, double* force, double* torque) {
  if (!h) return VLB_EINVAL;
  if (n < 0 || n > h->np) return fail(h, VLB_EINVAL, "n exceeds the particle count");
  if (n == 0) return VLB_OK;
  if (!h->initialized) {
    // state before the first step is the uploaded one
    for (int k = 0; k < n; ++k) {
      if (xy) { xy[2 * k] = h->hx[k]; xy[2 * k + 1] = h->hy[k]; }
      if (theta) theta[k] = 0.0;
      if (uv) { uv[2 * k] = h->hux[k]; uv[2 * k + 1] = h->huy[k]; }
      if (omega) omega[k] = h->hom[k];
      if (force) { force[2 * k] = 0.0; force[2 * k + 1] = 0.0; }
      if (torque) torque[k] = 0.0;
    }
    return VLB_OK;
  }
  // the twelve state arrays x, y, theta, ux, uy, om, the three previous
  // velocities, fcx, fcy, tc follow one another in the particle block, one
  // 256-byte-aligned sub-array each: one strided copy takes n of each
  const size_t stride = a256((size_t)std::max(h->cap, 1) * sizeof(double));
  if (!h->pstage) CK(h, cudaMallocHost(reinterpret_cast<void**>(&h->pstage), 12 * (size_t)std::max(h->cap, 1) * sizeof(double)));
  CK(h, cudaMemcpy2DAsync(h->pstage, n * sizeof(double), h->P.x, stride, n * sizeof(double), 12,
                          cudaMemcpyDeviceToHost, h->stream));
  CK(h, pull_flags(h));
  CK(h, cudaStreamSynchronize(h->stream));
  unpack_particle_state(h->pstage, n, xy, theta, uv, omega, force, torque);
  return device_flags(h);
}

vlb_status vlb_particle_state_async(vlb_handle* h, int32_t n) {
  if (!h) return VLB_EINVAL;
  if (n < 0 || n > h->np) return fail(h, VLB_EINVAL, "n exceeds the particle count");
  if (h->acount == 2) return fail(h, VLB_ESTATE, "two particle-state copies are pending");
  vlb_status st = device_flags(h);
  if (st != VLB_OK) return st;
  if (!h->initialized && (st = initialize(h)) != VLB_OK) return st;
  const int b = (h->ahead + h->acount) % 2;
  const size_t cap = (size_t)std::max(h->cap, 1);
  if (!h->aring[b]) CK(h, cudaMallocHost(reinterpret_cast<void**>(&h->aring[b]), 12 * cap * sizeof(double)));
  if (!h->aev[b]) CK(h, cudaEventCreateWithFlags(&h->aev[b], cudaEventDisableTiming));
  if (n > 0)
    CK(h, cudaMemcpy2DAsync(h->aring[b], n * sizeof(double), h->P.x, a256(cap * sizeof(double)), n * sizeof(double),
                            12, cudaMemcpyDeviceToHost, h->stream));
  CK(h, pull_flags(h));
  CK(h, cudaEventRecord(h->aev[b], h->stream));
  h->an[b] = n;
  h->astep[b] = h->step;
  ++h->acount;
  return VLB_OK;
}

vlb_status vlb_particle_state_wait(vlb_handle* h, int32_t n, double* xy, double* theta, double* uv, double* omega,
                                   double* force, double* torque, int64_t* step) {
  if (!h) return VLB_EINVAL;
  if (h->acount == 0) return fail(h, VLB_ESTATE, "no particle-state copy is pending");
  const int b = h->ahead;
  if (n != h->an[b]) return fail(h, VLB_EINVAL, "n differs from the queued copy's");
  CK(h, cudaEventSynchronize(h->aev[b]));
  h->ahead = 1 - h->ahead;
  --h->acount;
  unpack_particle_state(h->aring[b], n, xy, theta, uv, omega, force, torque);
  if (step) *step = h->astep[b];
  return device_flags(h);
}

vlb_status vlb_get_audit(vlb_handle* h, double* total_mass, double* total_eps, double* total_g) {
  if (!h) return VLB_EINVAL;
  vlb_status s = ensure_ready(h);
  if (s != VLB_OK) return s;
  cudaError_t e = h->p.precision == VLB_FP64
                      ? launch_audit_f64(h->K64, h->pop[h->cur], h->macro, h->audit_scratch, h->audit_blocks,
                                         h->audit_out, h->err_dev, h->stream)
                      : launch_audit_f32(h->K32, h->pop[h->cur], h->macro, h->audit_scratch, h->audit_blocks,
                                         h->audit_out, h->err_dev, h->stream, h->storage);
  if (e != cudaSuccess) return cuda_fail(h, e, "audit");
  double o[3];
  CK(h, cudaMemcpyAsync(o, h->audit_out, sizeof(o), cudaMemcpyDeviceToHost, h->stream));
  CK(h, pull_flags(h));
  CK(h, cudaStreamSynchronize(h->stream));
  if (total_mass) *total_mass = o[0];
  if (total_eps) *total_eps = o[1];
  if (total_g) *total_g = o[2];
  return device_flags(h);
}

vlb_status vlb_get_solid_fraction(vlb_handle* h, uint8_t* count, int32_t* owner, uint8_t* flag, double* fsp) {
  if (!h) return VLB_EINVAL;
  vlb_status s = ensure_ready(h);
  if (s != VLB_OK) return s;
  const size_t ncell = (size_t)h->nx * h->ny;
  unsigned char *dc = nullptr, *df = nullptr;
  int* dow = nullptr;
  double* dfs = nullptr;
  cudaError_t e = cudaMalloc(&dc, ncell);
  if (e == cudaSuccess) e = cudaMalloc(&df, 4 * ncell);
  if (e == cudaSuccess) e = cudaMalloc(&dow, 4 * ncell * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&dfs, 4 * ncell * sizeof(double));
  if (e == cudaSuccess)
    e = h->p.precision == VLB_FP64
            ? launch_raster_dump_f64(h->K64, h->P, h->TL[h->tl], dc, dow, df, dfs, h->err_dev, h->stream)
            : launch_raster_dump_f32(h->K32, h->P, h->TL[h->tl], dc, dow, df, dfs, h->err_dev, h->stream);
  if (e == cudaSuccess) e = pull_flags(h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && count) e = cudaMemcpy(count, dc, ncell, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && flag) e = cudaMemcpy(flag, df, 4 * ncell, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && owner) e = cudaMemcpy(owner, dow, 4 * ncell * sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && fsp) e = cudaMemcpy(fsp, dfs, 4 * ncell * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(dc);
  cudaFree(df);
  cudaFree(dow);
  cudaFree(dfs);
  if (e != cudaSuccess) return cuda_fail(h, e, "solid fraction dump");
  return device_flags(h);
}

vlb_status vlb_get_contact_pairs(vlb_handle* h, int32_t capacity, int32_t* pairs, int32_t* npairs) {
  if (!h || !npairs || capacity < 0 || (capacity > 0 && !pairs)) return VLB_EINVAL;
  vlb_status s = ensure_ready(h);
  if (s != VLB_OK) return s;
  const int n = h->np;
  std::vector<int> cnt(n), nbr((size_t)n * NBR_CAP);
  if (n > 0) {
    CK(h, cudaMemcpy(cnt.data(), h->P.nbr_count, n * sizeof(int), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(nbr.data(), h->P.nbr, (size_t)n * NBR_CAP * sizeof(int), cudaMemcpyDeviceToHost));
  }
  std::vector<std::pair<int, int>> pr;
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < std::min(cnt[i], NBR_CAP); ++a) {
      const int j = nbr[(size_t)i * NBR_CAP + a];
      if (j > i) pr.emplace_back(i, j);
    }
  std::sort(pr.begin(), pr.end());
  const int total = (int)pr.size();
  for (int k = 0; k < std::min(total, capacity); ++k) {
    pairs[2 * k] = pr[k].first;
    pairs[2 * k + 1] = pr[k].second;
  }
  *npairs = total;
  return VLB_OK;
}

// ---- checkpoint and resume -------------------------------------------------
// The image is a header followed by the device buffers that carry the state
// of the current level, byte for byte: both population buffers and S planes
// (the field read-back re-runs the last step's pre-collision part from the
// previous one), the particle block (state, constants, records, ranges,
// contact lists), the exchange accumulators, the band tables and both tile
// list buffers.  Restoring them and the host counters continues the run
// exactly as if it had not stopped.
namespace {
struct StateHeader {
  char magic[8];
  uint32_t version, header_bytes;
  int32_t nx, ny, pitch, precision, storage, np, tile_y, band_off;
  int32_t cur, tl, band_stamp, reserved;
  int64_t step;
  uint64_t pop_bytes, s_bytes, part_bytes, mes_bytes, band_bytes, tl_count_bytes, tl_ids_bytes;
};
constexpr char kStateMagic[8] = {'V', 'L', 'B', 'S', 'T', 'A', 'T', 'E'};

StateHeader state_header(const vlb_handle* h) {
  StateHeader H{};
  std::memcpy(H.magic, kStateMagic, 8);
  H.version = 1;
  H.header_bytes = sizeof(StateHeader);
  H.nx = h->nx; H.ny = h->ny; H.pitch = h->pitch; H.precision = h->p.precision; H.storage = h->storage;
  H.np = h->np; H.tile_y = TILE_Y; H.band_off = h->PC.band_off;
  H.cur = h->cur; H.tl = h->tl; H.band_stamp = h->PC.band_stamp;
  H.step = h->step;
  H.pop_bytes = (uint64_t)18 * h->plane * h->ssize;
  H.s_bytes = (uint64_t)h->plane * h->esize;
  H.part_bytes = h->pbytes;
  H.mes_bytes = h->np > 0 ? (uint64_t)h->np * 6 * sizeof(unsigned long long) : 0;
  const uint64_t bw = 2 * (uint64_t)h->PC.band_off + 1;
  H.band_bytes = h->np > 0 ? (uint64_t)h->np * bw * bw * sizeof(int2) : 0;
  H.tl_count_bytes = (uint64_t)h->ntx * h->nty * sizeof(int);
  H.tl_ids_bytes = H.tl_count_bytes * TILE_CAP;
  return H;
}

uint64_t state_bytes(const StateHeader& H) {
  return sizeof(StateHeader) + 2 * (H.pop_bytes + H.s_bytes) + H.part_bytes + H.mes_bytes + H.band_bytes +
         2 * (H.tl_count_bytes + H.tl_ids_bytes);
}
}  // namespace

vlb_status vlb_state_size(vlb_handle* h, uint64_t* bytes) {
  if (!h || !bytes) return VLB_EINVAL;
  vlb_status s;
  if (!h->initialized && (s = initialize(h)) != VLB_OK) return s;
  *bytes = state_bytes(state_header(h));
  return VLB_OK;
}

vlb_status vlb_save_state(vlb_handle* h, void* buf, uint64_t bytes) {
  if (!h || !buf) return VLB_EINVAL;
  vlb_status s;
  if (!h->initialized && (s = initialize(h)) != VLB_OK) return s;
  const StateHeader H = state_header(h);
  if (bytes < state_bytes(H)) return fail(h, VLB_EINVAL, "vlb_save_state: buffer smaller than vlb_state_size");
  CK(h, cudaStreamSynchronize(h->stream));
  if ((s = device_flags(h)) != VLB_OK) return s;
  char* o = static_cast<char*>(buf);
  std::memcpy(o, &H, sizeof(H));
  o += sizeof(H);
  auto get = [&](const void* src, uint64_t n) -> cudaError_t {
    cudaError_t e = n ? cudaMemcpy(o, src, n, cudaMemcpyDeviceToHost) : cudaSuccess;
    o += n;
    return e;
  };
  for (int b = 0; b < 2; ++b) {
    CK(h, get(h->pop[b], H.pop_bytes));
    CK(h, get(h->spl[b], H.s_bytes));
  }
  CK(h, get(h->pbase, H.part_bytes));
  CK(h, get(h->P.mes, H.mes_bytes));
  CK(h, get(h->P.band, H.band_bytes));
  for (int b = 0; b < 2; ++b) {
    CK(h, get(h->TL[b].count, H.tl_count_bytes));
    CK(h, get(h->TL[b].ids, H.tl_ids_bytes));
  }
  return VLB_OK;
}

vlb_status vlb_load_state(vlb_handle* h, const void* buf, uint64_t bytes) {
  if (!h || !buf) return VLB_EINVAL;
  if (bytes < sizeof(StateHeader)) return fail(h, VLB_EINVAL, "vlb_load_state: buffer too small for a state image");
  StateHeader I;
  std::memcpy(&I, buf, sizeof(I));
  if (std::memcmp(I.magic, kStateMagic, 8) != 0 || I.version != 1 || I.header_bytes != sizeof(StateHeader))
    return fail(h, VLB_EINVAL, "vlb_load_state: not a state image of this library version");
  vlb_status s;
  if (!h->initialized && (s = initialize(h)) != VLB_OK) return s;
  const StateHeader H = state_header(h);
  if (I.nx != H.nx || I.ny != H.ny || I.pitch != H.pitch || I.precision != H.precision || I.storage != H.storage ||
      I.np != H.np || I.tile_y != H.tile_y || I.band_off != H.band_off || I.pop_bytes != H.pop_bytes ||
      I.s_bytes != H.s_bytes || I.part_bytes != H.part_bytes || I.mes_bytes != H.mes_bytes ||
      I.band_bytes != H.band_bytes || I.tl_count_bytes != H.tl_count_bytes || I.tl_ids_bytes != H.tl_ids_bytes)
    return fail(h, VLB_EINVAL, "vlb_load_state: the image was saved from a handle with other parameters or particles");
  if (bytes < state_bytes(I)) return fail(h, VLB_EINVAL, "vlb_load_state: truncated state image");
  if (I.cur < 0 || I.cur > 1 || I.tl < 0 || I.tl > 1) return fail(h, VLB_EINVAL, "vlb_load_state: corrupt header");
  CK(h, cudaStreamSynchronize(h->stream));
  const char* o = static_cast<const char*>(buf) + sizeof(StateHeader);
  auto put = [&](void* dst, uint64_t n) -> cudaError_t {
    cudaError_t e = n ? cudaMemcpy(dst, o, n, cudaMemcpyHostToDevice) : cudaSuccess;
    o += n;
    return e;
  };
  for (int b = 0; b < 2; ++b) {
    CK(h, put(h->pop[b], I.pop_bytes));
    CK(h, put(h->spl[b], I.s_bytes));
  }
  CK(h, put(h->pbase, I.part_bytes));
  CK(h, put(h->P.mes, I.mes_bytes));
  CK(h, put(h->P.band, I.band_bytes));
  for (int b = 0; b < 2; ++b) {
    CK(h, put(h->TL[b].count, I.tl_count_bytes));
    CK(h, put(h->TL[b].ids, I.tl_ids_bytes));
  }
  // the held-temperature flags and the ellipses' axes came with the particle block
  if (h->np > 0) {
    CK(h, cudaMemcpy(h->hfix.data(), h->P.fixed_T, h->np * sizeof(int), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(h->hrb.data(), h->P.rb, h->np * sizeof(double), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(h->hr.data(), h->P.r, h->np * sizeof(double), cudaMemcpyDeviceToHost));
  }
  int any_held = 0;
  for (int v : h->hfix) any_held |= v;
  h->K32.any_held = h->K64.any_held = any_held;
  h->PC.any_ellipse = 0;
  for (int k = 0; k < h->np; ++k) h->PC.any_ellipse |= h->hrb[k] != h->hr[k];
  h->cur = I.cur;
  h->tl = I.tl;
  h->step = I.step;
  h->PC.band_stamp = I.band_stamp;
  h->K32.band_stamp = h->K64.band_stamp = I.band_stamp;
  h->macros_valid = false;
  return VLB_OK;
}

vlb_status vlb_profile_begin(vlb_handle* h, int32_t max_steps) {
  if (!h || max_steps < 0) return VLB_EINVAL;
  CK(h, cudaStreamSynchronize(h->stream));
  const int need = 2 * max_steps;
  while ((int)h->ev.size() < need) {
    cudaEvent_t e;
    CK(h, cudaEventCreate(&e));
    h->ev.push_back(e);
  }
  h->ev_cap = need;
  h->ev_used = 0;
  h->prof = true;
  return VLB_OK;
}

vlb_status vlb_profile_end(vlb_handle* h, double* lattice_ms, int32_t* lattice_launches,
                           int32_t* launches_per_step) {
  if (!h) return VLB_EINVAL;
  CK(h, cudaStreamSynchronize(h->stream));
  double tot = 0.0;
  for (int k = 0; k + 1 < h->ev_used; k += 2) {
    float ms = 0.f;
    CK(h, cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1]));
    tot += ms;
  }
  if (lattice_ms) *lattice_ms = tot;
  if (lattice_launches) *lattice_launches = h->ev_used / 2;
  // particle_step (and the ellipses' band pass) and the lattice kernel
  if (launches_per_step) *launches_per_step = h->np > 0 ? (h->PC.any_ellipse ? 3 : 2) : 1;
  h->prof = false;
  h->ev_used = 0;
  return VLB_OK;
}

void vlb_destroy(vlb_handle* h) {
  if (!h) return;
  // a handle in a memory pool (served mode) frees in stream order: the
  // stream, which other handles share, is not waited for
  if (h->stream && !h->pool) cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
}

}  // extern "C"

// ---- helpers of the allocation-free entry point (vlb_noalloc.cu) ------------

int64_t vlb_cells_of(const vlb_handle* h) { return (int64_t)h->nx * h->ny; }

int vlb_device_of(const vlb_handle* h) { return h->device; }

vlb_status vlb_fail_einval(vlb_handle* h, const char* msg) { return fail(h, VLB_EINVAL, msg); }

vlb_status vlb_fail_cuda(vlb_handle* h, cudaError_t e, const char* where) { return cuda_fail(h, e, where); }

// The solid-fraction dump of the current level into caller-provided device
// buffers, then to the host arrays.  Allocates nothing; with
// require_initialized it refuses a handle whose initial state (which
// allocates) has not been built yet.
vlb_status vlb_solid_fraction_into(vlb_handle* h, unsigned char* d_count, int* d_owner, unsigned char* d_flag,
                                   double* d_fsp, uint8_t* count, int32_t* owner, uint8_t* flag, double* fsp,
                                   bool require_initialized) {
  if (require_initialized && !h->initialized)
    return fail(h, VLB_ESTATE, "the handle has no initial state yet: call vlb_step(h, 0) first");
  const size_t ncell = (size_t)h->nx * h->ny;
  cudaError_t e = h->p.precision == VLB_FP64
                      ? launch_raster_dump_f64(h->K64, h->P, h->TL[h->tl], d_count, d_owner, d_flag, d_fsp,
                                               h->err_dev, h->stream)
                      : launch_raster_dump_f32(h->K32, h->P, h->TL[h->tl], d_count, d_owner, d_flag, d_fsp,
                                               h->err_dev, h->stream);
  if (e == cudaSuccess) e = pull_flags(h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && count) e = cudaMemcpy(count, d_count, ncell, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && flag) e = cudaMemcpy(flag, d_flag, 4 * ncell, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && owner) e = cudaMemcpy(owner, d_owner, 4 * ncell * sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && fsp) e = cudaMemcpy(fsp, d_fsp, 4 * ncell * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "solid fraction dump (no allocation)");
  return device_flags(h);
}
