// Host-side declarations of the kernel launchers (internal to the library).
#pragma once

#include "vlb_common.cuh"

namespace vlb {

// Constants of the particle kernels (Sec. 2.3 and the contact model).
struct ParticleConst {
  int np, nx, ny, per_x, per_y, ntx, nty;
  int outflow[4];    // open sides (no wall contact there)
  int any_ellipse;   // some particle is an ellipse (its band pass runs in a kernel of its own)
  int band_off;      // half-width of the band tables (cells)
  int band_stamp;    // level stamp written into the band tables
  double rho_ratio, gx, gy;
  double zeta, eps_p, eps_w, contact_scale;  // scale = |rho_r - 1| rho_f |g| pi
  double margin;                             // tile-range margin around each disk (cells)
  double inv_zeta;                           // 1 / zeta
};

// One case of a batched time step (vlb_step_batch): one launch of each kernel
// advances every case of a batch by a level.  The descriptors are written once
// per batch call; step k (0, 1, ...) of the call reads population buffer
// cur ^ (k & 1) and list buffer tl ^ (k & 1), fills list buffer
// 1 - (tl ^ (k & 1)), and stamps the band tables band_stamp_after(stamp, k + 1),
// which is what the k-th single-case step from the same state would do.
template <class C>
struct BatchLattice {
  LatticeConst<C> K;
  StepBuffers B[2];  // B[b]: the level in population buffer b, the next one into 1 - b
  TileLists TL[2];   // TL[l]: list buffer l; next_count = the counts of buffer 1 - l
  ParticleArrays P;
  int tile0;         // first tile of the case in the batched grid (tiles row by row)
  int cur, tl, stamp;
};
struct BatchParticles {
  ParticleConst c;
  ParticleArrays P;
  TileLists TL[2];
  unsigned* err;
  int tl, stamp;
};

// Storage of the populations of the FP32-arithmetic kernels.
enum : int { STORE_F32 = 0, STORE_F16 = 1, STORE_BF16 = 2 };

cudaError_t launch_lattice_f32(int mode, const LatticeConst<float>& K, const StepBuffers& B,
                               const ParticleArrays& P, const TileLists& TL, cudaStream_t st, int storage);
cudaError_t launch_lattice_f64(int mode, const LatticeConst<double>& K, const StepBuffers& B,
                               const ParticleArrays& P, const TileLists& TL, cudaStream_t st);

// Ownership dump of the current level (inspection of the integer raster).
cudaError_t launch_raster_dump_f32(const LatticeConst<float>& K, const ParticleArrays& P,
                                   const TileLists& TL, unsigned char* count, int* owner,
                                   unsigned char* flag, double* fsp, unsigned* err, cudaStream_t st);
cudaError_t launch_raster_dump_f64(const LatticeConst<double>& K, const ParticleArrays& P,
                                   const TileLists& TL, unsigned char* count, int* owner,
                                   unsigned char* flag, double* fsp, unsigned* err, cudaStream_t st);

// Particle step pieces.
cudaError_t launch_particle_range(const ParticleConst& c, const ParticleArrays& P, unsigned* err,
                                  cudaStream_t st);
cudaError_t launch_particle_band(const ParticleConst& c, const ParticleArrays& P, const TileLists& TL, unsigned* err,
                                 cudaStream_t st);

// Advance and band pass of every particle in one launch (list buffer TL, the
// stamp of ParticleConst).
cudaError_t launch_particle_step(const ParticleConst& c, const ParticleArrays& P, const TileLists& TL, unsigned* err,
                                 cudaStream_t st);
cudaError_t launch_particle_step_batch(const BatchParticles* cases, const int2* items, int nitems, int k,
                                       bool any_ellipse, cudaStream_t st);

// Batched step k: lattice tiles map to their case through tile_case.
// `held`: the held-temperature path (every case of the launch shares
// precision, storage and held).
cudaError_t launch_lattice_batch_f32(const BatchLattice<float>* cases, const int* tile_case, int ntiles, int k,
                                     int storage, bool held, cudaStream_t st);
cudaError_t launch_lattice_batch_f64(const BatchLattice<double>* cases, const int* tile_case, int ntiles, int k,
                                     bool held, cudaStream_t st);

// The persistent form of a batched step: one launch of a grid the size of the
// GPU's resident capacity per level.  Its CTAs take work chunks in order from
// a device counter: first the lattice tiles of level k -> k + 1 of every case
// (one tile each), then, with with_particles, the particle steps of the next
// level (one particle per warp), each after a bounded wait for the last tile
// of its own case.  Every chunk that a waiting warp depends on was taken
// earlier by a CTA that is running and never waits, so the waits end.  The
// last CTA to leave resets the counters and advances k.
struct BatchCtl {
  int next;    // next work chunk
  int exited;  // CTAs that have left this launch
  int k;       // level step of the call that this launch's tiles compute
  int pad;
};
template <class C>
struct PersistentBatch {
  const BatchLattice<C>* cases;  // the launch's cases
  const int* tile_case;          // case of every tile, tiles of one case together
  const BatchParticles* pcases;  // particle descriptors of the call's handles
  const int* case_handle;        // handle index of every case of the launch
  const int2* pitems;            // (case of the launch, particle) of its particles
  BatchCtl* ctl;
  int* done;                     // tiles finished per case in this launch
  int ntiles, npitems, ncases;
  int with_particles;            // 1: the particle steps of level k + 1 follow
  int stuck_case;                // test hook: this case's wait never ends (-1: none)
  long long wait_ns;             // limit of one wait (ns); past it ERR_TIMEOUT
};
// CTAs of one persistent launch (resident capacity of the variant on `device`).
int persistent_grid(int device, bool f64, int storage, bool held);
cudaError_t launch_lattice_persistent_f32(const PersistentBatch<float>& A, int grid, int storage, bool held,
                                          cudaStream_t st);
cudaError_t launch_lattice_persistent_f64(const PersistentBatch<double>& A, int grid, bool held, cudaStream_t st);
// The band pass of the batch's ellipses for step k, or for step *kdev when
// kdev is given (the level a persistent launch has just advanced to).
cudaError_t launch_particle_band_ellipse_batch(const BatchParticles* cases, const int2* items, int nitems, int k,
                                               const int* kdev, cudaStream_t st);

// FP64 audits: out[0] = sum f, out[1] = sum eps, out[2] = sum g (block partials
// in scratch[3 * nblocks], summed in block order).
cudaError_t launch_audit_f32(const LatticeConst<float>& K, const void* pop, const void* macro,
                             double* scratch, int nblocks, double* out, unsigned* err, cudaStream_t st,
                             int storage);
cudaError_t launch_audit_f64(const LatticeConst<double>& K, const void* pop, const void* macro,
                             double* scratch, int nblocks, double* out, unsigned* err, cudaStream_t st);

}  // namespace vlb
