// Host-side declarations of the kernel launchers (internal to the library).
#pragma once

#include "vlb_common.cuh"

namespace vlb {

// Constants of the particle kernels (Sec. 2.3 and the contact model).
struct ParticleConst {
  int np, nx, ny, per_x, per_y, ntx, nty;
  int band_off;      // half-width of the band tables (cells)
  int band_stamp;    // level stamp written into the band tables
  double rho_ratio, gx, gy;
  double zeta, eps_p, eps_w, contact_scale;  // scale = |rho_r - 1| rho_f |g| pi
  double margin;                             // tile-range margin around each disk (cells)
  double inv_zeta;                           // 1 / zeta
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
cudaError_t launch_particle_advance(const ParticleConst& c, const ParticleArrays& P, unsigned* err,
                                    cudaStream_t st);
cudaError_t launch_particle_band(const ParticleConst& c, const ParticleArrays& P, const TileLists& TL, unsigned* err,
                                 cudaStream_t st);

// FP64 audits: out[0] = sum f, out[1] = sum eps, out[2] = sum g (block partials
// in scratch[3 * nblocks], summed in block order).
cudaError_t launch_audit_f32(const LatticeConst<float>& K, const void* pop, const void* macro,
                             double* scratch, int nblocks, double* out, unsigned* err, cudaStream_t st,
                             int storage);
cudaError_t launch_audit_f64(const LatticeConst<double>& K, const void* pop, const void* macro,
                             double* scratch, int nblocks, double* out, unsigned* err, cudaStream_t st);

}  // namespace vlb
