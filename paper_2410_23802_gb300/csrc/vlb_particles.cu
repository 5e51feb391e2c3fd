// The single-case particle kernels (see vlb_particle_body.cuh).
#include "vlb_particle_body.cuh"

namespace vlb {

__global__ void particle_range_kernel(const ParticleConst c, const ParticleArrays P, unsigned* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= c.np) return;
  const int4 rg = tile_range(c, P.x[p], P.y[p], P.r[p]);
  P.prange[p] = rg;
  write_record(P, p, P.x[p], P.y[p], P.r[p], P.rb[p], P.ux[p], P.uy[p], P.om[p], float(P.lam_s[p]), float(P.T0[p]));
}

// The band pass of every disk (ELL false) or of every ellipse (ELL true),
// one warp per particle; the particles of the other kind are left alone.
template <bool ELL>
__global__ void __launch_bounds__(32 * BAND_WARPS) particle_band_kernel(const ParticleConst c, const ParticleArrays P,
                                                                        const TileLists TL, unsigned* err) {
  __shared__ int s_queue[BAND_WARPS][BAND_QUEUE];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x * BAND_WARPS + warp;
  if (p >= c.np || ((P.rb[p] != P.r[p]) != ELL)) return;  // the whole warp
  band_one<ELL>(c, P, TL, err, p, c.band_stamp, s_queue[warp], lane);
}

// One particle step (advance, then lists and band table) in one launch: the
// two depend on the particle alone.  A CTA of STEP_WARPS warps takes
// STEP_WARPS particles: warp 0 advances them, one lane each (so the FP64
// instructions stay shared by many particles and the advance is spread over
// the SMs), then each warp runs the band pass of one of them; the barrier
// between makes the new records visible.  Ellipses get their band pass from
// particle_band_kernel<true> after this kernel.

__global__ void __launch_bounds__(32 * STEP_WARPS, 1) particle_step_kernel(const ParticleConst c, const ParticleArrays P,
                                                                        const TileLists TL, unsigned* err) {
  __shared__ int s_queue[STEP_WARPS][BAND_QUEUE];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p0 = blockIdx.x * STEP_WARPS;
  if (warp == 0 && lane < STEP_WARPS && p0 + lane < c.np) advance_one(c, P, p0 + lane, err);
  __syncthreads();
  const int p = p0 + warp;
  if (p >= c.np || P.rb[p] != P.r[p]) return;  // the whole warp
  band_one<false>(c, P, TL, err, p, c.band_stamp, s_queue[warp], lane);
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
  const unsigned grid = (unsigned)((c.np + BAND_WARPS - 1) / BAND_WARPS);
  particle_band_kernel<false><<<grid, 32 * BAND_WARPS, 0, st>>>(c, P, TL, err);
  if (c.any_ellipse) particle_band_kernel<true><<<grid, 32 * BAND_WARPS, 0, st>>>(c, P, TL, err);
  return cudaGetLastError();
}
cudaError_t launch_particle_step(const ParticleConst& c, const ParticleArrays& P, const TileLists& TL, unsigned* err,
                                 cudaStream_t st) {
  if (c.np == 0) return cudaSuccess;
  particle_step_kernel<<<(unsigned)((c.np + STEP_WARPS - 1) / STEP_WARPS), 32 * STEP_WARPS, 0, st>>>(c, P, TL, err);
  if (c.any_ellipse)
    particle_band_kernel<true><<<(unsigned)((c.np + BAND_WARPS - 1) / BAND_WARPS), 32 * BAND_WARPS, 0, st>>>(c, P, TL,
                                                                                                          err);
  return cudaGetLastError();
}
}  // namespace vlb
