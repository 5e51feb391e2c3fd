// The single-case lattice kernels: the fused step (see vlb_lattice_body.cuh),
// the ownership dump and the FP64 audits.
#include "vlb_lattice_body.cuh"

namespace vlb {

template <class S, class C, int MODE, bool HOLD>
__global__ void __launch_bounds__(TILE_X * TILE_Y, sizeof(C) == 4 ? VLB_LATTICE_MIN_BLOCKS : 1)
lattice_kernel(const LatticeConst<C> K, const StepBuffers B, const ParticleArrays P, const TileLists TL) {
  __shared__ TileShared<C> sh;
  C f[9], g[9], s_old;
  pull_direct<S, C, MODE>(K, B, blockIdx.x, blockIdx.y, f, g, s_old);
  cell_body<S, C, MODE, HOLD>(K, B, P, TL, blockIdx.x, blockIdx.y, f, g, s_old, sh, K.band_stamp);
}

// Ownership of every cell at the current level, from the same raster code as
// the lattice kernel (inspection of the integer part of Sec. 2's f_s).
template <class C>
__global__ void __launch_bounds__(TILE_X * TILE_Y)
raster_dump_kernel(const LatticeConst<C> K, const ParticleArrays P, const TileLists TL, unsigned char* count,
                   int* owner, unsigned char* flag, double* fsp, unsigned* err) {
  __shared__ TileShared<C> sh;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int np = load_tile_particles<C>(K, P, TL, blockIdx.x, blockIdx.y, sh);
  const int x = blockIdx.x * TILE_X + tx, y = blockIdx.y * TILE_Y + ty;
  if (x >= K.nx || y >= K.ny) return;
  int nown, own[MAX_OWNERS], cls[MAX_OWNERS];
  C ofs[MAX_OWNERS];
  const PartTile<C>* s_p = sh.p;
  raster_cell<C>(tx, ty, x, y, np, s_p, P.band, K.band_off, K.band_stamp, nown, own, cls, ofs, err);
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
      const double v = double(stored_value<float, S>(pop[(long long)i * K.plane + cell]));
      const double w = double(stored_value<float, S>(pop[(long long)(9 + i) * K.plane + cell]));
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
  // kernels with the held-temperature path only where some particle is held
  if (mode == MODE_INIT) lattice_kernel<S, C, MODE_INIT, false><<<grid, block, 0, st>>>(K, B, P, TL);
  else if (mode == MODE_STEP && K.any_held) lattice_kernel<S, C, MODE_STEP, true><<<grid, block, 0, st>>>(K, B, P, TL);
  else if (mode == MODE_STEP) lattice_kernel<S, C, MODE_STEP, false><<<grid, block, 0, st>>>(K, B, P, TL);
  else if (K.any_held) lattice_kernel<S, C, MODE_MACROS, true><<<grid, block, 0, st>>>(K, B, P, TL);
  else lattice_kernel<S, C, MODE_MACROS, false><<<grid, block, 0, st>>>(K, B, P, TL);
  return cudaGetLastError();
}

cudaError_t launch_lattice_f32(int mode, const LatticeConst<float>& K, const StepBuffers& B,
                               const ParticleArrays& P, const TileLists& TL, cudaStream_t st, int storage) {
  if (storage == STORE_F16) return launch_mode<__half, float>(mode, K, B, P, TL, st);
  if (storage == STORE_BF16) return launch_mode<__nv_bfloat16, float>(mode, K, B, P, TL, st);
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
                             int nblocks, double* out, unsigned* err, cudaStream_t st, int storage) {
  if (storage == STORE_F16) return audit<__half, float>(K, pop, macro, scratch, nblocks, out, err, st);
  if (storage == STORE_BF16) return audit<__nv_bfloat16, float>(K, pop, macro, scratch, nblocks, out, err, st);
  return audit<float, float>(K, pop, macro, scratch, nblocks, out, err, st);
}
cudaError_t launch_audit_f64(const LatticeConst<double>& K, const void* pop, const void* macro,
                             double* scratch, int nblocks, double* out, unsigned* err, cudaStream_t st) {
  return audit<double, double>(K, pop, macro, scratch, nblocks, out, err, st);
}

}  // namespace vlb
