// Batched stepping of many cases (vlb_step_batch), in two forms: per step a
// particle kernel over the particles of every case and a lattice kernel of
// one CTA per tile of any case (form 0); or one persistent launch per step
// that takes the tiles and then the next level's particle steps from a
// device counter, each particle step after a bounded wait for its case's
// tiles (form 1).
#include <atomic>

#include "vlb_lattice_body.cuh"
#include "vlb_particle_body.cuh"

namespace vlb {

// Step k of a batch call (vlb_step_batch) over the tiles of many cases, one
// CTA per tile: the tile's case descriptor is copied to shared memory, then
// the single-case code (vlb_lattice_body.cuh) runs on it.
template <class S, class C, bool HOLD>
__global__ void __launch_bounds__(TILE_X * TILE_Y, sizeof(C) == 4 ? VLB_LATTICE_MIN_BLOCKS : 1)
lattice_batch_kernel(const BatchLattice<C>* __restrict__ cases, const int* __restrict__ tile_case, int k) {
  __shared__ TileShared<C> sh;
  __shared__ BatchLattice<C> d;
  static_assert(sizeof(BatchLattice<C>) % 4 == 0, "descriptor copied as words");
  {
    const int* src = reinterpret_cast<const int*>(cases + tile_case[blockIdx.x]);
    int* dst = reinterpret_cast<int*>(&d);
    for (int w = threadIdx.y * TILE_X + threadIdx.x; w < (int)(sizeof(d) / 4); w += TILE_X * TILE_Y)
      dst[w] = src[w];
  }
  __syncthreads();
  const int par = k & 1;
  const StepBuffers& B = d.B[d.cur ^ par];
  const TileLists& TL = d.TL[1 - (d.tl ^ par)];
  const int t = blockIdx.x - d.tile0;
  const int tile_y = t / d.K.ntx, tile_x = t - tile_y * d.K.ntx;
  C f[9], g[9], s_old;
  pull_direct<S, C, MODE_STEP>(d.K, B, tile_x, tile_y, f, g, s_old);
  cell_body<S, C, MODE_STEP, HOLD>(d.K, B, d.P, TL, tile_x, tile_y, f, g, s_old, sh,
                                   band_stamp_after(d.stamp, k + 1));
}

// The same over the particles of many cases, step k of a batch call.
__global__ void __launch_bounds__(32 * STEP_WARPS, 1)
    particle_step_batch_kernel(const BatchParticles* __restrict__ cases, const int2* __restrict__ items, int nitems,
                               int k) {
  __shared__ int s_queue[STEP_WARPS][BAND_QUEUE];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * STEP_WARPS;
  if (warp == 0 && lane < STEP_WARPS && i0 + lane < nitems) {
    const int2 it = items[i0 + lane];
    const BatchParticles& d = cases[it.x];
    advance_one(d.c, d.P, it.y, d.err);
  }
  __syncthreads();
  const int i = i0 + warp;
  if (i >= nitems) return;  // the whole warp
  const int2 it = items[i];
  const BatchParticles& d = cases[it.x];
  if (d.P.rb[it.y] != d.P.r[it.y]) return;
  const int nl = 1 - (d.tl ^ (k & 1));
  band_one<false>(d.c, d.P, d.TL[nl], d.err, it.y, band_stamp_after(d.stamp, k + 1), s_queue[warp], lane);
}
// The ellipses' band pass of step k (of step *kdev when kdev is given).
__global__ void __launch_bounds__(32 * BAND_WARPS)
    particle_band_ellipse_batch_kernel(const BatchParticles* __restrict__ cases, const int2* __restrict__ items,
                                       int nitems, int k, const int* __restrict__ kdev) {
  __shared__ int s_queue[BAND_WARPS][BAND_QUEUE];
  if (kdev) k = *kdev;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * BAND_WARPS + warp;
  if (i >= nitems) return;  // the whole warp
  const int2 it = items[i];
  const BatchParticles& d = cases[it.x];
  if (d.P.rb[it.y] == d.P.r[it.y]) return;
  const int nl = 1 - (d.tl ^ (k & 1));
  band_one<true>(d.c, d.P, d.TL[nl], d.err, it.y, band_stamp_after(d.stamp, k + 1), s_queue[warp], lane);
}

template <class S, class C>
static cudaError_t launch_batch(const BatchLattice<C>* cases, const int* tile_case, int ntiles, int k, bool held,
                                cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  const dim3 block(TILE_X, TILE_Y);
  if (held) lattice_batch_kernel<S, C, true><<<(unsigned)ntiles, block, 0, st>>>(cases, tile_case, k);
  else lattice_batch_kernel<S, C, false><<<(unsigned)ntiles, block, 0, st>>>(cases, tile_case, k);
  return cudaGetLastError();
}

cudaError_t launch_lattice_batch_f32(const BatchLattice<float>* cases, const int* tile_case, int ntiles, int k,
                                     int storage, bool held, cudaStream_t st) {
  if (storage == STORE_F16) return launch_batch<__half, float>(cases, tile_case, ntiles, k, held, st);
  if (storage == STORE_BF16) return launch_batch<__nv_bfloat16, float>(cases, tile_case, ntiles, k, held, st);
  return launch_batch<float, float>(cases, tile_case, ntiles, k, held, st);
}
cudaError_t launch_lattice_batch_f64(const BatchLattice<double>* cases, const int* tile_case, int ntiles, int k,
                                     bool held, cudaStream_t st) {
  return launch_batch<double, double>(cases, tile_case, ntiles, k, held, st);
}

cudaError_t launch_particle_step_batch(const BatchParticles* cases, const int2* items, int nitems, int k,
                                       bool any_ellipse, cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  particle_step_batch_kernel<<<(unsigned)((nitems + STEP_WARPS - 1) / STEP_WARPS), 32 * STEP_WARPS, 0, st>>>(
      cases, items, nitems, k);
  if (any_ellipse)
    particle_band_ellipse_batch_kernel<<<(unsigned)((nitems + BAND_WARPS - 1) / BAND_WARPS), 32 * BAND_WARPS, 0, st>>>(
        cases, items, nitems, k, nullptr);
  return cudaGetLastError();
}
cudaError_t launch_particle_band_ellipse_batch(const BatchParticles* cases, const int2* items, int nitems, int k,
                                               const int* kdev, cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  particle_band_ellipse_batch_kernel<<<(unsigned)((nitems + BAND_WARPS - 1) / BAND_WARPS), 32 * BAND_WARPS, 0, st>>>(
      cases, items, nitems, k, kdev);
  return cudaGetLastError();
}

// ---- the persistent form ------------------------------------------------------

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int load_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// One thread waits until *count >= target: true when it got there, false when
// limit_ns passed first (or, as a backstop should the timer stall, after an
// iteration count that takes longer than that limit at any sleep length).
__device__ bool wait_count(const int* count, int target, long long limit_ns) {
  if (load_acquire(count) >= target) return true;
  const unsigned long long t0 = global_ns();
  const long long max_iter = 4 * (limit_ns / 1024) + 4096;
  unsigned ns = 32;
  for (long long it = 0; it < max_iter; ++it) {
    __nanosleep(ns);
    if (load_acquire(count) >= target) return true;
    if ((long long)(global_ns() - t0) > limit_ns) return false;
    ns = ns < 1024u ? 2u * ns : 1024u;
  }
  return false;
}

// Particle item i of a persistent launch (one warp): the particle step of
// level kn, after the last tile of its case (whose exchange sums, contact
// partners and cleared list buffer it reads).  Inlined: as a call it cost
// the tile path more (spills around the call) than its own FP64 code does.
template <class C>
__device__ __forceinline__ void persistent_particle(const PersistentBatch<C>& A, int i, int kn, int* queue) {
  const int lane = threadIdx.x & 31;
  if (i >= A.npitems) return;
  const int2 it = A.pitems[i];
  const BatchParticles& pd = A.pcases[A.case_handle[it.x]];
  int ok = 1;
  if (lane == 0) {
    const LatticeConst<C>& K = A.cases[it.x].K;
    ok = wait_count(A.done + it.x, K.ntx * K.nty + (it.x == A.stuck_case ? 1 : 0), A.wait_ns);
    if (ok) advance_one(pd.c, pd.P, it.y, pd.err);
    else atomicOr(pd.err, ERR_TIMEOUT);
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok && pd.P.rb[it.y] == pd.P.r[it.y])
    band_one<false>(pd.c, pd.P, pd.TL[1 - (pd.tl ^ (kn & 1))], pd.err, it.y, band_stamp_after(pd.stamp, kn + 1), queue,
                    lane);
}

// Tiles per work chunk of the persistent launch: a CTA takes the next chunk
// from the counter (one atomic round trip, which its first warp waits for)
// only after its last one, so the trip is paid once per chunk.
#ifndef VLB_BATCH_CHUNK
#define VLB_BATCH_CHUNK 4
#endif
constexpr int BATCH_CHUNK = VLB_BATCH_CHUNK;

// The persistent batched step (see PersistentBatch).  Work items: tiles
// 0 .. ntiles - 1, then particle groups ntiles + m (particles 4m .. 4m + 3 of
// the launch, one per warp).  Chunk j of the counter is tiles
// BATCH_CHUNK j .. BATCH_CHUNK (j + 1) - 1 while j < tchunks, else the one
// particle group j - tchunks.  A CTA keeps its case's descriptor in shared
// memory while consecutive tiles share it.  The loop's state lives in shared
// memory.
template <class S, class C, bool HOLD>
__global__ void __launch_bounds__(TILE_X * TILE_Y, sizeof(C) == 4 ? VLB_LATTICE_MIN_BLOCKS : 1)
lattice_persistent_kernel(const __grid_constant__ PersistentBatch<C> A) {
  constexpr int NWARPS = TILE_X * TILE_Y / 32;
  union Shared {
    TileShared<C> tile;             // a tile's particles
    int queue[NWARPS][BAND_QUEUE];  // the band queues of a particle group
  };
  __shared__ Shared sh;
  __shared__ BatchLattice<C> d;
  __shared__ int s_item, s_end, s_case, s_k, s_pend, s_pend_case;
  static_assert(sizeof(BatchLattice<C>) % 4 == 0, "descriptor copied as words");
  const int tid = threadIdx.y * TILE_X + threadIdx.x;
  const int tchunks = (A.ntiles + BATCH_CHUNK - 1) / BATCH_CHUNK;
  const int nitems = A.ntiles + (A.with_particles ? (A.npitems + NWARPS - 1) / NWARPS : 0);
  // (thread 0) publish the finished tiles of one case: a fence, then one add
  auto publish = [&]() {
    if (s_pend > 0) {
      __threadfence();
      atomicAdd(A.done + s_pend_case, s_pend);
      s_pend = 0;
    }
  };
  auto take_chunk = [&]() {
    const int j = atomicAdd(&A.ctl->next, 1);
    s_item = j < tchunks ? j * BATCH_CHUNK : A.ntiles + (j - tchunks);
    s_end = j < tchunks ? min(A.ntiles, (j + 1) * BATCH_CHUNK) : s_item + 1;
  };
  if (tid == 0) {
    take_chunk();
    s_case = -1;
    s_k = A.ctl->k;
    s_pend = 0;
    s_pend_case = -1;
  }
  __syncthreads();
  int item = s_item, end = s_end;
  for (;;) {
    if (item >= nitems) break;
    if (item < A.ntiles) {
      const int c = A.tile_case[item];
      if (c != s_case) {  // (the barrier ending the previous item keeps d free)
        const int* src = reinterpret_cast<const int*>(A.cases + c);
        int* dst = reinterpret_cast<int*>(&d);
        for (int w = tid; w < (int)(sizeof(d) / 4); w += TILE_X * TILE_Y) dst[w] = src[w];
        __syncthreads();
        if (tid == 0) s_case = c;
      }
      const int par = s_k & 1;
      const StepBuffers& B = d.B[d.cur ^ par];
      const TileLists& TL = d.TL[1 - (d.tl ^ par)];
      const int lt = item - d.tile0;
      const int tile_y = lt / d.K.ntx, tile_x = lt - tile_y * d.K.ntx;
      C f[9], g[9], s_old;
      pull_direct<S, C, MODE_STEP>(d.K, B, tile_x, tile_y, f, g, s_old);
      cell_body<S, C, MODE_STEP, HOLD>(d.K, B, d.P, TL, tile_x, tile_y, f, g, s_old, sh.tile,
                                       band_stamp_after(d.stamp, s_k + 1));
      __syncthreads();  // every thread's stores and sums of this tile are issued; sh and d are free
      if (tid == 0 && A.with_particles && d.K.np > 0) {
        // counted now, published (fence + add) when the case changes or the
        // chunk ends, so that a chunk of one case pays one fence
        if (s_pend_case != s_case) {
          publish();
          s_pend_case = s_case;
        }
        ++s_pend;
      }
    } else {
      persistent_particle<C>(A, (item - A.ntiles) * NWARPS + (tid >> 5), s_k + 1, sh.queue[tid >> 5]);
      __syncthreads();  // the band queues are free
    }
    if (item + 1 < end) {  // the next tile of this chunk (every thread knows it)
      ++item;
      continue;
    }
    if (tid == 0) {
      publish();
      take_chunk();
    }
    __syncthreads();
    item = s_item;
    end = s_end;
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&A.ctl->exited, 1) == (int)gridDim.x - 1) {
      // the last CTA: every other one has left, so nothing reads these now
      for (int c = 0; c < A.ncases; ++c) A.done[c] = 0;
      A.ctl->next = 0;
      A.ctl->exited = 0;
      A.ctl->k = s_k + 1;
      __threadfence();
    }
  }
}

template <class S, class C, bool HOLD>
static int resident_ctas(int device) {
  // per device, filled by the first call (calls from several host threads
  // may race to fill it; they store the same value)
  static std::atomic<int> cached[64];
  if (device < 0 || device >= 64) return 0;
  const int known = cached[device].load(std::memory_order_relaxed);
  if (known > 0) return known;
  int nb = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, lattice_persistent_kernel<S, C, HOLD>, TILE_X * TILE_Y, 0) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return 0;
  cached[device].store(nb * nsm, std::memory_order_relaxed);
  return nb * nsm;
}

int persistent_grid(int device, bool f64, int storage, bool held) {
  if (f64) return held ? resident_ctas<double, double, true>(device) : resident_ctas<double, double, false>(device);
  if (storage == STORE_F16)
    return held ? resident_ctas<__half, float, true>(device) : resident_ctas<__half, float, false>(device);
  if (storage == STORE_BF16)
    return held ? resident_ctas<__nv_bfloat16, float, true>(device)
                : resident_ctas<__nv_bfloat16, float, false>(device);
  return held ? resident_ctas<float, float, true>(device) : resident_ctas<float, float, false>(device);
}

template <class S, class C>
static cudaError_t launch_persistent(const PersistentBatch<C>& A, int grid, bool held, cudaStream_t st) {
  const int nwarps = TILE_X * TILE_Y / 32;
  const int total = (A.ntiles + BATCH_CHUNK - 1) / BATCH_CHUNK +
                    (A.with_particles ? (A.npitems + nwarps - 1) / nwarps : 0);
  grid = grid < total ? grid : total;
  if (grid <= 0) return cudaSuccess;
  const dim3 block(TILE_X, TILE_Y);
  if (held) lattice_persistent_kernel<S, C, true><<<(unsigned)grid, block, 0, st>>>(A);
  else lattice_persistent_kernel<S, C, false><<<(unsigned)grid, block, 0, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_lattice_persistent_f32(const PersistentBatch<float>& A, int grid, int storage, bool held,
                                          cudaStream_t st) {
  if (storage == STORE_F16) return launch_persistent<__half, float>(A, grid, held, st);
  if (storage == STORE_BF16) return launch_persistent<__nv_bfloat16, float>(A, grid, held, st);
  return launch_persistent<float, float>(A, grid, held, st);
}
cudaError_t launch_lattice_persistent_f64(const PersistentBatch<double>& A, int grid, bool held, cudaStream_t st) {
  return launch_persistent<double, double>(A, grid, held, st);
}

}  // namespace vlb
