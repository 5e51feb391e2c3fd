// Allocation-free variant of vlb_get_solid_fraction.
//
// vlb_get_solid_fraction takes four temporary device buffers from cudaMalloc
// on every call.  Some callers cannot allow that: code running while another
// allocator owns the device memory (a caching allocator or a memory pool that
// must see every allocation), code that must not synchronise the device the
// way cudaMalloc/cudaFree can, and callers with a fixed memory budget.  This
// file keeps the dump's scratch in one file-scope device array instead, so the
// entry point below allocates nothing.
//
// Limits and behaviour:
//   * at most VLB_NOALLOC_MAX_CELLS = 65536 lattice cells (e.g. 256 x 256);
//     larger lattices are rejected with VLB_EINVAL;
//   * the array (about 3.5 MB) is part of the library's device image, so every
//     GPU that loads the library holds it until the process exits;
//   * every call shares it and it keeps the last call's contents; the kernel
//     overwrites every element the call reads back, so nothing needs clearing;
//   * calls that overlap on the GPU (two handles on different streams, or
//     several host threads) race on the array and must be serialised by the
//     caller;
//   * the first call on each device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current); make that first call
//     before any stream capture;
//   * the address is the one of the device that holds the handle, so the call
//     requires that device to be current (VLB_EINVAL otherwise); after a
//     cudaDeviceReset the library's handles and this address are both void.
#include <cstdint>
#include <mutex>

#include "../../include/vlb.h"
#include "vlb_common.cuh"
#include "vlb_kernels.h"

namespace {

constexpr size_t kMaxCells = VLB_NOALLOC_MAX_CELLS;
// per cell: 4 fractions (8 B each), 4 owner ids (4 B), 4 class bytes, 1 count byte
constexpr size_t kFspBytes = kMaxCells * 4 * sizeof(double);
constexpr size_t kOwnerBytes = kMaxCells * 4 * sizeof(int);
constexpr size_t kFlagBytes = kMaxCells * 4;
constexpr size_t kCountBytes = kMaxCells;
constexpr size_t kScratchBytes = kFspBytes + kOwnerBytes + kFlagBytes + kCountBytes;

// The scratch itself.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_raster_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on device dev, which must be the current one
// (looked up once per device).
cudaError_t scratch_address(int dev, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaError_t e;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_raster_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return cudaSuccess;
}

}  // namespace

// Implemented in vlb_capi.cu: runs the dump kernel of the current level into
// the given device buffers and copies them to the caller's host arrays.
vlb_status vlb_solid_fraction_into(vlb_handle* h, unsigned char* d_count, int* d_owner, unsigned char* d_flag,
                                   double* d_fsp, uint8_t* count, int32_t* owner, uint8_t* flag, double* fsp,
                                   bool require_initialized);
int64_t vlb_cells_of(const vlb_handle* h);
int vlb_device_of(const vlb_handle* h);
vlb_status vlb_fail_einval(vlb_handle* h, const char* msg);
vlb_status vlb_fail_cuda(vlb_handle* h, cudaError_t e, const char* where);

extern "C" vlb_status vlb_get_solid_fraction_noalloc(vlb_handle* h, uint8_t* count, int32_t* owner,
                                                     uint8_t* flag, double* fsp) {
  if (!h) return VLB_EINVAL;
  if (vlb_cells_of(h) > (int64_t)kMaxCells)
    return vlb_fail_einval(h, "vlb_get_solid_fraction_noalloc: the lattice has more than "
                              "VLB_NOALLOC_MAX_CELLS (65536) cells");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return vlb_fail_cuda(h, e, "cudaGetDevice");
  if (dev != vlb_device_of(h))
    return vlb_fail_einval(h, "vlb_get_solid_fraction_noalloc: the current device is not the one that holds the "
                              "handle (make it current first)");
  unsigned char* base = nullptr;
  e = scratch_address(dev, &base);
  if (e != cudaSuccess) return vlb_fail_cuda(h, e, "cudaGetSymbolAddress");
  double* d_fsp = reinterpret_cast<double*>(base);
  int* d_owner = reinterpret_cast<int*>(base + kFspBytes);
  unsigned char* d_flag = base + kFspBytes + kOwnerBytes;
  unsigned char* d_count = base + kFspBytes + kOwnerBytes + kFlagBytes;
  return vlb_solid_fraction_into(h, d_count, d_owner, d_flag, d_fsp, count, owner, flag, fsp, true);
}
