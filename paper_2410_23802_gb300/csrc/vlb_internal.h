// Library-internal calls shared by the C ABI and the served mode; not part
// of the public ABI (include/vlb.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/vlb.h"

// Where a served case's handle keeps its buffers: device memory from the
// server's stream-ordered pool (frees that do not synchronise the device)
// and the host copy of the device error word in the server's pinned arena
// (page-locked allocations synchronise the device too).
struct vlb_handle_alloc {
  cudaMemPool_t pool;
  unsigned* err_host;
};
vlb_status vlb_create_in(const vlb_params* p, const vlb_handle_alloc* a, vlb_handle** out);

// vlb_step_batch with the caller's pinned staging block for the descriptors
// (*stage of *stage_cap bytes, grown with cudaMallocHost when too small) and
// the event recorded after the block's copy (*stage_copied, created on first
// use); the block is reused once that event has completed.
vlb_status vlb_step_batch_staged(vlb_handle* const* hs, int32_t n, int32_t nsteps, int32_t* failed,
                                 unsigned char** stage, size_t* stage_cap, cudaEvent_t* stage_copied);

// Queue on the handle's stream the copy of the current level's fields
// (rho, ux, uy, T, f_s: five dense planes of nx * ny values of the handle's
// arithmetic type, into `fields`) and of its particle state ([12][n]
// doubles: x, y, theta, ux, uy, omega, the previous ux, uy, omega, F_c x, y,
// T_c, into `pstate`), both pinned host memory, then record ev.  Returns
// without waiting; the copies are valid once ev has completed.
vlb_status vlb_readback_async(vlb_handle* h, void* fields, double* pstate, cudaEvent_t ev);
// Bytes of one value of the handle's arithmetic type (4 or 8).
size_t vlb_value_bytes(const vlb_handle* h);

// The status the device error word's host copy holds (last pulled in stream
// order, e.g. by vlb_readback_async before its event), without waiting.
vlb_status vlb_check_flags(vlb_handle* h);
