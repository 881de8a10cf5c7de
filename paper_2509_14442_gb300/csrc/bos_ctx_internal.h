// Context helpers shared by the C-ABI layer and the request server (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/bos.h"

namespace bos {

struct BatchJob;

// Bind a context to a device arena (nullptr: back to its own allocations) and clear its
// device error word on `stream`.
void ctx_bind_arena(bos_ctx* c, void* base, size_t bytes, cudaStream_t stream);

// Descriptor checks shared by every entry point that takes descriptors (the context calls
// and the allocation-free render).  BOS_OK, or BOS_ERR_INVALID_ARG with a message for
// bos_last_error() prefixed by `who`.  They touch no GPU.
bos_status_t check_grid_desc(const bos_grid_desc* d, const char* who);
bos_status_t check_geometry_desc(const bos_camera_desc* cam, const bos_wall_desc* wall, const bos_light_desc* light,
                                 const float* pattern_dev, const bos_integrator_desc* it, const char* who);

// Device bytes a render (adjoint != 0: render with checkpoints + backward) carves from an arena.
size_t request_bytes(const bos_grid_desc& g, const bos_camera_desc& cam, const bos_light_desc& light,
                     const bos_integrator_desc& it, int adjoint);

// Hooks of the request server's batched launches.  ctx_batchable: the context's scene can
// join a batched launch (FP32_COMP or BF16_COMP, Sharma RKN or quasi-linear, light modes 0
// and 1, ckpt_every <= 64).  ctx_batch_render: everything bos_render does before its launch
// (checks, checkpoint buffers, counters), and the job's share of a batched render in J, its
// warp-tile count and an upper bound of its ray-steps per tile.  ctx_batch_backward:
// accumulators zeroed on `st` and the job's share of a batched adjoint in J->adj.
// ctx_gradient: the stencil transpose and chain rule after the batched adjoint.
bool ctx_batchable(const bos_ctx* c);
bos_status_t ctx_batch_render(bos_ctx* c, float* I, float* disp, int save, cudaStream_t st, BatchJob* J, int* ntiles,
                              double* steps_per_tile);
bos_status_t ctx_batch_backward(bos_ctx* c, const float* dLdI, cudaStream_t st, BatchJob* J);
bos_status_t ctx_gradient(bos_ctx* c, float* dLdT, cudaStream_t st);
int ctx_num_sms(const bos_ctx* c);

}  // namespace bos
