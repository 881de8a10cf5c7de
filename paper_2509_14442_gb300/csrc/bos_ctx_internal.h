// Context helpers shared by the C-ABI layer and the request server (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/bos.h"

namespace bos {

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

}  // namespace bos
