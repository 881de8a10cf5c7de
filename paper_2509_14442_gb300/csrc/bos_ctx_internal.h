// Context helpers shared by the C-ABI layer and the request server (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "../../include/bos.h"

namespace bos {

// Bind a context to a device arena (nullptr: back to its own allocations) and clear its
// device error word on `stream`.
void ctx_bind_arena(bos_ctx* c, void* base, size_t bytes, cudaStream_t stream);

// Device bytes a render (adjoint != 0: render with checkpoints + backward) carves from an arena.
size_t request_bytes(const bos_grid_desc& g, const bos_camera_desc& cam, const bos_light_desc& light,
                     const bos_integrator_desc& it, int adjoint);

}  // namespace bos
