// Host <-> device staging of a step's inputs (kernels_pre.cu).
#pragma once

#include <cuda_runtime.h>

namespace dj {

// Writes target[k] (FP64, n entries; a device-accessible pointer, e.g. the
// device mapping of a page-locked host array) as FP32 to float index flat[k]
// of the per-node prescribed-displacement table (float4 per prescribed node:
// x, y, z targets, w = component mask).  flat[k] < 4 * (table rows) and
// flat[k] % 4 < 3 for every k (the host builds and checks the list); n <= 0
// launches nothing.  A non-finite target[k] is skipped (the entry keeps its
// previous value) and, when bad_flags is given (a device int, e.g. the
// mesh state's error flags), ERR_BAD_TARGET is or-ed into it.
cudaError_t launch_bc_targets(const double* target, const int* flat, int n, float4* table, cudaStream_t s,
                              int* bad_flags = nullptr);

}  // namespace dj
