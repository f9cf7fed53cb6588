// Split-precision (bf16 slices, fp32 tensor-core accumulation, fp64
// reduction) corner x block products on the sm_103a tensor cores (tcgen05).
#pragma once

#include <cuda_runtime.h>

#include "ctm.h"

namespace ctm {

struct SplitCtx;

// State for N x N corners and N x k blocks of real (cx = false) or complex
// data; allocates the bf16 slice buffers of four corners.
ctm_status split_create(SplitCtx** out, bool cx, int N, int k, cudaStream_t s);
void split_destroy(SplitCtx* sc);

// Slice the four fp64 corners Q[0..3] (N x N) into bf16 operands, in both
// orientations (for op(Q) = Q and op(Q) = Q^H).
ctm_status split_prepare_corners(SplitCtx* sc, void* const* Q, int N, cudaStream_t s,
                                 long* launches);

// Zout = op(Q) Zin for one of the prepared corners (identified by pointer),
// Zin, Zout fp64 N x k row-major.
ctm_status split_apply(SplitCtx* sc, const void* Q, bool herm, const void* Zin, void* Zout,
                       int N, int k, cudaStream_t s, long* launches);

const char* split_last_error(const SplitCtx* sc);

}  // namespace ctm
