// Split-precision (bf16 slices, fp32 tensor-core accumulation, fp64
// reduction) corner x block products on the sm_103a tensor cores (tcgen05).
#pragma once

#include <cuda_runtime.h>

#include "ctm.h"

namespace ctm {

struct SplitCtx;

// State for N x N corners and N x k blocks of real (cx = false) or complex
// data; err is the owner's device error flag (bounded waits report there).
// Buffers are allocated on first use.
// tf32: 3xTF32 slices (two tf32 slices, three products, kind::tf32) instead
// of bf16 x3 (three bf16 slices, six products, kind::f16).
ctm_status split_create(SplitCtx** out, bool cx, bool tf32, int N, int k, int* err,
                        cudaStream_t s);
void split_destroy(SplitCtx* sc);

// Slice the fp64 corners Q[i] (N x N) whose bit i is set in mask into bf16
// operands, in both orientations (for op(Q) = Q and op(Q) = Q^H).
ctm_status split_prepare_corners(SplitCtx* sc, void* const* Q, int N, unsigned mask,
                                 cudaStream_t s, long* launches);

// Zout = op(Q) Zin for one of the prepared corners (identified by pointer),
// Zin, Zout fp64 N x k row-major.
ctm_status split_apply(SplitCtx* sc, const void* Q, bool herm, const void* Zin, void* Zout,
                       int N, int k, cudaStream_t s, long* launches);

// General C = op(A) op(B) (M x N, inner K; ops as in GemmDesc) in split
// precision: both operands are sliced on the fly.
ctm_status split_gemm(SplitCtx* sc, int opA, const void* A, long lda, int opB, const void* B,
                      long ldb, int M, int N, int K, void* C, long ldc, cudaStream_t s,
                      long* launches);

// C = op(A) op(B) to fp64 accuracy on the bf16 tensor cores: every operand
// row / column is written as a 56-bit fixed-point number against the
// exponent of its largest entry and cut into eight 7-bit digits; the digit
// products of weight <= 7 are accumulated exactly in fp32 tensor memory and
// combined as unevaluated fp32 pairs (about 2^-48 relative to the products
// of the row and column maxima, the bound of an fp64 product). Ops and
// layouts as in split_gemm.
ctm_status oz_gemm(SplitCtx* sc, int opA, const void* A, long lda, int opB, const void* B,
                   long ldb, int M, int N, int K, void* C, long ldc, cudaStream_t s,
                   long* launches);

// Profiling of the tensor-core kernel: on = 1 / 0 starts / stops recording
// CUDA events around every launch (and clears the totals); on = -1 reads the
// accumulated device time, launches, tensor-pipe flops and operand bytes.
ctm_status split_profile(SplitCtx* sc, int on, double* ms, long* launches, double* flops,
                         double* bytes);

// Largest number of split-K partials a product with inner dimension N (2N
// for complex) uses: each partial covers a bounded number of K blocks.
size_t split_partial_splits(size_t N, bool cx);

const char* split_last_error(const SplitCtx* sc);

}  // namespace ctm
