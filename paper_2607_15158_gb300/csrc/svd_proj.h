// Standard truncated-SVD projectors (comparison baseline, paper Eq.
// svd_projectors_diag): dense SVD of M = H_L H_R and the scaled singular
// vectors that P_l = H_R V s^-1/2 and P_r^H = H_L^H U s^-1/2 need.
#pragma once

#include <cuda_runtime.h>

#include "ctm.h"

namespace ctm {

struct SvdCtx;

// State for N x N matrices (buffers allocated here; chi: most kept columns).
ctm_status svd_create(SvdCtx** out, bool cx, int N, int chi);
void svd_destroy(SvdCtx* sc);

// M (N x N row-major, overwritten) = U S V^H; Us = U_chi diag(conj ph) S^-1/2,
// Vs = V_chi diag(conj ph) S^-1/2 (N x chi row-major), ph the phase of the
// largest-modulus entry of each column of U (sign_fix), s_j^-1/2 := 0 for
// s_j <= cutoff s_1. A failed factorisation sets DEV_NONFINITE in err.
ctm_status svd_truncated(SvdCtx* sc, void* M, int chi, double cutoff, bool sign_fix, void* Us,
                         void* Vs, int* err, cudaStream_t s, long* launches);

const char* svd_last_error(const SvdCtx* sc);

}  // namespace ctm
