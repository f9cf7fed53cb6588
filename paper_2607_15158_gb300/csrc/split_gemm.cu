// Placeholder: split-precision products are not available in this build.
#include "split_gemm.h"

namespace ctm {

struct SplitCtx {
  int dummy;
};

ctm_status split_create(SplitCtx** out, bool, int, int, cudaStream_t) {
  *out = nullptr;
  return CTM_EUNSUPPORTED;
}
void split_destroy(SplitCtx*) {}
ctm_status split_prepare_corners(SplitCtx*, void* const*, int, cudaStream_t, long*) {
  return CTM_EUNSUPPORTED;
}
ctm_status split_apply(SplitCtx*, const void*, bool, const void*, void*, int, int, cudaStream_t,
                       long*) {
  return CTM_EUNSUPPORTED;
}
const char* split_last_error(const SplitCtx*) { return "split precision not built"; }

}  // namespace ctm
