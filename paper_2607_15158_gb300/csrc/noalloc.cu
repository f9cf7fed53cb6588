// Singular values of one small matrix without any device allocation.
//
// Some callers of this library cannot let it allocate device memory: a host
// application that owns all device memory through its own allocator and
// forbids plug-ins from calling cudaMalloc, or a latency-sensitive loop in
// which cudaMalloc / cudaFree would stall on an implicit device-wide
// synchronisation. ctm_svdvals_noalloc serves them: it runs the same
// cooperative one-sided Jacobi kernel as the rest of the library, but its
// scratch (the kernel's work area, grid-barrier words and error word) lives
// in the fixed array g_noalloc_scratch below, reserved once in device memory
// for every GPU that loads the library and kept until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "common.cuh"
#include "ctm.h"
#include "kernels.h"

namespace {

// Largest matrices served: the Jacobi work area of either fits in the array
// below together with the 256-byte header that holds the error word.
constexpr int kMaxKComplex = 256;
constexpr int kMaxKReal = 362;
constexpr size_t kHeaderBytes = 256;
constexpr size_t kScratchBytes = (2u << 20) + 8192;  // 2 MiB + 8 KiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_dev_ptr[kMaxDevices] = {nullptr};
int g_num_sms[kMaxDevices] = {0};
thread_local char g_msg[256];

ctm_status nfail(ctm_status st, const char* m) {
  strncpy(g_msg, m, sizeof g_msg - 1);
  g_msg[sizeof g_msg - 1] = 0;
  return st;
}

}  // namespace

extern "C" ctm_status ctm_svdvals_noalloc(const void* A, int k, ctm_dtype dtype, double* s,
                                          void* stream) {
  if (!A || !s) return nfail(CTM_EINVAL, "A and s must be device pointers");
  if (dtype != CTM_F64 && dtype != CTM_C128) return nfail(CTM_EINVAL, "bad dtype");
  if (k < 1) return nfail(CTM_EINVAL, "k must be >= 1");
  const bool cx = dtype == CTM_C128;
  if (k > (cx ? kMaxKComplex : kMaxKReal) ||
      ctm::jacobi_coop_work_bytes(cx, k, 1) + kHeaderBytes > kScratchBytes)
    return nfail(CTM_EINVAL, "k exceeds the fixed scratch of ctm_svdvals_noalloc "
                             "(k <= 256 complex, k <= 362 real)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return nfail(CTM_ECUDA, "no usable current device");
  void* base = nullptr;
  int sms = 0;
  {
    // once per device, with that device current: the device address of the
    // scratch array (its name in host code is only a stand-in)
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_dev_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return nfail(CTM_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
      }
      int n = 0;
      if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return nfail(CTM_ECUDA, "cannot query the SM count");
      g_dev_ptr[dev] = p;
      g_num_sms[dev] = n;
    }
    base = g_dev_ptr[dev];
    sms = g_num_sms[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* b = static_cast<unsigned char*>(base);
  int* err = reinterpret_cast<int*>(b);          // error word, cleared per call
  void* jw = b + kHeaderBytes;                   // Jacobi work area
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess)
    return nfail(CTM_ECUDA, "clearing the error word failed");
  if (ctm::jacobi_svd_coop(cx, k, A, 0, s, nullptr, nullptr, false, jw, 1, 80, err, sms, st,
                           nullptr) != cudaSuccess) {
    cudaGetLastError();
    return nfail(CTM_ECUDA, "launch of the Jacobi kernel failed");
  }
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return nfail(CTM_ECUDA, "the Jacobi kernel failed on the device");
  if (h & ctm::DEV_MBAR_TIMEOUT) return nfail(CTM_ETIMEOUT, "grid barrier wait gave up");
  if (h & ctm::DEV_NONFINITE) return nfail(CTM_ENUMERIC, "non-finite singular value");
  if (h & ctm::DEV_JACOBI_NOCONV) return nfail(CTM_ENOCONV, "Jacobi sweep budget exhausted");
  return CTM_OK;
}

extern "C" const char* ctm_noalloc_last_error(void) { return g_msg; }
