// Shared device helpers of libctm: element types, complex arithmetic,
// launch checking. Real data is double, complex data is double2 (re, im).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace ctm {

typedef double2 cplx;

// ---------------------------------------------------------------- scalars
__host__ __device__ __forceinline__ double zero_of(double) { return 0.0; }
__host__ __device__ __forceinline__ cplx zero_of(cplx) { return make_double2(0.0, 0.0); }

__device__ __forceinline__ double conjv(double a) { return a; }
__device__ __forceinline__ cplx conjv(cplx a) { return make_double2(a.x, -a.y); }

__device__ __forceinline__ double addv(double a, double b) { return a + b; }
__device__ __forceinline__ cplx addv(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ double subv(double a, double b) { return a - b; }
__device__ __forceinline__ cplx subv(cplx a, cplx b) { return make_double2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ double mulv(double a, double b) { return a * b; }
__device__ __forceinline__ cplx mulv(cplx a, cplx b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double scalev(double a, double s) { return a * s; }
__device__ __forceinline__ cplx scalev(cplx a, double s) { return make_double2(a.x * s, a.y * s); }

// c += a * b
__device__ __forceinline__ void fmav(double& c, double a, double b) { c = fma(a, b, c); }
__device__ __forceinline__ void fmav(cplx& c, cplx a, cplx b) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
}
// c -= a * b
__device__ __forceinline__ void fnmav(double& c, double a, double b) { c = fma(-a, b, c); }
__device__ __forceinline__ void fnmav(cplx& c, cplx a, cplx b) {
  c.x = fma(-a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(-a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
}
// c += conj(a) * b
__device__ __forceinline__ void fmacv(double& c, double a, double b) { c = fma(a, b, c); }
__device__ __forceinline__ void fmacv(cplx& c, cplx a, cplx b) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
}
__device__ __forceinline__ double absq(double a) { return a * a; }
__device__ __forceinline__ double absq(cplx a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double realv(double a) { return a; }
__device__ __forceinline__ double realv(cplx a) { return a.x; }

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ cplx warp_sum(cplx v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}

// Device-side error flags written by bounded iterative kernels.
enum DevErr : int {
  DEV_OK = 0,
  DEV_CHOL_PIVOT = 1,     // non-positive or non-finite Cholesky pivot
  DEV_JACOBI_NOCONV = 2,  // Jacobi sweeps exhausted
  DEV_NONFINITE = 4,      // NaN / Inf met
  DEV_MBAR_TIMEOUT = 8,   // an mbarrier wait gave up
};

}  // namespace ctm

#define CTM_CUDA_OK(expr)                                   \
  do {                                                      \
    cudaError_t e__ = (expr);                               \
    if (e__ != cudaSuccess) return ::ctm::cuda_fail(e__, #expr, __FILE__, __LINE__); \
  } while (0)
