// Shared device helpers of libctm: element types, complex arithmetic,
// launch checking. Real data is double, complex data is double2 (re, im).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstring>

namespace ctm {

typedef double2 cplx;

// fp64 <-> fp32 conversions on the integer pipes, from the IEEE 754 binary64
// and binary32 layouts: the hardware conversions issue on this GPU's narrow
// fp64 pipe (about 1.6 operations per clock per SM), which bounds kernels that
// do little else than convert every element (operand slicing, split-K
// reduction). Round to nearest even; results below the fp32 normal range
// (|x| < 2^-126) become a signed zero; inf and NaN are kept.
__host__ __device__ __forceinline__ float f32_of(double x) {
#ifdef __CUDA_ARCH__
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
#else
  uint64_t b;
  memcpy(&b, &x, 8);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
#endif
  const unsigned sign = hi & 0x80000000u, ex = (hi >> 20) & 0x7ffu;
  const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);   // the 23 kept bits
  const unsigned rest = lo & 0x1fffffffu;                       // the 29 dropped bits
  const int e = (int)ex - 1023 + 127;
  unsigned bits;
  if (ex == 0x7ffu) {
    bits = 0x7f800000u | ((mant | rest) ? 0x400000u : 0u);
  } else if (e >= 255) {
    bits = 0x7f800000u;
  } else if (e <= 0) {
    bits = 0u;
  } else {
    bits = ((unsigned)e << 23) | mant;
    // a carry out of the mantissa correctly bumps the exponent (to inf at most)
    bits += (rest > 0x10000000u || (rest == 0x10000000u && (mant & 1u))) ? 1u : 0u;
  }
  bits |= sign;
#ifdef __CUDA_ARCH__
  return __uint_as_float(bits);
#else
  float f;
  memcpy(&f, &bits, 4);
  return f;
#endif
}

__host__ __device__ __forceinline__ double f64_of(float f) {
#ifdef __CUDA_ARCH__
  const unsigned u = __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, 4);
#endif
  const unsigned sign = u & 0x80000000u, ex = (u >> 23) & 0xffu, mant = u & 0x7fffffu;
  unsigned hi = sign;
  const unsigned lo = ex == 0u ? 0u : mant << 29;
  if (ex == 0xffu) hi |= 0x7ff00000u | (mant >> 3);
  else if (ex != 0u) hi |= ((ex + 1023u - 127u) << 20) | (mant >> 3);   // (zero: +-0)
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t b = ((uint64_t)hi << 32) | lo;
  double d;
  memcpy(&d, &b, 8);
  return d;
#endif
}

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
