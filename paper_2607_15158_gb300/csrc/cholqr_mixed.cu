// Last CholeskyQR pass of the split-precision path (paper step 1: only
// span(X) enters the projectors). After two fp64 CholeskyQR passes the block
// Q has Q^H Q = I + E with |E| small; its Cholesky factor is I + F with
// F = tril(E) - diag(E) / 2 to first order, so Q <- Q (I + F)^-H ~ Q - Q F^H.
// The correction Q F^H is small, so its split-precision product adds only
// ~1e-7 |E| error: Q leaves orthonormal to ~|E|^2 + 1e-15.

#include "common.cuh"
#include "kernels.h"

namespace ctm {

namespace {

// B = F^H for F = tril(G - I, -1) + diag(G - I) / 2 (G: fp64 Gram, lower
// triangle valid).
template <typename T>
__global__ void orth_correction_kernel(int k, const T* G, T* B) {
  const long n = (long)k * k;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / k), c = (int)(idx % k);
    T v = zero_of(T());
    if (c > r) {
      v = conjv(G[(size_t)c * k + r]);
    } else if (c == r) {
      const double e = 0.5 * (realv(G[(size_t)r * k + r]) - 1.0);
      if constexpr (sizeof(T) == 8) v = e;
      else v = make_double2(e, 0.0);
    }
    B[idx] = v;
  }
}

template <typename T>
__global__ void sub_inplace_kernel(long n, T* z, const T* d) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x)
    z[i] = subv(z[i], d[i]);
}

unsigned blocks_for(long n) {
  long g = (n + 255) / 256;
  if (g > 152L * 8) g = 152L * 8;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace

cudaError_t orth_correction(bool cx, int k, const void* G, void* B, cudaStream_t s,
                            long* launches) {
  const unsigned g = blocks_for((long)k * k);
  if (cx) orth_correction_kernel<cplx><<<g, 256, 0, s>>>(k, (const cplx*)G, (cplx*)B);
  else orth_correction_kernel<double><<<g, 256, 0, s>>>(k, (const double*)G, (double*)B);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t sub_inplace(bool cx, long n, void* z, const void* d, cudaStream_t s,
                        long* launches) {
  const unsigned g = blocks_for(n);
  if (cx) sub_inplace_kernel<cplx><<<g, 256, 0, s>>>(n, (cplx*)z, (const cplx*)d);
  else sub_inplace_kernel<double><<<g, 256, 0, s>>>(n, (double*)z, (const double*)d);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace ctm
