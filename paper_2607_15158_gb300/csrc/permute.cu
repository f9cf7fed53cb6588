// Axis permutation of dense row-major tensors (the reshapes between the
// pairwise contractions of the enlarged corners and of the absorption).
// HBM-bound: after fusing axes that stay adjacent, either the fastest axis is
// kept (contiguous row copies) or a 32 x 32 shared-memory tile transposes the
// input's fastest axis with the output's fastest axis, so that both the loads
// and the stores are coalesced.
#include "common.cuh"
#include "kernels.h"

namespace ctm {

namespace {

struct PermArgs {
  int rank;
  int a;          // output axis carrying the input's stride-1 axis (tile case)
  long od[8];     // output dims
  long os[8];     // input stride of each output axis
  long ostr[8];   // output stride of each output axis
  long total;
};

template <typename T, bool CONJ, typename I>
__global__ void __launch_bounds__(256) perm_rows(const T* __restrict__ in,
                                                 T* __restrict__ out,
                                                 PermArgs p) {
  // one warp per output row of length L = od[rank-1] (input stride 1)
  const I L = (I)p.od[p.rank - 1];
  const I nrows = (I)(p.total / p.od[p.rank - 1]);
  const int lane = threadIdx.x & 31;
  I w = (I)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
  const I nw = (I)(gridDim.x * (blockDim.x >> 5));
  for (I row = w; row < nrows; row += nw) {
    I rem = row, ioff = 0;
    for (int j = p.rank - 2; j >= 0; --j) {
      I q = rem / (I)p.od[j];
      ioff += (rem - q * (I)p.od[j]) * (I)p.os[j];
      rem = q;
    }
    const T* src = in + ioff;
    T* dst = out + row * L;
    for (I e = lane; e < L; e += 32) {
      T v = src[e];
      if (CONJ) v = conjv(v);
      dst[e] = v;
    }
  }
}

template <typename T, bool CONJ, typename I>
__global__ void __launch_bounds__(256) perm_elems(const T* __restrict__ in,
                                                  T* __restrict__ out,
                                                  PermArgs p) {
  // one thread per output element (short rows)
  const I total = (I)p.total;
  for (I o = (I)(blockIdx.x * blockDim.x + threadIdx.x); o < total;
       o += (I)(gridDim.x * blockDim.x)) {
    I rem = o, ioff = 0;
    for (int j = p.rank - 1; j >= 0; --j) {
      I q = rem / (I)p.od[j];
      ioff += (rem - q * (I)p.od[j]) * (I)p.os[j];
      rem = q;
    }
    T v = in[ioff];
    if (CONJ) v = conjv(v);
    out[o] = v;
  }
}

template <typename T, bool CONJ, typename I>
__global__ void __launch_bounds__(256) perm_tile(const T* __restrict__ in,
                                                 T* __restrict__ out,
                                                 PermArgs p, I tiles_a,
                                                 I tiles_b, I nblocks) {
  __shared__ T tile[32][33];
  const int last = p.rank - 1;
  const int a = p.a;
  const I da = (I)p.od[a], db = (I)p.od[last];
  const I sb_in = (I)p.os[last];      // input stride of the output-fastest axis
  const I sa_out = (I)p.ostr[a];      // output stride of the input-fastest axis
  for (I bid = blockIdx.x; bid < nblocks; bid += gridDim.x) {
    I tb = bid % tiles_b;
    I t2 = bid / tiles_b;
    I ta = t2 % tiles_a;
    I batch = t2 / tiles_a;
    I ioff = 0, ooff = 0, rem = batch;
    for (int j = last - 1; j >= 0; --j) {
      if (j == a) continue;
      I q = rem / (I)p.od[j];
      I i = rem - q * (I)p.od[j];
      ioff += i * (I)p.os[j];
      ooff += i * (I)p.ostr[j];
      rem = q;
    }
    const I a0 = ta * 32, b0 = tb * 32;
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      I ia = a0 + threadIdx.x, ib = b0 + yy;
      if (ia < da && ib < db) tile[yy][threadIdx.x] = in[ioff + ia + ib * sb_in];
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += 8) {
      I ia = a0 + yy, ib = b0 + threadIdx.x;
      if (ia < da && ib < db) {
        T v = tile[threadIdx.x][yy];
        if (CONJ) v = conjv(v);
        out[ooff + ia * sa_out + ib] = v;
      }
    }
    __syncthreads();
  }
}

template <typename T, bool CONJ, typename I>
cudaError_t launch(const void* in, void* out, const PermArgs& p,
                   cudaStream_t s, long* launches) {
  const T* src = static_cast<const T*>(in);
  T* dst = static_cast<T*>(out);
  const int last = p.rank - 1;
  const long maxgrid = 152L * 16;
  if (p.os[last] == 1) {
    if (p.od[last] >= 16) {
      long rows = p.total / p.od[last];
      long grid = (rows + 7) / 8;
      if (grid > maxgrid) grid = maxgrid;
      perm_rows<T, CONJ, I><<<(unsigned)grid, 256, 0, s>>>(src, dst, p);
    } else {
      long grid = (p.total + 255) / 256;
      if (grid > maxgrid) grid = maxgrid;
      perm_elems<T, CONJ, I><<<(unsigned)grid, 256, 0, s>>>(src, dst, p);
    }
  } else {
    I tiles_a = (I)((p.od[p.a] + 31) / 32);
    I tiles_b = (I)((p.od[last] + 31) / 32);
    I nbatch = (I)(p.total / (p.od[p.a] * p.od[last]));
    I nblocks = tiles_a * tiles_b * nbatch;
    long grid = (long)nblocks;
    if (grid > maxgrid * 2) grid = maxgrid * 2;
    perm_tile<T, CONJ, I><<<(unsigned)grid, dim3(32, 8), 0, s>>>(
        src, dst, p, tiles_a, tiles_b, nblocks);
  }
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace

cudaError_t permute(const void* in, void* out, int rank, const long* in_dims,
                    const int* perm, bool cx, bool conj, cudaStream_t s,
                    long* launches) {
  if (rank < 1 || rank > 8) return cudaErrorInvalidValue;
  long istr[8];
  long acc = 1;
  for (int j = rank - 1; j >= 0; --j) {
    istr[j] = acc;
    acc *= in_dims[j];
  }
  const long total = acc;
  if (total == 0) return cudaSuccess;
  // output axes, dropping size-1 axes, then fusing axes adjacent in both
  long od[8], os[8];
  int r = 0;
  for (int j = 0; j < rank; ++j) {
    long d = in_dims[perm[j]];
    if (d == 1) continue;
    od[r] = d;
    os[r] = istr[perm[j]];
    ++r;
  }
  PermArgs p{};
  if (r == 0) {
    od[0] = 1;
    os[0] = 1;
    r = 1;
  }
  int n = 0;
  long cd = od[r - 1], cs = os[r - 1];
  long fd[8], fs[8];
  for (int j = r - 2; j >= 0; --j) {
    if (os[j] == cs * cd) {
      cd *= od[j];
    } else {
      fd[n] = cd;
      fs[n] = cs;
      ++n;
      cd = od[j];
      cs = os[j];
    }
  }
  fd[n] = cd;
  fs[n] = cs;
  ++n;
  p.rank = n;
  for (int j = 0; j < n; ++j) {
    p.od[j] = fd[n - 1 - j];
    p.os[j] = fs[n - 1 - j];
  }
  long o = 1;
  for (int j = n - 1; j >= 0; --j) {
    p.ostr[j] = o;
    o *= p.od[j];
  }
  p.total = total;
  p.a = -1;
  for (int j = 0; j < n; ++j)
    if (p.os[j] == 1) p.a = j;
  if (p.rank == 1 && p.os[0] == 1 && !conj) {
    if (launches) ++*launches;
    return cudaMemcpyAsync(out, in, total * (cx ? 16 : 8),
                           cudaMemcpyDeviceToDevice, s);
  }
  if (p.a < 0) return cudaErrorInvalidValue;
  const bool small = total < (1L << 31);
  if (cx) {
    if (conj)
      return small ? launch<cplx, true, uint32_t>(in, out, p, s, launches)
                   : launch<cplx, true, uint64_t>(in, out, p, s, launches);
    return small ? launch<cplx, false, uint32_t>(in, out, p, s, launches)
                 : launch<cplx, false, uint64_t>(in, out, p, s, launches);
  }
  return small ? launch<double, false, uint32_t>(in, out, p, s, launches)
               : launch<double, false, uint64_t>(in, out, p, s, launches);
}

}  // namespace ctm
