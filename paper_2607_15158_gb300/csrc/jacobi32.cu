// fp32 pre-solve of the small SVD (mixed-precision one-sided Jacobi).
//
// The fp64 one-sided Jacobi (jacobi.cu) is bounded on this GPU by the fp64
// pipe and by the latency of its round-robin rounds: about 13 us per round,
// 1.9 ms per sweep for three 149 x 149 complex matrices. Most of its sweeps
// only turn the columns from their initial orientation to near
// orthogonality, which fp32 arithmetic does as well at a fraction of the
// cost. Here each matrix runs the same cyclic one-sided Jacobi (Hestenes;
// the same rotation and round-robin order as the fp64 kernel) in fp32 on a
// cluster of two CTAs: CTA 0 holds A in shared memory and computes and
// applies the rotations of each round; it writes their parameters into the
// shared memory of CTA 1 (distributed shared memory), which holds V and
// applies them one round behind. One cluster barrier separates the rounds.
// The result V0 is accurate to the fp32 threshold; the caller makes it
// unitary in fp64 and runs the fp64 sweeps on A V0, whose columns are then
// orthogonal to ~1e-6 and converge in a few sweeps (quadratic convergence of
// the cyclic method).
#include <cooperative_groups.h>

#include <cfloat>

#include "common.cuh"
#include "kernels.h"

namespace ctm {

namespace {

namespace cg = cooperative_groups;

constexpr int J32T = 1024;   // threads per CTA (32 warps)
constexpr int J32G = J32T / 8;   // 8-lane groups per CTA (one column pair each)

struct J32Args {
  int k, max_sweeps;
  const void* A;    // fp64 k x k row-major per matrix (stride strideA elements)
  long strideA;
  void* V0;         // fp64 k x k row-major per matrix (output)
  int* sweeps;      // sweeps used per matrix (or null)
};

__device__ __forceinline__ int player32(int pos, int t, int m) {
  return pos == 0 ? 0 : ((pos - 1 + t) % m) + 1;
}

// element access: real (float) or complex (float2) fp32
template <bool CX>
struct F32 {
  typedef float2 T;
  __device__ static T zero() { return make_float2(0.f, 0.f); }
  __device__ static T one() { return make_float2(1.f, 0.f); }
  __device__ static T load64s(const void* p, size_t i, double sc) {
    const double2 v = static_cast<const double2*>(p)[i];
    return make_float2(f32_of(v.x * sc), f32_of(v.y * sc));
  }
  __device__ static void store64(void* p, size_t i, T v) {
    static_cast<double2*>(p)[i] = make_double2(f64_of(v.x), f64_of(v.y));
  }
  __device__ static float nrm2(T v) { return v.x * v.x + v.y * v.y; }
  // g += conj(x) y
  __device__ static void dotc(float2& g, T x, T y) {
    g.x = fmaf(x.x, y.x, fmaf(x.y, y.y, g.x));
    g.y = fmaf(x.x, y.y, fmaf(-x.y, y.x, g.y));
  }
  // (x, y) -> (c x - s e y, s x + c e y), e a unit phase
  __device__ static void rot(T& x, T& y, float c, float s, float2 e) {
    const float2 ey = make_float2(e.x * y.x - e.y * y.y, e.x * y.y + e.y * y.x);
    const T xn = make_float2(c * x.x - s * ey.x, c * x.y - s * ey.y);
    const T yn = make_float2(s * x.x + c * ey.x, s * x.y + c * ey.y);
    x = xn;
    y = yn;
  }
};

template <>
struct F32<false> {
  typedef float T;
  __device__ static T zero() { return 0.f; }
  __device__ static T one() { return 1.f; }
  __device__ static T load64s(const void* p, size_t i, double sc) {
    return f32_of(static_cast<const double*>(p)[i] * sc);
  }
  __device__ static void store64(void* p, size_t i, T v) {
    static_cast<double*>(p)[i] = f64_of(v);
  }
  __device__ static float nrm2(T v) { return v * v; }
  __device__ static void dotc(float2& g, T x, T y) { g.x = fmaf(x, y, g.x); }
  __device__ static void rot(T& x, T& y, float c, float s, float2 e) {
    const float ey = e.x * y;
    const T xn = c * x - s * ey;
    y = s * x + c * ey;
    x = xn;
  }
};

// V <- V J for the rotations of round t (CTA 1): group gi takes pair gi
template <bool CX>
__device__ __forceinline__ void apply_round(typename F32<CX>::T* M, const float4* prm, int k,
                                            int kk, int m, int npairs, int t, int gi, int l8) {
  typedef F32<CX> E;
  typedef typename E::T T;
  for (int pr = gi; pr < npairs; pr += J32G) {
    int p = player32(pr, t, m), q = player32(kk - 1 - pr, t, m);
    if (p > q) {
      const int tmp = p;
      p = q;
      q = tmp;
    }
    const float4 rp = prm[pr];
    if (q >= k || rp.y == 0.f) continue;
    T* x = M + (size_t)p * k;
    T* y = M + (size_t)q * k;
    const float2 e = make_float2(rp.z, rp.w);
    #pragma unroll 4
    for (int r = l8; r < k; r += 8) {
      T xv = x[r], yv = y[r];
      E::rot(xv, yv, rp.x, rp.y, e);
      x[r] = xv;
      y[r] = yv;
    }
  }
}

template <bool CX>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(J32T, 1)
    jacobi32_kernel(J32Args a) {
  typedef F32<CX> E;
  typedef typename E::T T;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  const int b = blockIdx.x / 2;
  const int k = a.k;
  const int kk = k + (k & 1), m = kk - 1, npairs = kk / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  T* M = reinterpret_cast<T*>(smem);   // A (rank 0) or V (rank 1), column c at M[c k]
  const size_t mbytes = ((size_t)k * k * sizeof(T) + 15) & ~(size_t)15;
  float4* prm = reinterpret_cast<float4*>(smem + mbytes);   // [2][npairs] (c, s, e)
  __shared__ int rotated, stop;
  __shared__ unsigned long long amax;   // bits of max |a_ij| (non-negative doubles order as integers)
  const int lane = threadIdx.x & 31;
  // groups of 8 lanes, one column pair each: the 4 groups of a warp share its
  // instruction stream (scalar rotation math, reductions)
  const int gi = threadIdx.x >> 3, l8 = threadIdx.x & 7;
  const unsigned m8 = 0xffu << (lane & ~7);   // the lanes of this group (shuffle mask)
  const void* Ab = static_cast<const char*>(a.A) + (size_t)b * a.strideA * (CX ? 16 : 8);
  if (threadIdx.x == 0) {
    rotated = 0;
    stop = 0;
    amax = 0ull;
  }
  __syncthreads();
  if (rank == 0) {
    // scale A by a power of two so that its largest entry is O(1): the
    // rotations do not depend on the scale, and fp32 keeps the squares of
    // the entries in range
    double mx = 0.0;
    const double* Ad = static_cast<const double*>(Ab);
    for (long idx = threadIdx.x; idx < (long)k * k * (CX ? 2 : 1); idx += J32T)
      mx = fmax(mx, fabs(Ad[idx]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0 && mx > 0.0 && isfinite(mx))
      atomicMax(&amax, (unsigned long long)__double_as_longlong(mx));
    __syncthreads();
    const double mxa = __longlong_as_double((long long)amax);
    const double sc = mxa > 0.0 ? ldexp(1.0, -ilogb(mxa)) : 1.0;
    for (long idx = threadIdx.x; idx < (long)k * k; idx += J32T) {
      const int r = (int)(idx / k), c = (int)(idx % k);
      M[(size_t)c * k + r] = E::load64s(Ab, idx, sc);
    }
  } else {
    for (long idx = threadIdx.x; idx < (long)k * k; idx += J32T) {
      const int r = (int)(idx / k), c = (int)(idx % k);
      M[(size_t)c * k + r] = r == c ? E::one() : E::zero();
    }
  }
  float4* prm1 = cl.map_shared_rank(prm, 1);   // CTA 1's parameter slots
  int* stop1 = cl.map_shared_rank(&stop, 1);
  cl.sync();
  // rotate when |gamma| > tol sqrt(alpha beta): a few units of fp32 rounding
  // of a length-k dot product
  const float tol = fmaxf(1e-6f, 2.f * sqrtf((float)k) * FLT_EPSILON);
  int sweep = 0;
  long g = 0;   // rounds done (all sweeps)
  for (; sweep < a.max_sweeps; ++sweep) {
    for (int t = 0; t < m; ++t, ++g) {
      if (rank == 0) {
        for (int pr = gi; pr < npairs; pr += J32G) {
          int p = player32(pr, t, m), q = player32(kk - 1 - pr, t, m);
          if (p > q) {
            const int tmp = p;
            p = q;
            q = tmp;
          }
          float4 rp = make_float4(1.f, 0.f, 1.f, 0.f);   // identity
          if (q < k) {
            T* x = M + (size_t)p * k;
            T* y = M + (size_t)q * k;
            // exact squared norms and the overlap of the pair, every round
            float2 ga = make_float2(0.f, 0.f);
            float al = 0.f, be = 0.f;
            #pragma unroll 4
            for (int r = l8; r < k; r += 8) {
              const T xv = x[r], yv = y[r];
              al += E::nrm2(xv);
              be += E::nrm2(yv);
              E::dotc(ga, xv, yv);
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
              al += __shfl_xor_sync(m8, al, o);
              be += __shfl_xor_sync(m8, be, o);
              ga.x += __shfl_xor_sync(m8, ga.x, o);
              if (CX) ga.y += __shfl_xor_sync(m8, ga.y, o);
            }
            const float gm = sqrtf(ga.x * ga.x + ga.y * ga.y);
            if (gm > tol * sqrtf(al) * sqrtf(be) && gm > 0.f) {
              const float zeta = (be - al) / (2.f * gm);
              const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
              const float c = 1.f / sqrtf(1.f + tt * tt), s = c * tt;
              const float2 e = make_float2(ga.x / gm, -ga.y / gm);   // conj(gamma) / |gamma|
              #pragma unroll 4
              for (int r = l8; r < k; r += 8) {
                T xv = x[r], yv = y[r];
                E::rot(xv, yv, c, s, e);
                x[r] = xv;
                y[r] = yv;
              }
              rp = make_float4(c, s, e.x, e.y);
              if (l8 == 0) rotated = 1;
            }
          }
          if (l8 == 0) prm1[(g & 1) * npairs + pr] = rp;
        }
      } else if (g > 0) {
        // V <- V J for the rotations of the previous round
        const long g1 = g - 1;
        apply_round<CX>(M, prm + (g1 & 1) * npairs, k, kk, m, npairs, (int)(g1 % m), gi, l8);
      }
      cl.sync();
    }
    // a sweep without rotations ends the iteration (decided by CTA 0)
    if (rank == 0 && threadIdx.x == 0) {
      const int s = rotated == 0;
      stop = s;
      *stop1 = s;
      rotated = 0;
    }
    cl.sync();
    if (stop) {
      ++sweep;
      break;
    }
  }
  if (rank == 1) {
    if (g > 0) {
      const long g1 = g - 1;
      apply_round<CX>(M, prm + (g1 & 1) * npairs, k, kk, m, npairs, (int)(g1 % m), gi, l8);
    }
    __syncthreads();
    for (long idx = threadIdx.x; idx < (long)k * k; idx += J32T) {
      const int r = (int)(idx / k), c = (int)(idx % k);
      E::store64(a.V0, (size_t)b * k * k + idx, M[(size_t)c * k + r]);
    }
    if (a.sweeps && threadIdx.x == 0) a.sweeps[b] = sweep;
  }
  // neither CTA leaves while the other may still address its shared memory
  cl.sync();
}

size_t j32_smem(bool cx, int k) {
  const int npairs = (k + (k & 1)) / 2;
  return (((size_t)k * k * (cx ? 8 : 4) + 15) & ~(size_t)15) + 2 * (size_t)npairs * 16;
}

}  // namespace

bool jacobi32_supported(bool cx, int k) {
  return k >= 2 && (k + 1) / 2 <= J32G && j32_smem(cx, k) <= (size_t)227 * 1024;
}

cudaError_t jacobi32_presolve(bool cx, int k, const void* A, long strideA, void* V0, int batch,
                              int max_sweeps, int* sweeps, cudaStream_t s, long* launches) {
  if (!jacobi32_supported(cx, k) || batch < 1) return cudaErrorInvalidValue;
  const size_t shm = j32_smem(cx, k);
  static size_t configured[2] = {0, 0};
  const void* fn = cx ? (const void*)jacobi32_kernel<true> : (const void*)jacobi32_kernel<false>;
  cudaError_t e = raise_smem(fn, configured[cx ? 1 : 0], shm);
  if (e != cudaSuccess) return e;
  J32Args a;
  a.k = k;
  a.max_sweeps = max_sweeps;
  a.A = A;
  a.strideA = strideA;
  a.V0 = V0;
  a.sweeps = sweeps;
  if (cx) jacobi32_kernel<true><<<2 * batch, J32T, shm, s>>>(a);
  else jacobi32_kernel<false><<<2 * batch, J32T, shm, s>>>(a);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace ctm
