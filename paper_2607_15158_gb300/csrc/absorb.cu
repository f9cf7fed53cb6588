// Single-layer absorption of the ket and bra tensors into a corner / edge
// block (paper Eq. rho_M_diag, Fig. ctmrg-step: A and conj(A) are absorbed
// one after the other, never as the double-layer A (x) conj(A)):
//
//   Out[t,d,D,n,e,E] = sum_{s,u,l,v,w} A[s,u,l,d,e] B[s,v,w,D,E] In[t,l,w,n,u,v]
//
// In and Out are [chi, Dk, Db, chi, Dk, Db] row-major. For every (t, n) the
// work is two small matrix products per physical index s,
//   Y_s = A_s X       (Dk^2 x Dk^2) (Dk^2 x Db^2),  X[(u,l),(w,v)] = In[t,l,w,n,u,v]
//   Out += Y_s B_s    (Dk^2 x Db^2) (Db^2 x Db^2),  B_s[(w,v),(D,E)] = B[s,v,w,D,E]
// so one kernel reads In once and writes Out once (the unfused form is two
// permutes, two GEMMs and a final permute); the fp32 arithmetic, not HBM,
// bounds it. Each CTA holds A and B in shared memory and runs NG groups of
// GT x GT threads, one (t, n) pair each; a thread owns a TL x TL register
// tile of the products, rows ti + GT a and columns tj + GT b (consecutive
// threads read consecutive shared-memory words). Geometries: GT = 12,
// TL = 3 for Dk^2, Db^2 <= 36 (D <= 6), with four groups and the next
// pair's input staged by cp.async in fp32, else two groups; GT = 16, TL = 4,
// one group for <= 64 (D <= 8). D = 6 and D = 8 also have compile-time
// variants. Arithmetic in F: fp32 (split-precision contexts, ~1e-7 relative
// like the bf16x3 products) or fp64.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace ctm {

namespace {

constexpr size_t SMEM_MAX = 227 * 1024;   // shared memory of one block

// hardware conversions here: they issue on the narrow fp64 pipe, but that
// pipe is otherwise idle in this kernel and other warps' fp32 work covers
// them (the integer-pipe conversions of common.cuh measured 12 % slower)
__device__ __forceinline__ float cvt(double a, float) { return (float)a; }
__device__ __forceinline__ float2 cvt(cplx a, float2) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double cvt(double a, double) { return a; }
__device__ __forceinline__ cplx cvt(cplx a, cplx) { return a; }
__device__ __forceinline__ double back(float a) { return (double)a; }
__device__ __forceinline__ cplx back(float2 a) { return make_double2((double)a.x, (double)a.y); }
__device__ __forceinline__ double back(double a) { return a; }
__device__ __forceinline__ cplx back(cplx a) { return a; }

__device__ __forceinline__ void mac(float& c, float a, float b) { c = fmaf(a, b, c); }
__device__ __forceinline__ void mac(float2& c, float2 a, float2 b) {
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
}
__device__ __forceinline__ void mac(double& c, double a, double b) { c = fma(a, b, c); }
__device__ __forceinline__ void mac(cplx& c, cplx a, cplx b) { fmav(c, a, b); }
template <typename F> __device__ __forceinline__ F fz();
template <> __device__ __forceinline__ float fz<float>() { return 0.f; }
template <> __device__ __forceinline__ float2 fz<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double fz<double>() { return 0.0; }
template <> __device__ __forceinline__ cplx fz<cplx>() { return make_double2(0.0, 0.0); }

// asynchronous global -> shared copies of one input element (Ampere+ cp.async)
__device__ __forceinline__ void cp_async_elem(cplx* dst, const cplx* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_elem(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// two blocks per SM where their shared memory allows (two groups, 8-byte F)
template <typename F, int NG>
constexpr int ab_min_blocks() {
  return (NG == 2 && sizeof(F) <= 8) ? 2 : 1;
}

// ST: the next pair's input block is copied into a staging buffer with
// cp.async while the current pair is computed (fp32 arithmetic, D <= 6)
// DK > 0: Dk = Db = DK fixed at compile time (constant index arithmetic, and
// no bounds tests when the DK^2 x DK^2 tile fills the threads exactly)
template <typename T, typename F, int GT, int TL, int NG, bool ST, int DK>
__global__ void __launch_bounds__(NG * GT * GT, ab_min_blocks<F, NG>())
    absorb_ab_kernel(int chi, int dk_arg, int db_arg, int d, const T* __restrict__ In,
                     const T* __restrict__ A, const T* __restrict__ B, T* __restrict__ Out) {
  constexpr int GROUP = GT * GT;   // threads per (t, n) pair
  constexpr int TILE = TL;         // register tile per thread
  constexpr bool kFull = DK > 0 && DK * DK == GT * TL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Dk = DK > 0 ? DK : dk_arg, Db = DK > 0 ? DK : db_arg;
  const int K1 = Dk * Dk, N1 = Db * Db;          // (u,l) and (w,v); M1 = K1 rows (d,e)
  F* As = reinterpret_cast<F*>(smem_raw);         // [d][(d,e)][(u,l)]
  F* Bs = As + (size_t)d * K1 * K1;               // [d][(w,v)][(D,E)]
  const int grp = threadIdx.x / GROUP, lt = threadIdx.x % GROUP;
  F* Xs = Bs + (size_t)d * N1 * N1 + (size_t)grp * 2 * K1 * N1;   // [(u,l)][(w,v)]
  F* Ys = Xs + (size_t)K1 * N1;                                   // [(d,e)][(w,v)], then Out
  const int ti = lt / GT, tj = lt % GT;
  // staging buffers (raw input elements, 16-byte aligned) after all groups' X, Y
  T* St = nullptr;
  if constexpr (ST) {
    const uintptr_t end = reinterpret_cast<uintptr_t>(Bs + (size_t)d * N1 * N1 +
                                                      (size_t)NG * 2 * K1 * N1);
    St = reinterpret_cast<T*>((end + 15) & ~(uintptr_t)15) + (size_t)grp * K1 * N1;
  }
  for (int i = threadIdx.x; i < d * K1 * K1; i += blockDim.x) {
    // As[s][(d,e)][(u,l)] = A[s,u,l,d,e]
    const int s = i / (K1 * K1), rem = i % (K1 * K1);
    const int r = rem / K1, kk = rem % K1;
    const int dd = r / Dk, e = r % Dk, u = kk / Dk, l = kk % Dk;
    As[i] = cvt(A[(((size_t)(s * Dk + u) * Dk + l) * Dk + dd) * Dk + e], F());
  }
  for (int i = threadIdx.x; i < d * N1 * N1; i += blockDim.x) {
    // Bs[s][(w,v)][(D,E)] = B[s,v,w,D,E]
    const int s = i / (N1 * N1), rem = i % (N1 * N1);
    const int kk = rem / N1, c = rem % N1;
    const int w = kk / Db, v = kk % Db, D = c / Db, E = c % Db;
    Bs[i] = cvt(B[(((size_t)(s * Db + v) * Db + w) * Db + D) * Db + E], F());
  }
  const size_t row = (size_t)chi * Dk * Db;       // stride of the (first chi, Dk, Db) index
  const long npairs = (long)chi * chi;
  // element i = (l w, u v) of pair pp's block: In[t,l,w,n,u,v], runs of Dk Db
  // contiguous (u, v)
  auto src_of = [&](long pp, int i) {
    const int tt = (int)(pp / chi), nn = (int)(pp % chi);
    const int lw = i / (Dk * Db), uv = i % (Dk * Db);
    const int l = lw / Db, w = lw % Db;
    return In + ((size_t)tt * Dk + l) * Db * row + (size_t)w * row + (size_t)nn * Dk * Db + uv;
  };
  if constexpr (ST) {
    const long pf = (long)NG * blockIdx.x + grp;
    if (pf < npairs)
      for (int i = lt; i < K1 * N1; i += GROUP) cp_async_elem(St + i, src_of(pf, i));
    cp_async_commit();
  }
  for (long p0 = (long)NG * blockIdx.x; p0 < npairs; p0 += (long)NG * gridDim.x) {
    const long p = p0 + grp;
    const bool live = p < npairs;
    const int t = live ? (int)(p / chi) : 0, n = live ? (int)(p % chi) : 0;
    if constexpr (ST) {
      cp_async_wait_all();
      __syncthreads();   // staged blocks complete; previous output staging consumed
      if (live)
        for (int i = lt; i < K1 * N1; i += GROUP) {
          const int lw = i / (Dk * Db), uv = i % (Dk * Db);
          const int l = lw / Db, w = lw % Db, u = uv / Db, v = uv % Db;
          Xs[(u * Dk + l) * N1 + w * Db + v] = cvt(St[i], F());
        }
      __syncthreads();   // the staging buffers are free again
      const long pn = p + (long)NG * gridDim.x;
      if (pn < npairs)
        for (int i = lt; i < K1 * N1; i += GROUP) cp_async_elem(St + i, src_of(pn, i));
      cp_async_commit();
    } else {
      __syncthreads();   // previous pair's output staging is consumed
      if (live) {
        // X[(u,l),(w,v)] = In[t,l,w,n,u,v]
        for (int i = lt; i < K1 * N1; i += GROUP) {
          const int lw = i / (Dk * Db), uv = i % (Dk * Db);
          const int l = lw / Db, w = lw % Db, u = uv / Db, v = uv % Db;
          Xs[(u * Dk + l) * N1 + w * Db + v] = cvt(*src_of(p, i), F());
        }
      }
    }
    F acc[TILE][TILE];
#pragma unroll
    for (int a = 0; a < TILE; ++a)
#pragma unroll
      for (int b = 0; b < TILE; ++b) acc[a][b] = fz<F>();
    for (int s = 0; s < d; ++s) {
      __syncthreads();   // X loaded / previous Y consumed
      const F* Asb = As + (size_t)s * K1 * K1;
      if (live) {
        F y[TILE][TILE];
#pragma unroll
        for (int a = 0; a < TILE; ++a)
#pragma unroll
          for (int b = 0; b < TILE; ++b) y[a][b] = fz<F>();
#pragma unroll 4
        for (int kk = 0; kk < K1; ++kk) {
          F xa[TILE], xb[TILE];
#pragma unroll
          for (int a = 0; a < TILE; ++a) {
            const int r = ti + GT * a;
            xa[a] = (kFull || r < K1) ? Asb[r * K1 + kk] : fz<F>();
          }
#pragma unroll
          for (int b = 0; b < TILE; ++b) {
            const int c = tj + GT * b;
            xb[b] = (kFull || c < N1) ? Xs[kk * N1 + c] : fz<F>();
          }
#pragma unroll
          for (int a = 0; a < TILE; ++a)
#pragma unroll
            for (int b = 0; b < TILE; ++b) mac(y[a][b], xa[a], xb[b]);
        }
#pragma unroll
        for (int a = 0; a < TILE; ++a)
#pragma unroll
          for (int b = 0; b < TILE; ++b) {
            const int r = ti + GT * a, c = tj + GT * b;
            if (kFull || (r < K1 && c < N1)) Ys[r * N1 + c] = y[a][b];
          }
      }
      __syncthreads();
      const F* Bsb = Bs + (size_t)s * N1 * N1;
      if (live) {
#pragma unroll 4
        for (int kk = 0; kk < N1; ++kk) {
          F ya[TILE], bb[TILE];
#pragma unroll
          for (int a = 0; a < TILE; ++a) {
            const int r = ti + GT * a;
            ya[a] = (kFull || r < K1) ? Ys[r * N1 + kk] : fz<F>();
          }
#pragma unroll
          for (int b = 0; b < TILE; ++b) {
            const int c = tj + GT * b;
            bb[b] = (kFull || c < N1) ? Bsb[kk * N1 + c] : fz<F>();
          }
#pragma unroll
          for (int a = 0; a < TILE; ++a)
#pragma unroll
            for (int b = 0; b < TILE; ++b) mac(acc[a][b], ya[a], bb[b]);
        }
      }
    }
    __syncthreads();   // all Y reads done: Ys becomes the output staging
    if (live) {
#pragma unroll
      for (int a = 0; a < TILE; ++a)
#pragma unroll
        for (int b = 0; b < TILE; ++b) {
          const int r = ti + GT * a, c = tj + GT * b;
          if (kFull || (r < K1 && c < N1)) Ys[r * N1 + c] = acc[a][b];
        }
    }
    __syncthreads();
    if (live) {
      // Out[t,d,D,n,e,E] = O[(d,e),(D,E)]: runs of Dk Db contiguous (e, E)
      for (int i = lt; i < K1 * N1; i += GROUP) {
        const int dD = i / (Dk * Db), eE = i % (Dk * Db);
        const int dd = dD / Db, D = dD % Db, e = eE / Db, E = eE % Db;
        Out[((size_t)t * Dk + dd) * Db * row + (size_t)D * row + (size_t)n * Dk * Db + eE] =
            back(Ys[(dd * Dk + e) * N1 + D * Db + E]);
      }
    }
  }
}

// shared memory of a geometry with ng groups: A and B, then X and Y per
// group, then (staged) one raw input block per group
size_t ab_smem(int Dk, int Db, int d, int ng, size_t fsize, size_t tsize, bool staged) {
  const size_t K1 = (size_t)Dk * Dk, N1 = (size_t)Db * Db;
  size_t b = ((size_t)d * K1 * K1 + (size_t)d * N1 * N1 + 2 * (size_t)ng * K1 * N1) * fsize;
  if (staged) b = (b + 15) / 16 * 16 + (size_t)ng * K1 * N1 * tsize;
  return b;
}

// 0: no fused kernel; 3: 12 x 12 threads x 3 x 3 tiles, four groups with
// staged input (fp32, D <= 6); 1: the same tiles, two groups; 2: 16 x 16
// threads x 4 x 4 tiles, one group (D <= 8)
int ab_geometry(int Dk, int Db, int d, size_t fsize, size_t tsize) {
  if (Dk < 1 || Db < 1 || d < 1) return 0;
  const int m = std::max(Dk * Dk, Db * Db);
  if (m <= 36 && fsize < tsize && ab_smem(Dk, Db, d, 4, fsize, tsize, true) <= SMEM_MAX) return 3;
  if (m <= 36 && ab_smem(Dk, Db, d, 2, fsize, tsize, false) <= SMEM_MAX) return 1;
  if (m <= 64 && ab_smem(Dk, Db, d, 1, fsize, tsize, false) <= SMEM_MAX) return 2;
  return 0;
}

template <typename T, typename F, int GT, int TL, int NG, bool ST, int DK>
cudaError_t launch_ab(int chi, int Dk, int Db, int d, const void* In, const void* A,
                      const void* B, void* Out, int num_sms, cudaStream_t s) {
  const size_t shm = ab_smem(Dk, Db, d, NG, sizeof(F), sizeof(T), ST);
  static size_t configured = 0;
  auto* fn = absorb_ab_kernel<T, F, GT, TL, NG, ST, DK>;
  cudaError_t e = raise_smem((const void*)fn, configured, shm);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NG * GT * GT, shm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long grid = (long)num_sms * per_sm;
  const long tiles = ((long)chi * chi + NG - 1) / NG;
  if (grid > tiles) grid = tiles;
  fn<<<(unsigned)grid, NG * GT * GT, shm, s>>>(chi, Dk, Db, d, static_cast<const T*>(In),
                                                 static_cast<const T*>(A),
                                                 static_cast<const T*>(B), static_cast<T*>(Out));
  return cudaGetLastError();
}

template <typename T, typename F>
cudaError_t launch_geom(int geom, int chi, int Dk, int Db, int d, const void* In, const void* A,
                        const void* B, void* Out, int num_sms, cudaStream_t s) {
  const bool sq = Dk == Db;
  if constexpr (sizeof(F) < sizeof(T)) {
    if (geom == 3 && sq && Dk == 6)
      return launch_ab<T, F, 12, 3, 4, true, 6>(chi, Dk, Db, d, In, A, B, Out, num_sms, s);
    if (geom == 3)
      return launch_ab<T, F, 12, 3, 4, true, 0>(chi, Dk, Db, d, In, A, B, Out, num_sms, s);
    if (geom == 2 && sq && Dk == 8)
      return launch_ab<T, F, 16, 4, 1, false, 8>(chi, Dk, Db, d, In, A, B, Out, num_sms, s);
  }
  if (geom == 1)
    return launch_ab<T, F, 12, 3, 2, false, 0>(chi, Dk, Db, d, In, A, B, Out, num_sms, s);
  return launch_ab<T, F, 16, 4, 1, false, 0>(chi, Dk, Db, d, In, A, B, Out, num_sms, s);
}

size_t elem_size(bool cx, bool fp32) { return (cx ? 2 : 1) * (fp32 ? 4 : 8); }

}  // namespace

bool absorb_ab_supported(bool cx, bool fp32, int Dk, int Db, int d) {
  return ab_geometry(Dk, Db, d, elem_size(cx, fp32), elem_size(cx, false)) != 0;
}

cudaError_t absorb_ab(bool cx, bool fp32, int chi, int Dk, int Db, int d, const void* In,
                      const void* A, const void* B, void* Out, int num_sms, cudaStream_t s,
                      long* launches) {
  const int geom = ab_geometry(Dk, Db, d, elem_size(cx, fp32), elem_size(cx, false));
  if (geom == 0 || chi < 1) return cudaErrorInvalidValue;
  cudaError_t e;
  if (cx)
    e = fp32 ? launch_geom<cplx, float2>(geom, chi, Dk, Db, d, In, A, B, Out, num_sms, s)
             : launch_geom<cplx, cplx>(geom, chi, Dk, Db, d, In, A, B, Out, num_sms, s);
  else
    e = fp32 ? launch_geom<double, float>(geom, chi, Dk, Db, d, In, A, B, Out, num_sms, s)
             : launch_geom<double, double>(geom, chi, Dk, Db, d, In, A, B, Out, num_sms, s);
  if (launches) ++*launches;
  return e;
}

}  // namespace ctm
