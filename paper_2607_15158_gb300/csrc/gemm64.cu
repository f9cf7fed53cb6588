// FP64 / complex-FP64 GEMM on the CUDA cores: C = alpha op(A) op(B) + beta C.
// 64 x 64 output tile per 256-thread block, 4 x 4 outputs per thread, K
// staged through shared memory in slices of 16. Long-K, small-output
// products (Gram matrices, rho = Z_L^H Z_R) split K over blocks and reduce
// the partials in a second, deterministic pass.
#include "common.cuh"
#include "kernels.h"

namespace ctm {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

struct GemmP {
  long M, N, K, kchunk;
  const void* A; long lda, sA;
  const void* B; long ldb, sB;
  void* C; long ldc, sC;
  double2 alpha, beta;
  int splits;
  void* work;
  int lower_only;
};

template <typename T> __device__ __forceinline__ T from2(double2 v);
template <> __device__ __forceinline__ double from2<double>(double2 v) { return v.x; }
template <> __device__ __forceinline__ cplx from2<cplx>(double2 v) { return v; }

__device__ __forceinline__ bool is_zero(double2 v) { return v.x == 0.0 && v.y == 0.0; }

template <typename T, int OPA, int OPB>
__global__ void __launch_bounds__(256) gemm_kernel(GemmP p) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const long m0 = (long)blockIdx.y * BM, n0 = (long)blockIdx.x * BN;
  if (p.lower_only && n0 > m0 + BM - 1) return;   // tile strictly above the diagonal
  const int z = blockIdx.z;
  const int b = z / p.splits, sp = z % p.splits;
  const long kbeg = sp * p.kchunk;
  const long kend = min(p.K, kbeg + p.kchunk);
  const T* A = static_cast<const T*>(p.A) + b * p.sA;
  const T* B = static_cast<const T*>(p.B) + b * p.sB;
  const T zero = zero_of(T());
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zero;

  for (long k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + 256 * i;
      int mm, kk;
      if (OPA == OP_N || OPA == OP_R) { mm = e / BK; kk = e % BK; }
      else { kk = e / BM; mm = e % BM; }
      const long gm = m0 + mm, gk = k0 + kk;
      T v = zero;
      if (gm < p.M && gk < kend) {
        v = (OPA == OP_N || OPA == OP_R) ? A[gm * p.lda + gk] : A[gk * p.lda + gm];
        if (OPA == OP_C || OPA == OP_R) v = conjv(v);
      }
      As[kk][mm] = v;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + 256 * i;
      int nn, kk;
      if (OPB == OP_N || OPB == OP_R) { kk = e / BN; nn = e % BN; }
      else { nn = e / BK; kk = e % BK; }
      const long gn = n0 + nn, gk = k0 + kk;
      T v = zero;
      if (gn < p.N && gk < kend) {
        v = (OPB == OP_N || OPB == OP_R) ? B[gk * p.ldb + gn] : B[gn * p.ldb + gk];
        if (OPB == OP_C || OPB == OP_R) v = conjv(v);
      }
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) fmav(acc[i][j], a[i], bb[j]);
    }
    __syncthreads();
  }

  if (p.splits == 1) {
    T* C = static_cast<T*>(p.C) + b * p.sC;
    const T alpha = from2<T>(p.alpha), beta = from2<T>(p.beta);
    const bool use_beta = !is_zero(p.beta);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long gm = m0 + ty + 16 * i;
      if (gm >= p.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const long gn = n0 + tx + 16 * j;
        if (gn >= p.N) continue;
        T v = mulv(alpha, acc[i][j]);
        if (use_beta) v = addv(v, mulv(beta, C[gm * p.ldc + gn]));
        C[gm * p.ldc + gn] = v;
      }
    }
  } else {
    T* W = static_cast<T*>(p.work) + ((long)b * p.splits + sp) * p.M * p.N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long gm = m0 + ty + 16 * i;
      if (gm >= p.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const long gn = n0 + tx + 16 * j;
        if (gn < p.N) W[gm * p.N + gn] = acc[i][j];
      }
    }
  }
}

template <typename T>
__global__ void splitk_reduce(GemmP p, int batch) {
  const long MN = p.M * p.N;
  const T alpha = from2<T>(p.alpha), beta = from2<T>(p.beta);
  const bool use_beta = !is_zero(p.beta);
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < MN * batch;
       idx += (long)gridDim.x * blockDim.x) {
    const long b = idx / MN, e = idx % MN;
    const T* W = static_cast<const T*>(p.work) + b * p.splits * MN + e;
    T s = zero_of(T());
    for (int k = 0; k < p.splits; ++k) s = addv(s, W[k * MN]);
    T* C = static_cast<T*>(p.C) + b * p.sC;
    const long m = e / p.N, n = e % p.N;
    T v = mulv(alpha, s);
    if (use_beta) v = addv(v, mulv(beta, C[m * p.ldc + n]));
    C[m * p.ldc + n] = v;
  }
}

// ------------------------------------------- tall-skinny C = op(A) B
// op(A) = A^T or A^H with A (K x M) and B (K x N) tall (K >> M, N): the
// Gram matrices of the CholeskyQR passes and rho = Z_L^H Z_R. Each CTA
// takes a contiguous chunk of the K rows (staged through shared memory,
// TS_ROWS at a time) and a slice of the outputs (TS_OUTS per thread, in
// registers); per-chunk partials are summed in a second pass in chunk order.
constexpr int TS_THREADS = 512, TS_OUTS = 12, TS_ROWS = 16, TS_MAXMN = 384;

template <typename T, bool CONJ>
__global__ void __launch_bounds__(TS_THREADS) gemm_ts_kernel(long K, int M, int N, int lower,
                                                             const T* __restrict__ A, long lda,
                                                             const T* __restrict__ B, long ldb,
                                                             long chunk, long nout,
                                                             T* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);   // [TS_ROWS][M]
  T* Bs = As + (size_t)TS_ROWS * M;          // [TS_ROWS][N]
  const long r0 = blockIdx.x * chunk;
  const long r1 = min(K, r0 + chunk);
  const long e0 = (long)blockIdx.y * TS_THREADS * TS_OUTS;
  int oi[TS_OUTS], oj[TS_OUTS];
  T acc[TS_OUTS];
#pragma unroll
  for (int m = 0; m < TS_OUTS; ++m) {
    const long e = e0 + threadIdx.x + (long)m * TS_THREADS;
    oi[m] = -1;
    oj[m] = 0;
    acc[m] = zero_of(T());
    if (e < nout) {
      if (lower) {
        int i = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
        while ((long)i * (i + 1) / 2 > e) --i;
        while ((long)(i + 1) * (i + 2) / 2 <= e) ++i;
        oi[m] = i;
        oj[m] = (int)(e - (long)i * (i + 1) / 2);
      } else {
        oi[m] = (int)(e / N);
        oj[m] = (int)(e % N);
      }
    }
  }
  for (long rb = r0; rb < r1; rb += TS_ROWS) {
    const int nr = (int)min((long)TS_ROWS, r1 - rb);
    __syncthreads();
    for (int idx = threadIdx.x; idx < TS_ROWS * M; idx += TS_THREADS) {
      const int rr = idx / M, i = idx % M;
      T v = zero_of(T());
      if (rr < nr) v = A[(rb + rr) * lda + i];
      As[idx] = CONJ ? conjv(v) : v;
    }
    for (int idx = threadIdx.x; idx < TS_ROWS * N; idx += TS_THREADS) {
      const int rr = idx / N, j = idx % N;
      Bs[idx] = rr < nr ? B[(rb + rr) * ldb + j] : zero_of(T());
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < TS_ROWS; ++rr) {
      const T* ar = As + (size_t)rr * M;
      const T* br = Bs + (size_t)rr * N;
#pragma unroll
      for (int m = 0; m < TS_OUTS; ++m)
        if (oi[m] >= 0) fmav(acc[m], ar[oi[m]], br[oj[m]]);
    }
  }
#pragma unroll
  for (int m = 0; m < TS_OUTS; ++m) {
    const long e = e0 + threadIdx.x + (long)m * TS_THREADS;
    if (e < nout) part[(size_t)blockIdx.x * nout + e] = acc[m];
  }
}

template <typename T>
__global__ void gemm_ts_reduce(int nchunks, long nout, int N, int lower, const T* part, T* C,
                               long ldc) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nout;
       e += (long)gridDim.x * blockDim.x) {
    T s = zero_of(T());
    for (int b = 0; b < nchunks; ++b) s = addv(s, part[(size_t)b * nout + e]);
    long i, j;
    if (lower) {
      i = (long)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
      while (i * (i + 1) / 2 > e) --i;
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      j = e - i * (i + 1) / 2;
    } else {
      i = e / N;
      j = e % N;
    }
    C[i * ldc + j] = s;
  }
}

struct TsPlan {
  bool use = false;
  long nout = 0;
  int gy = 1, gx = 1;
  long chunk = 0;
};

TsPlan ts_plan(const GemmDesc& g) {
  TsPlan t;
  const bool plain = g.alpha[0] == 1.0 && g.alpha[1] == 0.0 && g.beta[0] == 0.0 &&
                     g.beta[1] == 0.0;
  if (!(plain && g.batch == 1 && (g.opA == OP_T || g.opA == OP_C) && g.opB == OP_N &&
        g.M <= TS_MAXMN && g.N <= TS_MAXMN && g.K >= 4096 && (!g.lower_only || g.M == g.N)))
    return t;
  t.use = true;
  t.nout = g.lower_only ? g.M * (g.M + 1) / 2 : g.M * g.N;
  t.gy = (int)((t.nout + (long)TS_THREADS * TS_OUTS - 1) / ((long)TS_THREADS * TS_OUTS));
  t.gx = 152 / t.gy;
  if (t.gx < 1) t.gx = 1;
  t.chunk = (g.K + t.gx - 1) / t.gx;
  t.chunk = (t.chunk + TS_ROWS - 1) / TS_ROWS * TS_ROWS;
  t.gx = (int)((g.K + t.chunk - 1) / t.chunk);
  return t;
}

template <typename T>
cudaError_t run_ts(const GemmDesc& g, const TsPlan& t, void* work, cudaStream_t s,
                   long* launches) {
  const size_t shm = (size_t)TS_ROWS * (g.M + g.N) * sizeof(T);
  static size_t configured[2] = {0, 0};
  const cudaError_t e =
      g.opA == OP_C ? raise_smem((const void*)gemm_ts_kernel<T, true>, configured[1], shm)
                    : raise_smem((const void*)gemm_ts_kernel<T, false>, configured[0], shm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)t.gx, (unsigned)t.gy);
  if (g.opA == OP_C)
    gemm_ts_kernel<T, true><<<grid, TS_THREADS, shm, s>>>(
        g.K, (int)g.M, (int)g.N, g.lower_only ? 1 : 0, static_cast<const T*>(g.A), g.lda,
        static_cast<const T*>(g.B), g.ldb, t.chunk, t.nout, static_cast<T*>(work));
  else
    gemm_ts_kernel<T, false><<<grid, TS_THREADS, shm, s>>>(
        g.K, (int)g.M, (int)g.N, g.lower_only ? 1 : 0, static_cast<const T*>(g.A), g.lda,
        static_cast<const T*>(g.B), g.ldb, t.chunk, t.nout, static_cast<T*>(work));
  long rg = (t.nout + 255) / 256;
  if (rg > 152 * 8) rg = 152 * 8;
  gemm_ts_reduce<T><<<(unsigned)rg, 256, 0, s>>>(t.gx, t.nout, (int)g.N, g.lower_only ? 1 : 0,
                                                  static_cast<const T*>(work),
                                                  static_cast<T*>(g.C), g.ldc);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

int choose_splits(const GemmDesc& g) {
  const long tiles = ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN) * g.batch;
  const long target = 152L * 2;
  if (tiles >= target / 2) return 1;
  long s = target / tiles;
  const long kmax = (g.K + 4 * BK - 1) / (4 * BK);  // at least 4 k-slices each
  if (s > kmax) s = kmax;
  if (s > 64) s = 64;
  return s < 1 ? 1 : (int)s;
}

template <typename T, int OPA, int OPB>
cudaError_t run(const GemmP& p, int batch, cudaStream_t s, long* launches) {
  dim3 grid((unsigned)((p.N + BN - 1) / BN), (unsigned)((p.M + BM - 1) / BM),
            (unsigned)(batch * p.splits));
  gemm_kernel<T, OPA, OPB><<<grid, 256, 0, s>>>(p);
  if (launches) ++*launches;
  if (p.splits > 1) {
    long n = p.M * p.N * batch;
    long g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    splitk_reduce<T><<<(unsigned)g, 256, 0, s>>>(p, batch);
    if (launches) ++*launches;
  }
  return cudaGetLastError();
}

template <typename T, int OPA>
cudaError_t dispatch_b(const GemmP& p, int opB, int batch, cudaStream_t s, long* l) {
  switch (opB) {
    case OP_N: return run<T, OPA, OP_N>(p, batch, s, l);
    case OP_T: return run<T, OPA, OP_T>(p, batch, s, l);
    case OP_C: return run<T, OPA, OP_C>(p, batch, s, l);
    default: return run<T, OPA, OP_R>(p, batch, s, l);
  }
}

template <typename T>
cudaError_t dispatch(const GemmP& p, int opA, int opB, int batch, cudaStream_t s, long* l) {
  switch (opA) {
    case OP_N: return dispatch_b<T, OP_N>(p, opB, batch, s, l);
    case OP_T: return dispatch_b<T, OP_T>(p, opB, batch, s, l);
    case OP_C: return dispatch_b<T, OP_C>(p, opB, batch, s, l);
    default: return dispatch_b<T, OP_R>(p, opB, batch, s, l);
  }
}

// ---------------------------------------------------------------- dot
template <typename T, bool CONJ>
__global__ void dot_partial(long n, const T* x, long sx, const T* y, long sy,
                            T* part, int nblk) {
  const int b = blockIdx.y;
  const T* xb = x + b * sx;
  const T* yb = y + b * sy;
  T acc = zero_of(T());
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    if (CONJ) fmacv(acc, xb[i], yb[i]);
    else fmav(acc, xb[i], yb[i]);
  }
  __shared__ T red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    T v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : zero_of(T());
    v = warp_sum(v);
    if (threadIdx.x == 0) part[b * nblk + blockIdx.x] = v;
  }
}

template <typename T>
__global__ void dot_final(const T* part, int nblk, T* out) {
  const int b = blockIdx.x;
  T acc = zero_of(T());
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc = addv(acc, part[b * nblk + i]);
  __shared__ T red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    T v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : zero_of(T());
    v = warp_sum(v);
    if (threadIdx.x == 0) out[b] = v;
  }
}

}  // namespace

size_t gemm64_work_bytes(const GemmDesc& g) {
  const TsPlan t = ts_plan(g);
  if (t.use) return (size_t)t.gx * t.nout * (g.cx ? 16 : 8);
  const int splits = choose_splits(g);
  if (splits == 1) return 0;
  return (size_t)splits * g.batch * g.M * g.N * (g.cx ? 16 : 8);
}

cudaError_t gemm64(const GemmDesc& g, void* work, size_t work_bytes,
                   cudaStream_t s, long* launches) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  const TsPlan t = ts_plan(g);
  if (t.use && work && work_bytes >= gemm64_work_bytes(g))
    return g.cx ? run_ts<cplx>(g, t, work, s, launches) : run_ts<double>(g, t, work, s, launches);
  GemmP p{};
  p.M = g.M; p.N = g.N; p.K = g.K;
  p.A = g.A; p.lda = g.lda; p.sA = g.strideA;
  p.B = g.B; p.ldb = g.ldb; p.sB = g.strideB;
  p.C = g.C; p.ldc = g.ldc; p.sC = g.strideC;
  p.alpha = make_double2(g.alpha[0], g.alpha[1]);
  p.beta = make_double2(g.beta[0], g.beta[1]);
  p.lower_only = g.lower_only ? 1 : 0;
  p.splits = choose_splits(g);
  if (p.splits > 1 && work_bytes < gemm64_work_bytes(g)) p.splits = 1;
  p.work = work;
  long kc = (g.K + p.splits - 1) / p.splits;
  kc = (kc + BK - 1) / BK * BK;
  p.kchunk = kc > 0 ? kc : BK;
  if (g.K == 0) p.kchunk = 0;
  if (g.cx) return dispatch<cplx>(p, g.opA, g.opB, g.batch, s, launches);
  return dispatch<double>(p, g.opA, g.opB, g.batch, s, launches);
}

cudaError_t dot64(bool cx, bool conj_x, long n, const void* x, long sx,
                  const void* y, long sy, void* out, int batch, void* work,
                  size_t work_bytes, cudaStream_t s, long* launches) {
  int nblk = (int)((n + 255) / 256);
  if (nblk > 304) nblk = 304;
  if (nblk < 1) nblk = 1;
  const size_t need = (size_t)nblk * batch * (cx ? 16 : 8);
  if (work_bytes < need) return cudaErrorInvalidValue;
  dim3 grid(nblk, batch);
  if (cx) {
    if (conj_x)
      dot_partial<cplx, true><<<grid, 256, 0, s>>>(n, (const cplx*)x, sx, (const cplx*)y, sy, (cplx*)work, nblk);
    else
      dot_partial<cplx, false><<<grid, 256, 0, s>>>(n, (const cplx*)x, sx, (const cplx*)y, sy, (cplx*)work, nblk);
    dot_final<cplx><<<batch, 256, 0, s>>>((const cplx*)work, nblk, (cplx*)out);
  } else {
    dot_partial<double, false><<<grid, 256, 0, s>>>(n, (const double*)x, sx, (const double*)y, sy, (double*)work, nblk);
    dot_final<double><<<batch, 256, 0, s>>>((const double*)work, nblk, (double*)out);
  }
  if (launches) *launches += 2;
  return cudaGetLastError();
}

}  // namespace ctm
