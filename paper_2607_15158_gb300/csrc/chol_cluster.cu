// Cholesky factor (and inverse) of the k x k Gram of a CholeskyQR pass on a
// cluster of eight CTAs.
//
// GB300 executes about 1.6 fp64 multiply-adds per clock per SM, so the
// right-looking factorisation of a 149 x 149 complex Gram (k^3 / 6 complex
// multiply-adds) takes ~0.8 ms on one SM. Here the rows are dealt
// cyclically to the eight CTAs of a cluster (row i to CTA i mod 8), each CTA
// keeping its rows of the packed lower triangle in shared memory. Step j:
// every CTA writes its unscaled entries G(i, j), i > j, into the column
// buffer of every CTA (distributed shared memory) and the owner of row j
// publishes the pivot sqrt(G(j, j)); after one cluster barrier every CTA
// scales its entries of column j and updates its rows of the trailing
// matrix. Column and pivot buffers alternate between steps, so one barrier
// per column suffices. The options (Jacobi scaling D^-1 G D^-1, the shift of
// shifted CholeskyQR, the detection of numerically dependent columns) are
// those of the one-block kernel (linalg.cu). With want_inv the CTAs then
// gather the whole factor and each computes every eighth column of L^-1 by
// forward substitution, writing W = D^-1 L^-H.
#include <cooperative_groups.h>

#include <cfloat>

#include "common.cuh"
#include "kernels.h"

namespace ctm {

namespace {

namespace cg = cooperative_groups;

constexpr int CC = 8;     // CTAs per cluster
constexpr int CT = 256;   // threads per CTA

__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }   // i >= j

struct Pivot {
  double piv, inv;   // pivot and its reciprocal (formed once, by the owner)
  int dead;
  int pad;
};

struct CholClusterArgs {
  int k, shift, scale, want_inv;
  long n;            // rows of the block whose Gram this is (for the shift)
  const void* G;     // k x k, lower triangle read
  void* L;           // k x k factor (row-major, zero above the diagonal)
  void* W;           // k x k D^-1 L^-H (row-major upper) when want_inv
  double* dsc;       // k column scales D
  int* dead;         // k flags or null
  int* err;
};

template <typename T>
__device__ __forceinline__ T one_of() {
  if constexpr (sizeof(T) == 8) return T(1.0);
  else return make_double2(1.0, 0.0);
}

template <typename T>
__global__ void __cluster_dims__(CC, 1, 1) __launch_bounds__(CT, 1)
    chol_cluster_kernel(CholClusterArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int k = a.k;
  extern __shared__ __align__(16) unsigned char smem[];
  T* S = reinterpret_cast<T*>(smem);                        // packed lower triangle
  T* colbuf = S + (size_t)k * (k + 1) / 2;                  // [2][k] conj of column j
  double* dsc = reinterpret_cast<double*>(colbuf + 2 * k);  // [k]
  double* orig = dsc + k;                                   // [k] scaled diagonal
  T* xs = reinterpret_cast<T*>(orig + k);                   // [CT / 32][k] inverse columns
  __shared__ Pivot pivbuf[2];
  __shared__ double red[CT / 32];
  __shared__ double sft_s;
  const T* G = static_cast<const T*>(a.G);
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = CT / 32;
  // scales, shift (every CTA computes them from the diagonal of G)
  double tr = 0.0;
  for (int i = threadIdx.x; i < k; i += CT) {
    const double d = realv(G[(size_t)i * k + i]);
    const double s = a.scale ? (d > 0.0 ? sqrt(d) : 1.0) : 1.0;
    dsc[i] = s;
    orig[i] = d / (s * s);
    tr += orig[i];
    if (a.dead && i % CC == rank) a.dead[i] = 0;
  }
  tr = warp_sum(tr);
  if (lane == 0) red[wp] = tr;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    sft_s = a.shift ? 11.0 * ((double)a.n * k + (double)k * (k + 1)) * DBL_EPSILON * t : 0.0;
  }
  __syncthreads();
  const double sft = sft_s;
  // own rows of D^-1 G D^-1 + sft I (one warp per row)
  for (int i = rank + CC * wp; i < k; i += CC * nw) {
    for (int l = lane; l <= i; l += 32) {
      T v = scalev(G[(size_t)i * k + l], 1.0 / (dsc[i] * dsc[l]));
      if (l == i) {
        if constexpr (sizeof(T) == 8) v += sft;
        else v.x += sft;
      }
      S[tri(i, l)] = v;
    }
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    const int slot = j & 1;
    // phase A: broadcast the unscaled column j and the pivot
    {
      const int first = j + 1 + ((rank - (j + 1)) % CC + CC) % CC;   // first own row > j
      const int nown = first < k ? (k - 1 - first) / CC + 1 : 0;
      for (int idx = threadIdx.x; idx < nown * CC; idx += CT) {
        const int i = first + CC * (idx / CC), dst = idx % CC;
        T* cb = cl.map_shared_rank(colbuf, dst);
        cb[slot * k + i] = conjv(S[tri(i, j)]);
      }
      if (j % CC == rank && threadIdx.x == 0) {
        const double d = realv(S[tri(j, j)]);
        Pivot pv;
        pv.pad = 0;
        pv.dead = 0;
        if (a.dead && (a.shift ? !(d - sft > fmax(1e-9 * sft, 8.0 * k * DBL_EPSILON * (orig[j] + sft)))
                               : !(d > 1e-10 * orig[j]))) {
          pv.dead = 1;
          pv.piv = 1.0;
          a.dead[j] = 1;
        } else if (!(d > 0.0) || !isfinite(d)) {
          pv.piv = 1.0;
          atomicOr(a.err, DEV_CHOL_PIVOT);
        } else {
          pv.piv = sqrt(d);
        }
        // one division per column: on this GPU's narrow fp64 pipe a division
        // by every warp would cost more than the column's update
        pv.inv = 1.0 / pv.piv;
        for (int dst = 0; dst < CC; ++dst) cl.map_shared_rank(pivbuf, dst)[slot] = pv;
      }
    }
    cl.sync();
    // phase B: scale own entries of column j, update own rows
    const Pivot pv = pivbuf[slot];
    const double inv = pv.inv;
    if (j % CC == rank && threadIdx.x == 0) {
      T dv = one_of<T>();
      if (!pv.dead) dv = scalev(one_of<T>(), pv.piv);
      S[tri(j, j)] = dv;
    }
    const int first = j + 1 + ((rank - (j + 1)) % CC + CC) % CC;
    for (int i = first + CC * wp; i < k; i += CC * nw) {
      const T lij = pv.dead ? zero_of(T()) : scalev(S[tri(i, j)], inv);
      __syncwarp();
      if (lane == 0) S[tri(i, j)] = lij;
      if (!pv.dead) {
        const T* cb = colbuf + slot * k;
        T* Si = S + tri(i, 0);
        // S(i, l) -= L(i, j) conj(L(l, j)) = (L(i, j) / piv) conj(G(l, j)),
        // j < l <= i: one complex multiply-add per entry
        const T a = scalev(lij, inv);
        for (int l = j + 1 + lane; l <= i; l += 32) fnmav(Si[l], a, cb[l]);
      }
    }
    __syncthreads();
  }
  // the factor: own rows
  T* L = static_cast<T*>(a.L);
  for (int i = rank + CC * wp; i < k; i += CC * nw)
    for (int l = lane; l < k; l += 32) L[(size_t)i * k + l] = l <= i ? S[tri(i, l)] : zero_of(T());
  if (rank == 0)
    for (int i = threadIdx.x; i < k; i += CT) a.dsc[i] = dsc[i];
  if (a.want_inv) {
    // gather the rows of the other CTAs (all factor entries are final)
    cl.sync();
    for (int i = wp; i < k; i += nw) {
      if (i % CC == rank) continue;
      const T* src = cl.map_shared_rank(S, i % CC) + tri(i, 0);
      T* dst = S + tri(i, 0);
      for (int l = lane; l <= i; l += 32) dst[l] = src[l];
    }
    // every CTA has its copy before any CTA rescales its own rows below
    cl.sync();
    // L' = L diag(1 / L_ll) (rinv kept in orig), so that the substitution
    // below needs no division per step
    double* rinv = orig;
    for (int i = threadIdx.x; i < k; i += CT) rinv[i] = 1.0 / realv(S[tri(i, i)]);
    __syncthreads();
    for (int i = wp; i < k; i += nw) {
      T* Si = S + tri(i, 0);
      for (int l = lane; l <= i; l += 32) Si[l] = scalev(Si[l], rinv[l]);
    }
    __syncthreads();
    // columns c = rank, rank + 8, ... of X = L^-1, right-looking: acc_i =
    // delta_ic - sum_{l < i} L'(i, l) acc_l, x_i = acc_i / L_ii (one warp per
    // column, lanes along i, acc in shared memory), written as
    // W[c][i] = conj(X[i][c]) / D_c
    T* Wm = static_cast<T*>(a.W);
    T* x = xs + (size_t)wp * k;
    for (int c = rank + CC * wp; c < k; c += CC * nw) {
      for (int i = c + lane; i < k; i += 32) x[i] = i == c ? one_of<T>() : zero_of(T());
      __syncwarp();
      for (int l = c; l + 1 < k; ++l) {
        const T al = x[l];
        for (int i = l + 1 + lane; i < k; i += 32) fnmav(x[i], S[tri(i, l)], al);
        __syncwarp();
      }
      const double id = 1.0 / dsc[c];
      T* wrow = Wm + (size_t)c * k;
      for (int i = lane; i < k; i += 32)
        wrow[i] = i >= c ? scalev(conjv(x[i]), rinv[i] * id) : zero_of(T());
      __syncwarp();
    }
  }
  // no CTA leaves while another may still read its shared memory
  cl.sync();
}

// The same factorisation for a k whose packed factor does not fit one CTA:
// each CTA keeps only its own rows (row i = rank + 8 t at offset
// t (rank + 1) + 8 t (t - 1) / 2 of its packed store), and the inverse reads
// the rows of the other CTAs through distributed shared memory instead of
// gathering them.
__device__ __forceinline__ int own_ofs(int i) {
  const int o = i % CC, t = i / CC;
  return t * (o + 1) + CC * t * (t - 1) / 2;
}

template <typename T>
__global__ void __cluster_dims__(CC, 1, 1) __launch_bounds__(CT, 1)
    chol_dist_kernel(CholClusterArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int k = a.k;
  const int nt = (k + CC - 1) / CC;
  const int own_max = CC * nt * (nt + 1) / 2;   // packed entries of the largest share
  extern __shared__ __align__(16) unsigned char smem[];
  T* S = reinterpret_cast<T*>(smem);                        // own rows, packed
  T* colbuf = S + own_max;                                  // [2][k]
  double* dsc = reinterpret_cast<double*>(colbuf + 2 * k);  // [k]
  double* orig = dsc + k;                                   // [k] (then 1 / L_ll)
  T* xs = reinterpret_cast<T*>(orig + k);                   // [CT / 32][k]
  __shared__ Pivot pivbuf[2];
  __shared__ double red[CT / 32];
  __shared__ double sft_s;
  const T* G = static_cast<const T*>(a.G);
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = CT / 32;
  double tr = 0.0;
  for (int i = threadIdx.x; i < k; i += CT) {
    const double d = realv(G[(size_t)i * k + i]);
    const double s = a.scale ? (d > 0.0 ? sqrt(d) : 1.0) : 1.0;
    dsc[i] = s;
    orig[i] = d / (s * s);
    tr += orig[i];
    if (a.dead && i % CC == rank) a.dead[i] = 0;
  }
  tr = warp_sum(tr);
  if (lane == 0) red[wp] = tr;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    sft_s = a.shift ? 11.0 * ((double)a.n * k + (double)k * (k + 1)) * DBL_EPSILON * t : 0.0;
  }
  __syncthreads();
  const double sft = sft_s;
  for (int i = rank + CC * wp; i < k; i += CC * nw) {
    T* Si = S + own_ofs(i);
    for (int l = lane; l <= i; l += 32) {
      T v = scalev(G[(size_t)i * k + l], 1.0 / (dsc[i] * dsc[l]));
      if (l == i) {
        if constexpr (sizeof(T) == 8) v += sft;
        else v.x += sft;
      }
      Si[l] = v;
    }
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    const int slot = j & 1;
    const int first = j + 1 + ((rank - (j + 1)) % CC + CC) % CC;
    {
      const int nown = first < k ? (k - 1 - first) / CC + 1 : 0;
      for (int idx = threadIdx.x; idx < nown * CC; idx += CT) {
        const int i = first + CC * (idx / CC), dst = idx % CC;
        T* cb = cl.map_shared_rank(colbuf, dst);
        cb[slot * k + i] = conjv(S[own_ofs(i) + j]);
      }
      if (j % CC == rank && threadIdx.x == 0) {
        const double d = realv(S[own_ofs(j) + j]);
        Pivot pv;
        pv.pad = 0;
        pv.dead = 0;
        if (a.dead && (a.shift ? !(d - sft > fmax(1e-9 * sft, 8.0 * k * DBL_EPSILON * (orig[j] + sft)))
                               : !(d > 1e-10 * orig[j]))) {
          pv.dead = 1;
          pv.piv = 1.0;
          a.dead[j] = 1;
        } else if (!(d > 0.0) || !isfinite(d)) {
          pv.piv = 1.0;
          atomicOr(a.err, DEV_CHOL_PIVOT);
        } else {
          pv.piv = sqrt(d);
        }
        pv.inv = 1.0 / pv.piv;
        for (int dst = 0; dst < CC; ++dst) cl.map_shared_rank(pivbuf, dst)[slot] = pv;
      }
    }
    cl.sync();
    const Pivot pv = pivbuf[slot];
    const double inv = pv.inv;
    if (j % CC == rank && threadIdx.x == 0) {
      T dv = one_of<T>();
      if (!pv.dead) dv = scalev(one_of<T>(), pv.piv);
      S[own_ofs(j) + j] = dv;
    }
    for (int i = first + CC * wp; i < k; i += CC * nw) {
      T* Si = S + own_ofs(i);
      const T lij = pv.dead ? zero_of(T()) : scalev(Si[j], inv);
      __syncwarp();
      if (lane == 0) Si[j] = lij;
      if (!pv.dead) {
        const T* cb = colbuf + slot * k;
        const T av = scalev(lij, inv);
        for (int l = j + 1 + lane; l <= i; l += 32) fnmav(Si[l], av, cb[l]);
      }
    }
    __syncthreads();
  }
  T* L = static_cast<T*>(a.L);
  for (int i = rank + CC * wp; i < k; i += CC * nw) {
    const T* Si = S + own_ofs(i);
    for (int l = lane; l < k; l += 32) L[(size_t)i * k + l] = l <= i ? Si[l] : zero_of(T());
  }
  if (rank == 0)
    for (int i = threadIdx.x; i < k; i += CT) a.dsc[i] = dsc[i];
  if (a.want_inv) {
    // 1 / L_ll of the own rows into every CTA (orig is free now)
    double* rinv = orig;
    for (int i = rank + CC * threadIdx.x; i < k; i += CC * CT) {
      const double r = 1.0 / realv(S[own_ofs(i) + i]);
      for (int dst = 0; dst < CC; ++dst) cl.map_shared_rank(rinv, dst)[i] = r;
    }
    cl.sync();
    // own rows scaled by column: L' = L diag(1 / L_ll)
    for (int i = rank + CC * wp; i < k; i += CC * nw) {
      T* Si = S + own_ofs(i);
      for (int l = lane; l <= i; l += 32) Si[l] = scalev(Si[l], rinv[l]);
    }
    cl.sync();
    // columns c = rank, rank + 8, ...: right-looking substitution as in the
    // gathering kernel, L'(i, l) read from the CTA that owns row i
    T* Wm = static_cast<T*>(a.W);
    T* x = xs + (size_t)wp * k;
    const T* Sr[CC];
    for (int o = 0; o < CC; ++o) Sr[o] = cl.map_shared_rank(S, o);
    for (int c = rank + CC * wp; c < k; c += CC * nw) {
      for (int i = c + lane; i < k; i += 32) x[i] = i == c ? one_of<T>() : zero_of(T());
      __syncwarp();
      for (int l = c; l + 1 < k; ++l) {
        const T al = x[l];
        for (int i = l + 1 + lane; i < k; i += 32) fnmav(x[i], Sr[i % CC][own_ofs(i) + l], al);
        __syncwarp();
      }
      const double id = 1.0 / dsc[c];
      T* wrow = Wm + (size_t)c * k;
      for (int i = lane; i < k; i += 32)
        wrow[i] = i >= c ? scalev(conjv(x[i]), rinv[i] * id) : zero_of(T());
      __syncwarp();
    }
  }
  // no CTA leaves while another may still read its shared memory
  cl.sync();
}

}  // namespace

size_t chol_cluster_smem(bool cx, int k) {
  const size_t es = cx ? 16 : 8;
  return ((size_t)k * (k + 1) / 2 + 2 * (size_t)k + (size_t)(CT / 32) * k) * es +
         2 * (size_t)k * sizeof(double);
}

size_t chol_dist_smem(bool cx, int k) {
  const size_t es = cx ? 16 : 8;
  const size_t T = (size_t)(k + CC - 1) / CC;
  return (CC * T * (T + 1) / 2 + 2 * (size_t)k + (size_t)(CT / 32) * k) * es +
         2 * (size_t)k * sizeof(double);
}

bool chol_cluster_supported(bool cx, int k) {
  return k >= 1 && (chol_cluster_smem(cx, k) <= (size_t)220 * 1024 ||
                    chol_dist_smem(cx, k) <= (size_t)220 * 1024);
}

cudaError_t chol_cluster(bool cx, int k, long rows, bool shift, bool scale, const void* G,
                         void* L, double* dsc, int* dead, void* W, int* err, cudaStream_t s,
                         long* launches) {
  if (!chol_cluster_supported(cx, k)) return cudaErrorInvalidValue;
  // the gathering kernel where the whole packed factor fits one CTA, else
  // the distributed one
  const bool gather = chol_cluster_smem(cx, k) <= (size_t)220 * 1024;
  const size_t shm = gather ? chol_cluster_smem(cx, k) : chol_dist_smem(cx, k);
  static size_t configured[2][2] = {{0, 0}, {0, 0}};
  const void* fn = gather ? (cx ? (const void*)chol_cluster_kernel<cplx>
                                : (const void*)chol_cluster_kernel<double>)
                          : (cx ? (const void*)chol_dist_kernel<cplx>
                                : (const void*)chol_dist_kernel<double>);
  cudaError_t e = raise_smem(fn, configured[gather ? 0 : 1][cx ? 1 : 0], shm);
  if (e != cudaSuccess) return e;
  CholClusterArgs a;
  a.k = k;
  a.shift = shift ? 1 : 0;
  a.scale = scale ? 1 : 0;
  a.want_inv = W != nullptr;
  a.n = rows;
  a.G = G;
  a.L = L;
  a.W = W;
  a.dsc = dsc;
  a.dead = dead;
  a.err = err;
  if (gather) {
    if (cx) chol_cluster_kernel<cplx><<<CC, CT, shm, s>>>(a);
    else chol_cluster_kernel<double><<<CC, CT, shm, s>>>(a);
  } else {
    if (cx) chol_dist_kernel<cplx><<<CC, CT, shm, s>>>(a);
    else chol_dist_kernel<double><<<CC, CT, shm, s>>>(a);
  }
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace ctm
