// Cooperative small dense fp64 kernels: each k x k matrix of a batch is
// spread over G thread blocks of one cooperative grid.
//
// 1. One-sided Jacobi SVD (Hestenes 1958; Demmel & Veselic 1992).
//
// GB300 has ~6.6 fp64 GFLOP/s per SM, so one block per matrix is bounded by a
// single SM's fp64 units (a 149 x 149 complex sweep is ~1.2e8 flops). Here
// the k/2 disjoint column pairs of each round-robin round are shared by the
// warps of G blocks on G SMs, one pair per warp; columns of A and V live in
// global memory (L2 resident, accessed with .cg loads and stores that bypass
// the incoherent L1). A pair waits only for the two pairs of the previous
// round that wrote its columns (per-column version counters, release /
// acquire), and grid barriers separate the sweeps. Every wait is bounded
// (2 s of %globaltimer); a timeout sets DEV_MBAR_TIMEOUT and a global abort
// flag after which every block leaves.
//
// Result: A = U diag(s) V^H with s descending (ties keep the lower column
// first); exactly-zero columns of U are completed to a unitary by
// Gram-Schmidt against unit vectors.
#include <cfloat>

#include "common.cuh"
#include "kernels.h"

namespace ctm {

namespace {

constexpr int JT = 64;   // threads per block (two warps)

struct JacobiArgs {
  int k, batch, G, max_sweeps, want_uv;
  const void* A;
  long strideA;
  double* s_out;
  void* U;
  void* V;
  const void* Vinit;     // row-major k x k per matrix (V starts here), or null (identity)
  void* work;            // per matrix: 2 k^2 elements (A and V, column-major)
  double* off;           // per matrix: 2 sweep slots (largest rotated ratio
                         // |gamma| / sqrt(alpha beta) of the sweep) and a check slot
  double* norms;         // per matrix: k
  unsigned* ver;         // per matrix: k column versions (rounds applied)
  unsigned* bar;         // [count, generation, abort]
  int* err;
};

__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded grid barrier over all blocks of the launch. bar[0] counts
// arrivals, bar[32] is the generation and bar[64] the abort flag (separate
// 128-byte lines, so that polling does not contend with the arrivals).
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* err) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    unsigned* cnt = bar;
    unsigned* gen = bar + 32;
    unsigned* abrt = bar + 64;
    if (ld_acquire(abrt)) {
      ok = 0;
    } else {
      const unsigned my_gen = ld_acquire(gen);
      __threadfence();   // this block's writes before the arrival
      const unsigned arrived = atomicAdd(cnt, 1u) + 1u;
      if (arrived == nblocks) {
        atomicExch(cnt, 0u);
        __threadfence();
        atomicAdd(gen, 1u);
      } else {
        const uint64_t t0 = gtime();
        unsigned polls = 0;
        while (ld_acquire(gen) == my_gen) {
          if ((++polls & 63u) == 0 && (ld_acquire(abrt) || gtime() - t0 > 2000000000ull)) {
            atomicExch(abrt, 1u);
            atomicOr(err, DEV_MBAR_TIMEOUT);
            ok = 0;
            break;
          }
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p);
template <>
__device__ __forceinline__ double ldcg<double>(const double* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ cplx ldcg<cplx>(const cplx* p) { return __ldcg(p); }
template <typename T>
__device__ __forceinline__ void stcg(T* p, T v);
template <>
__device__ __forceinline__ void stcg<double>(double* p, double v) { __stcg(p, v); }
template <>
__device__ __forceinline__ void stcg<cplx>(cplx* p, cplx v) { __stcg(p, v); }

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// the warp waits until columns p and q (q < 0: none) have been through
// round r; every lane polls with acquire loads, so each lane's later reads of
// the columns are ordered after the release that published them. Bounded
// like the grid barrier (abort flag, 2 s, decided by lane 0). Returns false
// on abort.
__device__ bool wait_columns(const unsigned* ver, int p, int q, unsigned r, unsigned* bar,
                             int* err, int lane) {
  unsigned* abrt = bar + 64;
  const uint64_t t0 = gtime();
  unsigned polls = 0;
  while (true) {
    const bool ready = ld_acquire(ver + p) == r && (q < 0 || ld_acquire(ver + q) == r);
    if (__all_sync(0xffffffffu, ready)) return true;
    int stop = 0;
    if (lane == 0 && (++polls & 63u) == 0 && (ld_acquire(abrt) || gtime() - t0 > 2000000000ull)) {
      atomicExch(abrt, 1u);
      atomicOr(err, DEV_MBAR_TIMEOUT);
      stop = 1;
    }
    if (__shfl_sync(0xffffffffu, stop, 0)) return false;
  }
}

__device__ __forceinline__ int player(int pos, int t, int m) {
  return pos == 0 ? 0 : ((pos - 1 + t) % m) + 1;
}

// (x, y) -> (c x - se y, s x + ce y) with se = s eph and ce = c eph folded
// once per pair: 12 fp64 operations per complex element pair instead of 16
// (the fp64 pipe bounds a rotation on this GPU)
__device__ __forceinline__ double rot_lo(double x, double y, double c, double se) {
  return fma(-se, y, c * x);
}
__device__ __forceinline__ double rot_hi(double x, double y, double s, double ce) {
  return fma(ce, y, s * x);
}
__device__ __forceinline__ cplx rot_lo(cplx x, cplx y, double c, cplx se) {
  return make_double2(fma(-se.x, y.x, fma(se.y, y.y, c * x.x)),
                      fma(-se.x, y.y, fma(-se.y, y.x, c * x.y)));
}
__device__ __forceinline__ cplx rot_hi(cplx x, cplx y, double s, cplx ce) {
  return make_double2(fma(ce.x, y.x, fma(-ce.y, y.y, s * x.x)),
                      fma(ce.x, y.y, fma(ce.y, y.x, s * x.y)));
}

template <typename T, int R>
__global__ void __launch_bounds__(JT) jacobi_coop(JacobiArgs a) {
  // R: elements of a column held per lane (k <= 32 R); the pair's columns
  // stay in registers between the dot product and the rotation, and the
  // squared column norms are kept in nsq (exact at the start of each sweep,
  // updated by alpha' = alpha - t |gamma|, beta' = beta + t |gamma|)
  const int k = a.k, G = a.G;
  const int b = blockIdx.x / G, g = blockIdx.x % G;
  const unsigned nblocks = gridDim.x;
  T* wa = static_cast<T*>(a.work) + (size_t)b * 2 * k * k;   // column c at wa[c*k]
  T* wv = wa + (size_t)k * k;
  double* nsq = a.norms + (size_t)b * k;
  const T* Ab = static_cast<const T*>(a.A) + (size_t)b * a.strideA;
  const T* Vi = a.Vinit ? static_cast<const T*>(a.Vinit) + (size_t)b * k * k : nullptr;
  const T one = [] {
    if constexpr (sizeof(T) == 8) return T(1.0);
    else return make_double2(1.0, 0.0);
  }();
  for (long idx = (long)g * JT + threadIdx.x; idx < (long)k * k; idx += (long)G * JT) {
    const int r = (int)(idx / k), c = (int)(idx % k);
    stcg(wa + (size_t)c * k + r, Ab[idx]);
    if (a.want_uv)
      stcg(wv + (size_t)c * k + r, Vi ? Vi[idx] : ((r == c) ? one : zero_of(T())));
  }
  unsigned* ver = a.ver + (size_t)b * k;
  for (int c = g * JT + threadIdx.x; c < k; c += G * JT) ver[c] = 0u;
  if (g == 0 && threadIdx.x == 0) {
    a.off[3 * b] = 0.0;
    a.off[3 * b + 1] = 0.0;
    a.off[3 * b + 2] = 0.0;
  }
  if (!grid_barrier(a.bar, nblocks, a.err)) return;
  const double tol = fmax(1.0, (double)k) * DBL_EPSILON;
  const int kk = k + (k & 1), m = kk - 1, npairs = kk / 2;
  const int lane = threadIdx.x & 31;
  const int gw = g * (JT / 32) + (threadIdx.x >> 5), nw = G * (JT / 32);
  int sweep = 0;
  bool converged = false;
  for (; sweep < a.max_sweeps; ++sweep) {
    // exact squared norms at the start of the sweep (one warp per column)
    for (int c = gw; c < k; c += nw) {
      double acc = 0.0;
      for (int r = lane; r < k; r += 32) acc += absq(ldcg(wa + (size_t)c * k + r));
      acc = warp_sum(acc);
      if (lane == 0) __stcg(nsq + c, acc);
    }
    if (!grid_barrier(a.bar, nblocks, a.err)) return;
    // every block read the previous sweep's flag before this barrier: clear
    // the slot of the next sweep
    if (g == 0 && threadIdx.x == 0) {
      a.off[3 * b + ((sweep + 1) & 1)] = 0.0;
      a.off[3 * b + 2] = 0.0;
    }
    // the largest ratio |gamma| / sqrt(alpha beta) of the pairs rotated in
    // this sweep (non-negative doubles order like their bit patterns)
    unsigned long long* offb =
        reinterpret_cast<unsigned long long*>(a.off + 3 * b + (sweep & 1));
    // rounds without grid barriers: a pair waits only for the two pairs of
    // the previous round that wrote its columns (column versions), so the
    // rotations are the same as with a barrier per round
    bool dead = false;
    for (int t = 0; t < m; ++t) {
      const unsigned rg = (unsigned)(sweep * m + t);
      for (int pr = gw; pr < npairs; pr += nw) {
        int p = player(pr, t, m), q = player(kk - 1 - pr, t, m);
        if (p > q) { const int tmp = p; p = q; q = tmp; }
        const bool real = q < k;
        if (!dead) dead = !wait_columns(ver, p, real ? q : -1, rg, a.bar, a.err, lane);
        if (!dead && real) {
          T* ap = wa + (size_t)p * k;
          T* aq = wa + (size_t)q * k;
          T xr[R], yr[R];
          // V's columns are fetched with A's (independent loads) when they
          // fit in registers
          constexpr bool kPrefetchV = R <= 9;
          T vxr[kPrefetchV ? R : 1], vyr[kPrefetchV ? R : 1];
          T* vp = wv + (size_t)p * k;
          T* vq = wv + (size_t)q * k;
          T ga = zero_of(T());
#pragma unroll
          for (int e = 0; e < R; ++e) {
            const int r = lane + 32 * e;
            if (r < k) {
              xr[e] = ldcg(ap + r);
              yr[e] = ldcg(aq + r);
              if constexpr (kPrefetchV) {
                if (a.want_uv) {
                  vxr[e] = ldcg(vp + r);
                  vyr[e] = ldcg(vq + r);
                }
              }
            }
          }
#pragma unroll
          for (int e = 0; e < R; ++e)
            if (lane + 32 * e < k) fmacv(ga, xr[e], yr[e]);
          ga = warp_sum(ga);
          const double al = __ldcg(nsq + p), be = __ldcg(nsq + q);
          // the rotation's scalars on lane 0 only, then broadcast: every
          // fp64 instruction a whole warp executes costs the SM's narrow fp64
          // pipe its full width
          double gm = 0.0, tt = 0.0, c = 1.0, s = 0.0, ex = 0.0, ey = 0.0;
          int rot = 0;
          if (lane == 0) {
            gm = sqrt(absq(ga));
            const double nrm = sqrt(al) * sqrt(be);
            // rotate when |gamma| > tol sqrt(alpha beta)
            rot = gm > tol * nrm && gm != 0.0;
            if (rot) {
              atomicMax(offb, (unsigned long long)__double_as_longlong(
                                  nrm > 0.0 ? fmin(gm / nrm, 1.0) : 1.0));   // this sweep rotated
              const double zeta = (be - al) / (2.0 * gm);
              tt = copysign(1.0, zeta) / (fabs(zeta) + hypot(1.0, zeta));
              c = 1.0 / hypot(1.0, tt);
              s = c * tt;
              // conj(gamma) / |gamma|
              const double ig = 1.0 / gm;
              if constexpr (sizeof(T) == 8) {
                ex = ga * ig;
              } else {
                ex = ga.x * ig;
                ey = -ga.y * ig;
              }
            }
          }
          rot = __shfl_sync(0xffffffffu, rot, 0);
          if (rot) {
            gm = __shfl_sync(0xffffffffu, gm, 0);
            tt = __shfl_sync(0xffffffffu, tt, 0);
            c = __shfl_sync(0xffffffffu, c, 0);
            s = __shfl_sync(0xffffffffu, s, 0);
            ex = __shfl_sync(0xffffffffu, ex, 0);
            if constexpr (sizeof(T) == 16) ey = __shfl_sync(0xffffffffu, ey, 0);
            T eph;
            if constexpr (sizeof(T) == 8) eph = ex;
            else eph = make_double2(ex, ey);
            const T se = scalev(eph, s), ce = scalev(eph, c);
#pragma unroll
            for (int e = 0; e < R; ++e) {
              const int r = lane + 32 * e;
              if (r < k) {
                stcg(ap + r, rot_lo(xr[e], yr[e], c, se));
                stcg(aq + r, rot_hi(xr[e], yr[e], s, ce));
              }
            }
            if (lane == 0) {
              __stcg(nsq + p, al - tt * gm);
              __stcg(nsq + q, be + tt * gm);
            }
            if (a.want_uv) {
#pragma unroll
              for (int e = 0; e < R; ++e) {
                const int r = lane + 32 * e;
                if (r < k) {
                  T x, y;
                  if constexpr (kPrefetchV) {
                    x = vxr[e];
                    y = vyr[e];
                  } else {
                    x = ldcg(vp + r);
                    y = ldcg(vq + r);
                  }
                  stcg(vp + r, rot_lo(x, y, c, se));
                  stcg(vq + r, rot_hi(x, y, s, ce));
                }
              }
            }
          }
        }
        // publish: columns p and q have been through round rg
        __syncwarp();
        if (lane == 0 && !dead) {
          __threadfence();
          st_release(ver + p, rg + 1u);
          if (real) st_release(ver + q, rg + 1u);
        }
      }
    }
    if (!grid_barrier(a.bar, nblocks, a.err)) return;
    // convergence of the whole batch: every block reads every flag
    bool all = true;
    double mxr = 0.0;
    for (int bb = 0; bb < a.batch; ++bb) {
      const double r = __ldcg(a.off + 3 * bb + (sweep & 1));
      all = all && (r <= tol);
      mxr = fmax(mxr, r);
    }
    if (!all && mxr < 1e-6 && sweep + 1 < a.max_sweeps) {
      // quadratic regime: the next sweep most likely rotates nothing. Its
      // decision is taken here at once, from every pair's exact ratio on the
      // current columns (the dot products such a sweep would compute before
      // any rotation), in parallel instead of round by round
      for (int c = gw; c < k; c += nw) {
        double acc = 0.0;
        for (int r = lane; r < k; r += 32) acc += absq(ldcg(wa + (size_t)c * k + r));
        acc = warp_sum(acc);
        if (lane == 0) __stcg(nsq + c, acc);
      }
      if (!grid_barrier(a.bar, nblocks, a.err)) return;
      double* chk = a.off + 3 * b + 2;
      // fold f holds the columns f and k - 2 - f: k - 1 pairs (p, q > p) each
      for (int f = gw; 2 * f <= k - 2; f += nw) {
        for (int side = 0; side < 2; ++side) {
          const int p = side == 0 ? f : k - 2 - f;
          if (side == 1 && p == f) break;
          T xr[R];
#pragma unroll
          for (int e = 0; e < R; ++e) {
            const int r = lane + 32 * e;
            xr[e] = r < k ? ldcg(wa + (size_t)p * k + r) : zero_of(T());
          }
          const double np_ = __ldcg(nsq + p);
          bool bad = false;
          for (int q = p + 1; q < k && !bad; ++q) {
            const T* aq = wa + (size_t)q * k;
            T ga = zero_of(T());
#pragma unroll
            for (int e = 0; e < R; ++e) {
              const int r = lane + 32 * e;
              if (r < k) fmacv(ga, xr[e], ldcg(aq + r));
            }
            ga = warp_sum(ga);
            bad = absq(ga) > tol * tol * np_ * __ldcg(nsq + q) && absq(ga) != 0.0;
          }
          if (bad) {
            if (lane == 0) __stcg(chk, 1.0);
            break;
          }
        }
      }
      if (!grid_barrier(a.bar, nblocks, a.err)) return;
      bool pass = true;
      for (int bb = 0; bb < a.batch; ++bb) pass = pass && __ldcg(a.off + 3 * bb + 2) == 0.0;
      if (pass) {
        converged = true;
        ++sweep;
        break;
      }
    }
    if (all) {
      converged = true;
      ++sweep;
      break;
    }
  }
  if (!converged && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.err, DEV_JACOBI_NOCONV);
  // singular values: column norms (one warp per column)
  double* nb = a.norms + (size_t)b * k;
  for (int c = gw; c < k; c += nw) {
    double acc = 0.0;
    for (int r = lane; r < k; r += 32) acc += absq(ldcg(wa + (size_t)c * k + r));
    acc = warp_sum(acc);
    if (lane == 0) __stcg(nb + c, sqrt(acc));
  }
  if (!grid_barrier(a.bar, nblocks, a.err)) return;
  // descending order, ties to the lower index; write s, U, V
  for (int c = g * JT + threadIdx.x; c < k; c += G * JT) {
    const double x = __ldcg(nb + c);
    int rk = 0;
    for (int j = 0; j < k; ++j) {
      const double y = __ldcg(nb + j);
      rk += (y > x) || (y == x && j < c);
    }
    a.s_out[(size_t)b * k + rk] = x;
    if (!isfinite(x)) atomicOr(a.err, DEV_NONFINITE);
    if (a.want_uv) {
      T* Ub = static_cast<T*>(a.U) + (size_t)b * k * k;
      T* Vb = static_cast<T*>(a.V) + (size_t)b * k * k;
      for (int r = 0; r < k; ++r) {
        const T xv = ldcg(wa + (size_t)c * k + r);
        stcg(Ub + (size_t)r * k + rk, x > 0.0 ? scalev(xv, 1.0 / x) : zero_of(T()));
        stcg(Vb + (size_t)r * k + rk, ldcg(wv + (size_t)c * k + r));
      }
    }
  }
  if (!a.want_uv) return;
  if (!grid_barrier(a.bar, nblocks, a.err)) return;
  // completion of exactly-zero columns of U (block 0 of the matrix, warp 0)
  if (g != 0 || threadIdx.x >= 32) return;
  int nzero = 0;
  for (int c = 0; c < k; ++c) nzero += (__ldcg(nb + c) == 0.0);
  if (nzero == 0) return;
  T* Ub = static_cast<T*>(a.U) + (size_t)b * k * k;
  T* tmp = wa;
  int cand = 0;
  for (int col = k - nzero; col < k; ++col) {
    for (; cand < k; ++cand) {
      for (int r = lane; r < k; r += 32) stcg(tmp + r, (r == cand) ? one : zero_of(T()));
      __syncwarp();
      for (int rep = 0; rep < 2; ++rep) {
        for (int j = 0; j < col; ++j) {
          T dd = zero_of(T());
          for (int r = lane; r < k; r += 32) fmacv(dd, ldcg(Ub + (size_t)r * k + j), ldcg(tmp + r));
          dd = warp_sum(dd);
          __syncwarp();
          for (int r = lane; r < k; r += 32)
            stcg(tmp + r, subv(ldcg(tmp + r), mulv(ldcg(Ub + (size_t)r * k + j), dd)));
          __syncwarp();
        }
      }
      double nn = 0.0;
      for (int r = lane; r < k; r += 32) nn += absq(ldcg(tmp + r));
      nn = warp_sum(nn);
      if (nn > 0.25) {
        const double inv = 1.0 / sqrt(nn);
        for (int r = lane; r < k; r += 32) stcg(Ub + (size_t)r * k + col, scalev(ldcg(tmp + r), inv));
        __syncwarp();
        ++cand;
        break;
      }
    }
  }
}

// ------------------------------------------------------------------------
// 2. Blocked right-looking Cholesky G = L L^H (optionally shifted, with the
// dead-column detection of CholeskyQR) and the triangular inverse L^-1.
// Panels of CB columns are factored by block 0 of the matrix; the trailing
// update is shared by all G blocks; grid barriers separate the phases; the
// inverse is column-parallel.
constexpr int CB = 16;

struct CholArgs {
  int k, batch, G, shift, detect, scale;
  long n;             // rows of the block whose Gram this is (for the shift)
  void* Gm;           // [batch][k][k], overwritten by L
  void* Linv;         // [batch][k][k]
  int* dead;          // [batch][k] or null
  double* aux;        // [batch][2k + 2]: original diagonal, shift, bad, scales
  unsigned* bar;
  int* err;
};

template <typename T>
__global__ void __launch_bounds__(JT) chol_coop(CholArgs a) {
  const int k = a.k, G = a.G;
  const int b = blockIdx.x / G, g = blockIdx.x % G;
  const unsigned nblocks = gridDim.x;
  T* L = static_cast<T*>(a.Gm) + (size_t)b * k * k;
  T* Li = static_cast<T*>(a.Linv) + (size_t)b * k * k;
  double* orig = a.aux + (size_t)b * (2 * k + 2);
  double* sft_p = orig + k;
  double* bad_p = orig + k + 1;
  double* dsc = orig + k + 2;      // column scales (Jacobi preconditioning)
  int* dead = a.dead ? a.dead + (size_t)b * k : nullptr;
  __shared__ double red[JT / 32];
  __shared__ double piv;
  __shared__ int isdead;
  // optional symmetric diagonal scaling G <- D^-1 G D^-1 (D_i = sqrt(G_ii)),
  // undone on L^-1 at the end; then diagonal and shift
  if (a.scale) {
    for (int i = g * JT + threadIdx.x; i < k; i += G * JT) {
      const double d = realv(ldcg(L + (size_t)i * k + i));
      __stcg(dsc + i, d > 0.0 ? sqrt(d) : 1.0);
    }
    if (!grid_barrier(a.bar, nblocks, a.err)) return;
    for (long idx = (long)g * JT + threadIdx.x; idx < (long)k * k; idx += (long)G * JT) {
      const int i = (int)(idx / k), l = (int)(idx % k);
      stcg(L + idx, scalev(ldcg(L + idx), 1.0 / (__ldcg(dsc + i) * __ldcg(dsc + l))));
    }
    if (!grid_barrier(a.bar, nblocks, a.err)) return;
  }
  if (g == 0) {
    double tr = 0.0;
    for (int i = threadIdx.x; i < k; i += JT) {
      const double d = realv(ldcg(L + (size_t)i * k + i));
      __stcg(orig + i, d);
      tr += d;
      if (dead) dead[i] = 0;
    }
    tr = warp_sum(tr);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tr;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < JT / 32; ++w) t += red[w];
      const double sft =
          a.shift ? 11.0 * ((double)a.n * k + (double)k * (k + 1)) * DBL_EPSILON * t : 0.0;
      __stcg(sft_p, sft);
      __stcg(bad_p, 0.0);
    }
    __syncthreads();
    const double sft = __ldcg(sft_p);
    if (sft != 0.0)
      for (int i = threadIdx.x; i < k; i += JT) {
        T v = ldcg(L + (size_t)i * k + i);
        if constexpr (sizeof(T) == 8) v += sft;
        else v.x += sft;
        stcg(L + (size_t)i * k + i, v);
      }
  }
  if (!grid_barrier(a.bar, nblocks, a.err)) return;
  const double sft = __ldcg(sft_p);
  for (int j0 = 0; j0 < k; j0 += CB) {
    const int jb = min(CB, k - j0);
    if (g == 0) {
      // unblocked factorisation of the panel L[j0:k, j0:j0+jb]
      for (int j = j0; j < j0 + jb; ++j) {
        if (threadIdx.x == 0) {
          const double d = realv(ldcg(L + (size_t)j * k + j));
          const double o = __ldcg(orig + j);
          isdead = 0;
          if (dead && (a.shift ? !(d - sft > fmax(1e-9 * sft, 8.0 * k * DBL_EPSILON * (o + sft)))
                               : !(d > 1e-10 * o))) {
            isdead = 1;
            piv = 1.0;
            dead[j] = 1;
          } else if (!(d > 0.0) || !isfinite(d)) {
            piv = 1.0;
            __stcg(bad_p, 1.0);
            atomicOr(a.err, DEV_CHOL_PIVOT);
          } else {
            piv = sqrt(d);
          }
        }
        __syncthreads();
        const double inv = 1.0 / piv;
        for (int i = j + 1 + threadIdx.x; i < k; i += JT) {
          const T v = ldcg(L + (size_t)i * k + j);
          stcg(L + (size_t)i * k + j, isdead ? zero_of(T()) : scalev(v, inv));
        }
        if (threadIdx.x == 0) {
          T dv;
          if constexpr (sizeof(T) == 8) dv = isdead ? 1.0 : piv;
          else dv = make_double2(isdead ? 1.0 : piv, 0.0);
          stcg(L + (size_t)j * k + j, dv);
        }
        __threadfence_block();
        __syncthreads();
        // update the rest of the panel: columns j+1 .. j0+jb-1, rows >= col
        if (!isdead) {
          const int nc = j0 + jb - (j + 1);
          const int nr = k - (j + 1);
          for (long idx = threadIdx.x; idx < (long)nc * nr; idx += JT) {
            const int l = j + 1 + (int)(idx % nc), i = j + 1 + (int)(idx / nc);
            if (i < l) continue;
            T v = ldcg(L + (size_t)i * k + l);
            v = subv(v, mulv(ldcg(L + (size_t)i * k + j), conjv(ldcg(L + (size_t)l * k + j))));
            stcg(L + (size_t)i * k + l, v);
          }
        }
        __threadfence_block();
        __syncthreads();
      }
    }
    if (!grid_barrier(a.bar, nblocks, a.err)) return;
    // trailing update of L[j0+jb:k, j0+jb:k] (lower triangle) by all blocks
    const int t0 = j0 + jb, m = k - t0;
    if (m > 0) {
      for (long idx = (long)g * JT + threadIdx.x; idx < (long)m * m; idx += (long)G * JT) {
        const int i = t0 + (int)(idx / m), l = t0 + (int)(idx % m);
        if (i < l) continue;
        T v = ldcg(L + (size_t)i * k + l);
        for (int c = j0; c < j0 + jb; ++c)
          v = subv(v, mulv(ldcg(L + (size_t)i * k + c), conjv(ldcg(L + (size_t)l * k + c))));
        stcg(L + (size_t)i * k + l, v);
      }
    }
    if (!grid_barrier(a.bar, nblocks, a.err)) return;
  }
  const bool bad = __ldcg(bad_p) != 0.0;
  // inverse: one column of L^-1 per thread (forward substitution)
  for (int c = g * JT + threadIdx.x; c < k; c += G * JT) {
    for (int i = 0; i < k; ++i) {
      T v = zero_of(T());
      if (bad) {
        if (i == c) {
          if constexpr (sizeof(T) == 8) v = 1.0;
          else v = make_double2(1.0, 0.0);
        }
      } else if (i >= c) {
        if (i == c) {
          if constexpr (sizeof(T) == 8) v = 1.0;
          else v = make_double2(1.0, 0.0);
        }
        for (int j = c; j < i; ++j)
          v = subv(v, mulv(ldcg(L + (size_t)i * k + j), ldcg(Li + (size_t)j * k + c)));
        v = scalev(v, 1.0 / realv(ldcg(L + (size_t)i * k + i)));
      }
      stcg(Li + (size_t)i * k + c, v);
    }
  }
  if (!a.scale) return;
  // with scaling, Q = Z D^-1 L_s^-H = Z (L_s^-1 D^-1)^H: scale column c of
  // L^-1 by 1 / D_c (after every column of L^-1 is complete)
  if (!grid_barrier(a.bar, nblocks, a.err)) return;
  for (long idx = (long)g * JT + threadIdx.x; idx < (long)k * k; idx += (long)G * JT) {
    const int c = (int)(idx % k);
    stcg(Li + idx, scalev(ldcg(Li + idx), 1.0 / __ldcg(dsc + c)));
  }
}

}  // namespace

// aux block, then the grid-barrier words (count, generation and abort flag at
// word offsets 0, 32 and 64, see grid_barrier) after a 16-byte alignment
size_t chol_coop_work_bytes(int k, int batch) {
  return (size_t)batch * (2 * k + 2) * sizeof(double) + 16 + 65 * sizeof(unsigned);
}

cudaError_t chol_inv_coop(bool cx, int k, long n, bool shift, bool scale, void* Gm, void* Linv,
                          int batch, int* dead, void* work, int* err, int max_blocks,
                          cudaStream_t s, long* launches) {
  int G = (k * k / 2 + JT * 8 - 1) / (JT * 8);
  int cap = max_blocks / (batch > 0 ? batch : 1);
  if (cap < 1) cap = 1;
  if (G > cap) G = cap;
  if (G > 48) G = 48;
  if (G < 1) G = 1;
  CholArgs a;
  a.k = k;
  a.batch = batch;
  a.G = G;
  a.shift = shift ? 1 : 0;
  a.detect = dead ? 1 : 0;
  a.scale = scale ? 1 : 0;
  a.n = n;
  a.Gm = Gm;
  a.Linv = Linv;
  a.dead = dead;
  char* w = static_cast<char*>(work);
  a.aux = reinterpret_cast<double*>(w);
  w += (size_t)batch * (2 * k + 2) * sizeof(double);
  a.bar = reinterpret_cast<unsigned*>((reinterpret_cast<uintptr_t>(w) + 15) & ~(uintptr_t)15);
  a.err = err;
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 65 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  const void* fn = cx ? (const void*)chol_coop<cplx> : (const void*)chol_coop<double>;
  e = cudaLaunchCooperativeKernel(fn, dim3(batch * G), dim3(JT), args, 0, s);
  if (launches) ++*launches;
  return e;
}

size_t jacobi_coop_work_bytes(bool cx, int k, int batch) {
  const size_t es = cx ? 16 : 8;
  return (size_t)batch * 2 * k * k * es + (size_t)batch * (3 + k) * sizeof(double) +
         (size_t)batch * k * sizeof(unsigned) + 16 + 65 * sizeof(unsigned);
}

cudaError_t jacobi_svd_coop(bool cx, int k, const void* A, long strideA, double* sv, void* U,
                            void* V, bool want_uv, void* work, int batch, int max_sweeps,
                            int* err, int max_blocks, cudaStream_t s, long* launches,
                            const void* Vinit) {
  const size_t es = cx ? 16 : 8;
  const int kk = k + (k & 1);
  const int npairs = kk / 2;
  const void* fn;
  if (k <= 32 * 5)
    fn = cx ? (const void*)jacobi_coop<cplx, 5> : (const void*)jacobi_coop<double, 5>;
  else if (k <= 32 * 9)
    fn = cx ? (const void*)jacobi_coop<cplx, 9> : (const void*)jacobi_coop<double, 9>;
  else if (k <= 32 * 16)
    fn = cx ? (const void*)jacobi_coop<cplx, 16> : (const void*)jacobi_coop<double, 16>;
  else
    return cudaErrorInvalidValue;
  // one column pair per warp when the co-resident blocks allow it: several
  // small blocks per SM (max_blocks counts SMs), shared by the batch
  int per_sm = 1;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, JT, 0);
  if (e != cudaSuccess) return e;
  if (per_sm > 8) per_sm = 8;
  if (per_sm < 1) per_sm = 1;
  int G = (npairs + (JT / 32) - 1) / (JT / 32);
  int cap = max_blocks * per_sm / (batch > 0 ? batch : 1);
  if (cap < 1) cap = 1;
  if (G > cap) G = cap;
  if (G < 1) G = 1;
  JacobiArgs a;
  a.k = k;
  a.batch = batch;
  a.G = G;
  a.max_sweeps = max_sweeps;
  a.want_uv = want_uv ? 1 : 0;
  a.A = A;
  a.strideA = strideA;
  a.s_out = sv;
  a.U = U;
  a.V = V;
  char* w = static_cast<char*>(work);
  a.work = w;
  w += (size_t)batch * 2 * k * k * es;
  a.Vinit = want_uv ? Vinit : nullptr;
  a.off = reinterpret_cast<double*>(w);
  w += (size_t)batch * 3 * sizeof(double);
  a.norms = reinterpret_cast<double*>(w);
  w += (size_t)batch * k * sizeof(double);
  a.ver = reinterpret_cast<unsigned*>(w);
  w += (size_t)batch * k * sizeof(unsigned);
  a.bar = reinterpret_cast<unsigned*>((reinterpret_cast<uintptr_t>(w) + 15) & ~(uintptr_t)15);
  a.err = err;
  e = cudaMemsetAsync(a.bar, 0, 65 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel(fn, dim3(batch * G), dim3(JT), args, 0, s);
  if (launches) ++*launches;
  return e;
}

}  // namespace ctm
