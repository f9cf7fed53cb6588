// Small dense FP64 linear algebra of the projector construction, one thread
// block per matrix (batched over the cuts of a column):
//   * Cholesky factor and triangular inverse of a k x k Gram matrix, the core
//     of (shifted) CholeskyQR (Fukaya, Kannan, Nakatsukasa, Yamamoto,
//     Yanagisawa 2020) that re-orthonormalises the rangefinders;
//   * one-sided Jacobi SVD (Hestenes 1958; Demmel & Veselic 1992) of the
//     (chi+p) x (chi+p) matrix rho and of the corners, with round-robin pair
//     ordering and a bounded number of sweeps;
//   * the phase fix of singular vectors, s^-1/2 with cutoff, normalisation
//     and the corner-spectrum convergence measure.
#include <cfloat>

#include "common.cuh"
#include "kernels.h"

namespace ctm {

namespace {

__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------ Cholesky
template <typename T>
__global__ void __launch_bounds__(256) chol_inv_kernel(int k, long n, int shift,
                                                       T* G, T* Linv, int* dead,
                                                       int* err) {
  T* g = G + (long)blockIdx.x * k * k;
  T* L = Linv + (long)blockIdx.x * k * k;
  __shared__ double sh[32];
  __shared__ double piv;
  __shared__ int bad, isdead;
  extern __shared__ double orig[];      // k original diagonal entries
  if (threadIdx.x == 0) bad = 0;
  double sft = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    orig[i] = realv(g[(long)i * k + i]);
    if (dead) dead[(long)blockIdx.x * k + i] = 0;
  }
  if (shift) {
    double tr = 0.0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) tr += realv(g[(long)i * k + i]);
    tr = block_sum(tr, sh);
    sft = 11.0 * ((double)n * k + (double)k * (k + 1)) * DBL_EPSILON * tr;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      const double re = realv(g[(long)i * k + i]) + sft;
      if constexpr (sizeof(T) == 8) g[(long)i * k + i] = re;
      else g[(long)i * k + i] = make_double2(re, 0.0);
    }
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      const double d = realv(g[(long)j * k + j]);
      isdead = 0;
      // dead-column detection. Shifted pass: a column whose residual (pivot
      // minus the shift) is below 1e-9 of the shift leaves the pass with a
      // norm below ~3e-5 made of rounding noise; plain pass: a pivot below
      // 1e-10 of the column's own squared norm. Either column lies
      // numerically in the span of the previous ones.
      const bool is_dead =
          dead && (shift ? !(d - sft > fmax(1e-9 * sft, 8.0 * k * DBL_EPSILON * (orig[j] + sft)))
                         : !(d > 1e-10 * orig[j]));
      if (is_dead) {
        isdead = 1;
        piv = 1.0;
      } else if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
        piv = 1.0;
      } else {
        piv = sqrt(d);
      }
    }
    __syncthreads();
    if (bad) break;
    if (isdead) {
      // unit column of L: the column is excluded from the elimination and
      // replaced by a fresh direction after the product with L^-H
      for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) g[(long)i * k + j] = zero_of(T());
      if (threadIdx.x == 0) {
        if constexpr (sizeof(T) == 8) g[(long)j * k + j] = 1.0;
        else g[(long)j * k + j] = make_double2(1.0, 0.0);
        dead[(long)blockIdx.x * k + j] = 1;
      }
      __syncthreads();
      continue;
    }
    const double dj = piv, inv = 1.0 / piv;
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x)
      g[(long)i * k + j] = scalev(g[(long)i * k + j], inv);
    if (threadIdx.x == 0) {
      if constexpr (sizeof(T) == 8) g[(long)j * k + j] = dj;
      else g[(long)j * k + j] = make_double2(dj, 0.0);
    }
    __syncthreads();
    const int m = k - j - 1;
    for (long idx = threadIdx.x; idx < (long)m * m; idx += blockDim.x) {
      const int i = j + 1 + (int)(idx / m), l = j + 1 + (int)(idx % m);
      if (l > i) continue;
      // G_il -= L_ij conj(L_lj)
      T v = g[(long)i * k + l];
      T lij = g[(long)i * k + j], llj = g[(long)l * k + j];
      v = subv(v, mulv(lij, conjv(llj)));
      g[(long)i * k + l] = v;
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) atomicOr(err, DEV_CHOL_PIVOT);
    // leave an identity inverse so that downstream products stay finite
    for (long idx = threadIdx.x; idx < (long)k * k; idx += blockDim.x) {
      const int i = (int)(idx / k), c = (int)(idx % k);
      T v = zero_of(T());
      if (i == c) {
        if constexpr (sizeof(T) == 8) v = 1.0;
        else v = make_double2(1.0, 0.0);
      }
      L[idx] = v;
    }
    return;
  }
  // forward substitution, one column of L^-1 per thread
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int i = 0; i < k; ++i) {
      T v = zero_of(T());
      if (i >= c) {
        if (i == c) {
          if constexpr (sizeof(T) == 8) v = 1.0;
          else v = make_double2(1.0, 0.0);
        }
        for (int j = c; j < i; ++j) v = subv(v, mulv(g[(long)i * k + j], L[(long)j * k + c]));
        v = scalev(v, 1.0 / realv(g[(long)i * k + i]));
      }
      L[(long)i * k + c] = v;
    }
  }
}

// --------------------------------------------------------------- Jacobi
template <typename T>
__device__ __forceinline__ T phase_of(T g, double mag);
template <>
__device__ __forceinline__ double phase_of<double>(double g, double mag) { return g / mag; }
template <>
__device__ __forceinline__ cplx phase_of<cplx>(cplx g, double mag) {
  return make_double2(g.x / mag, -g.y / mag);  // conj(g) / |g|
}

__device__ __forceinline__ int rr_player(int pos, int t, int m) {
  // circle method: position 0 fixed, the others rotate
  return pos == 0 ? 0 : ((pos - 1 + t) % m) + 1;
}

template <typename T>
__global__ void __launch_bounds__(512) jacobi_kernel(int k, const T* A, long strideA,
                                                     double* s_out, T* U, T* V,
                                                     int want_uv, T* work,
                                                     int max_sweeps, int* err) {
  const int b = blockIdx.x;
  T* a = work + (long)b * 2 * k * k;   // column c of A at a[c*k .. c*k+k)
  T* v = a + (long)k * k;              // column c of V
  const T* Ab = A + b * strideA;
  const T one = [] {
    if constexpr (sizeof(T) == 8) return T(1.0);
    else return make_double2(1.0, 0.0);
  }();
  for (long idx = threadIdx.x; idx < (long)k * k; idx += blockDim.x) {
    const int r = (int)(idx / k), c = (int)(idx % k);
    a[(long)c * k + r] = Ab[idx];
    if (want_uv) v[(long)c * k + r] = (r == c) ? one : zero_of(T());
  }
  __shared__ unsigned long long off_bits;
  __shared__ int done;
  __syncthreads();
  const double tol = fmax(1.0, (double)k) * DBL_EPSILON;
  const int kk = k + (k & 1), m = kk - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  int sweep = 0;
  if (threadIdx.x == 0) done = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) off_bits = 0ull;
    __syncthreads();
    for (int t = 0; t < m; ++t) {
      for (int pr = warp; pr < kk / 2; pr += nwarps) {
        int p = rr_player(pr, t, m), q = rr_player(kk - 1 - pr, t, m);
        if (p > q) { int tmp = p; p = q; q = tmp; }
        if (q >= k) continue;
        T* ap = a + (long)p * k;
        T* aq = a + (long)q * k;
        double al = 0.0, be = 0.0;
        T ga = zero_of(T());
        for (int r = lane; r < k; r += 32) {
          const T x = ap[r], y = aq[r];
          al += absq(x);
          be += absq(y);
          fmacv(ga, x, y);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        const double g = sqrt(absq(ga));
        const double nrm = sqrt(al) * sqrt(be);
        if (!(g > tol * nrm) || g == 0.0) continue;
        if (lane == 0) atomicMax(&off_bits, (unsigned long long)__double_as_longlong(g / nrm));
        const double zeta = (be - al) / (2.0 * g);
        const double tt = copysign(1.0, zeta) / (fabs(zeta) + hypot(1.0, zeta));
        const double c = 1.0 / hypot(1.0, tt), s = c * tt;
        const T eph = phase_of<T>(ga, g);
        for (int r = lane; r < k; r += 32) {
          const T x = ap[r], y = mulv(eph, aq[r]);
          ap[r] = subv(scalev(x, c), scalev(y, s));
          aq[r] = addv(scalev(x, s), scalev(y, c));
        }
        if (want_uv) {
          T* vp = v + (long)p * k;
          T* vq = v + (long)q * k;
          for (int r = lane; r < k; r += 32) {
            const T x = vp[r], y = mulv(eph, vq[r]);
            vp[r] = subv(scalev(x, c), scalev(y, s));
            vq[r] = addv(scalev(x, s), scalev(y, c));
          }
        }
      }
      __syncthreads();
    }
    const double off = __longlong_as_double((long long)off_bits);
    __syncthreads();
    if (off <= tol) break;
  }
  if (sweep == max_sweeps && threadIdx.x == 0) atomicOr(err, DEV_JACOBI_NOCONV);
  // singular values and their descending order (ties: lower index first)
  extern __shared__ double sv[];        // k values
  int* rk = reinterpret_cast<int*>(sv + k);
  for (int c = warp; c < k; c += nwarps) {
    double acc = 0.0;
    for (int r = lane; r < k; r += 32) acc += absq(a[(long)c * k + r]);
    acc = warp_sum(acc);
    if (lane == 0) sv[c] = sqrt(acc);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    int r = 0;
    const double x = sv[c];
    for (int j = 0; j < k; ++j) r += (sv[j] > x) || (sv[j] == x && j < c);
    rk[c] = r;
    if (!isfinite(x)) atomicOr(err, DEV_NONFINITE);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) s_out[(long)b * k + rk[c]] = sv[c];
  if (!want_uv) return;
  T* Ub = U + (long)b * k * k;
  T* Vb = V + (long)b * k * k;
  for (long idx = threadIdx.x; idx < (long)k * k; idx += blockDim.x) {
    const int c = (int)(idx / k), r = (int)(idx % k);
    const double sc = sv[c];
    const T x = a[idx];
    Ub[(long)r * k + rk[c]] = sc > 0.0 ? scalev(x, 1.0 / sc) : zero_of(T());
    Vb[(long)r * k + rk[c]] = v[idx];
  }
  __syncthreads();
  // exactly-zero singular values leave zero columns of U: complete U to a
  // unitary by Gram-Schmidt against unit vectors (warp 0, rare path)
  if (warp != 0) return;
  int nzero = 0;
  for (int c = 0; c < k; ++c) nzero += (sv[c] == 0.0);
  if (nzero == 0) return;
  int cand = 0;
  for (int col = k - nzero; col < k; ++col) {
    T* tmp = a;   // reuse the work area as a length-k scratch vector
    for (; cand < k; ++cand) {
      for (int r = lane; r < k; r += 32) tmp[r] = (r == cand) ? one : zero_of(T());
      __syncwarp();
      for (int rep = 0; rep < 2; ++rep) {
        for (int j = 0; j < col; ++j) {
          T d = zero_of(T());
          for (int r = lane; r < k; r += 32) fmacv(d, Ub[(long)r * k + j], tmp[r]);
          d = warp_sum(d);
          __syncwarp();
          for (int r = lane; r < k; r += 32) tmp[r] = subv(tmp[r], mulv(Ub[(long)r * k + j], d));
          __syncwarp();
        }
      }
      double nn = 0.0;
      for (int r = lane; r < k; r += 32) nn += absq(tmp[r]);
      nn = warp_sum(nn);
      if (nn > 0.25) {
        const double inv = 1.0 / sqrt(nn);
        for (int r = lane; r < k; r += 32) Ub[(long)r * k + col] = scalev(tmp[r], inv);
        __syncwarp();
        ++cand;
        break;
      }
    }
  }
}

// ---------------------------------------------------------- phase fixing
template <typename T>
__global__ void colphase_kernel(long n, int ncol, long ld, const T* Z, long strideZ,
                                T* ph) {
  const int c = blockIdx.x, b = blockIdx.y;
  const T* z = Z + b * strideZ;
  double best = -1.0;
  long bi = 0;
  for (long r = threadIdx.x; r < n; r += blockDim.x) {
    const double m = absq(z[r * ld + c]);
    if (m > best) { best = m; bi = r; }
  }
  __shared__ double sb[256];
  __shared__ long si[256];
  sb[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double m2 = sb[threadIdx.x + o];
      const long i2 = si[threadIdx.x + o];
      if (m2 > sb[threadIdx.x] || (m2 == sb[threadIdx.x] && i2 < si[threadIdx.x])) {
        sb[threadIdx.x] = m2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const T piv = z[si[0] * ld + c];
    const double mag = sqrt(absq(piv));
    T out;
    if constexpr (sizeof(T) == 8) out = mag > 0.0 ? piv / mag : 1.0;
    else out = mag > 0.0 ? make_double2(piv.x / mag, piv.y / mag) : make_double2(1.0, 0.0);
    ph[(long)b * ncol + c] = out;
  }
}

template <typename T>
__global__ void scale_cols_kernel(long rows, int ncol, long ld, T* Z, const T* ph) {
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < rows * ncol;
       idx += (long)gridDim.x * blockDim.x) {
    const long r = idx / ncol;
    const int c = (int)(idx % ncol);
    Z[r * ld + c] = mulv(Z[r * ld + c], conjv(ph[c]));
  }
}

template <typename T>
__global__ void inv_sqrt_kernel(int k, int c, const T* V, const double* s, double cutoff,
                                T* Vs) {
  const double s0 = s[0];
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)k * c;
       idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / c), j = (int)(idx % c);
    const double sj = s[j];
    const double f = (s0 > 0.0 && sj > cutoff * s0) ? 1.0 / sqrt(sj) : 0.0;
    Vs[idx] = scalev(V[(long)i * k + j], f);
  }
}

// ------------------------------------------------------------ normalise
template <typename T>
__global__ void sumsq_partial(long n, const T* x, long stride, double* part, int nblk) {
  const int b = blockIdx.y;
  const T* xb = x + b * stride;
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x)
    acc += absq(xb[i]);
  __shared__ double sh[32];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[b * nblk + blockIdx.x] = acc;
}

__global__ void sumsq_final(const double* part, int nblk, double* nrm) {
  const int b = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[b * nblk + i];
  __shared__ double sh[32];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) nrm[b] = sqrt(acc);
}

template <typename T>
__global__ void scale_kernel(long n, T* x, long stride, const double* nrm) {
  const int b = blockIdx.y;
  const double inv = 1.0 / nrm[b];
  T* xb = x + b * stride;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x)
    xb[i] = scalev(xb[i], inv);
}

__global__ void spectra_delta_kernel(int c, int batch, double* snew, double* sold,
                                     double* delta) {
  __shared__ double sh[32];
  double dmax = 0.0;
  for (int b = 0; b < batch; ++b) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < c; i += blockDim.x) acc += snew[(long)b * c + i] * snew[(long)b * c + i];
    acc = block_sum(acc, sh);
    const double inv = acc > 0.0 ? 1.0 / sqrt(acc) : 0.0;
    double d = 0.0;
    for (int i = threadIdx.x; i < c; i += blockDim.x) {
      const double x = snew[(long)b * c + i] * inv;
      const double e = x - sold[(long)b * c + i];
      d += e * e;
      snew[(long)b * c + i] = x;
      sold[(long)b * c + i] = x;
    }
    d = block_sum(d, sh);
    dmax = fmax(dmax, sqrt(d));
  }
  if (threadIdx.x == 0) delta[0] = dmax;
}

template <typename T>
__global__ void add_identity_kernel(int k, T* G, double alpha, int batch) {
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)k * batch;
       idx += (long)gridDim.x * blockDim.x) {
    const long b = idx / k, i = idx % k;
    T* g = G + b * k * k + i * k + i;
    if constexpr (sizeof(T) == 8) *g += alpha;
    else g->x += alpha;
  }
}

template <typename T>
__global__ void trace_products_kernel(int d2, const T* O, const T* R, double* out4) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  T tor = zero_of(T()), tr = zero_of(T());
  for (int i = 0; i < d2; ++i) {
    tr = addv(tr, R[(long)i * d2 + i]);
    for (int j = 0; j < d2; ++j) fmav(tor, O[(long)i * d2 + j], R[(long)j * d2 + i]);
  }
  if constexpr (sizeof(T) == 8) {
    out4[0] = tor; out4[1] = 0.0; out4[2] = tr; out4[3] = 0.0;
  } else {
    out4[0] = tor.x; out4[1] = tor.y; out4[2] = tr.x; out4[3] = tr.y;
  }
}

__device__ __forceinline__ double hash_uniform(uint64_t a, uint64_t b, uint64_t c) {
  // splitmix64 finaliser of a counter: uniform in [-1, 1)
  uint64_t z = a * 0x9E3779B97F4A7C15ull ^ (b + 0x632BE59BD9B4E019ull) * 0xBF58476D1CE4E5B9ull ^
               (c + 0x8CB92BA72F3D8DD7ull) * 0x94D049BB133111EBull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

template <typename T>
__global__ void repair_kernel(long rows, int k, T* Q, const int* dead, uint64_t seed) {
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < rows * k;
       idx += (long)gridDim.x * blockDim.x) {
    const long r = idx / k;
    const int c = (int)(idx % k);
    if (!dead[c]) continue;
    const double x = hash_uniform(seed, (uint64_t)c, (uint64_t)r);
    if constexpr (sizeof(T) == 8) Q[idx] = x;
    else Q[idx] = make_double2(x, hash_uniform(seed ^ 0x5bd1e995ull, (uint64_t)c, (uint64_t)r));
  }
}

// per tensor: sum of |x|^2 and the first index of the largest |x|
template <typename T>
__global__ void normph_partial(long n, const T* x, long stride, double* ps, double* pm,
                               long* pi, int nblk) {
  const int b = blockIdx.y;
  const T* xb = x + b * stride;
  double acc = 0.0, best = -1.0;
  long bi = 0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const double m = absq(xb[i]);
    acc += m;
    if (m > best) { best = m; bi = i; }
  }
  __shared__ double sm[256];
  __shared__ long si[256];
  __shared__ double sh[32];
  acc = block_sum(acc, sh);
  sm[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double m2 = sm[threadIdx.x + o];
      const long i2 = si[threadIdx.x + o];
      if (m2 > sm[threadIdx.x] || (m2 == sm[threadIdx.x] && i2 < si[threadIdx.x])) {
        sm[threadIdx.x] = m2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ps[b * nblk + blockIdx.x] = acc;
    pm[b * nblk + blockIdx.x] = sm[0];
    pi[b * nblk + blockIdx.x] = si[0];
  }
}

template <typename T>
__global__ void normph_final(const T* x, long stride, const double* ps, const double* pm,
                             const long* pi, int nblk, T* fac) {
  const int b = blockIdx.x;
  if (threadIdx.x != 0) return;
  double acc = 0.0, best = -1.0;
  long bi = 0;
  for (int i = 0; i < nblk; ++i) {
    acc += ps[b * nblk + i];
    const double m = pm[b * nblk + i];
    const long j = pi[b * nblk + i];
    if (m > best || (m == best && j < bi)) { best = m; bi = j; }
  }
  const double nrm = sqrt(acc);
  const T piv = x[b * stride + bi];
  const double mag = sqrt(absq(piv));
  if constexpr (sizeof(T) == 8) {
    fac[b] = (mag > 0.0 ? (piv > 0.0 ? 1.0 : -1.0) : 1.0) / nrm;
  } else {
    fac[b] = mag > 0.0 ? make_double2(piv.x / (mag * nrm), -piv.y / (mag * nrm))
                       : make_double2(1.0 / nrm, 0.0);
  }
}

template <typename T>
__global__ void scale_by_kernel(long n, T* x, long stride, const T* fac) {
  const int b = blockIdx.y;
  const T f = fac[b];
  T* xb = x + b * stride;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x)
    xb[i] = mulv(xb[i], f);
}

// ---------------------------------------------------------------------
// CholeskyQR pass with the Gram factor in shared memory: one block factors
// the (optionally Jacobi-scaled, shifted) k x k Gram in packed lower storage
// (fp64 bound on one SM; k(k+1)/2 elements must fit in shared memory), then
// every block solves rows of Q L^H = Z D^-1 by forward substitution.
__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }  // i >= j

template <typename T>
__global__ void __launch_bounds__(256) chol_smem_kernel(int k, long n, int shift, int scale,
                                                        const T* G, T* L, double* dsc,
                                                        int* dead, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);
  T* colj = S + (size_t)k * (k + 1) / 2;   // conj of column j of L, contiguous
  double* orig = reinterpret_cast<double*>(colj + k);
  __shared__ double red[8];
  __shared__ double piv, sft_s;
  __shared__ int isdead, bad;
  // scales and packed load (lower triangle)
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double d = realv(G[(size_t)i * k + i]);
    dsc[i] = scale ? (d > 0.0 ? sqrt(d) : 1.0) : 1.0;
  }
  __syncthreads();
  for (long idx = threadIdx.x; idx < (long)k * (k + 1) / 2; idx += blockDim.x) {
    // invert the packed index
    int i = (int)((sqrt(8.0 * idx + 1.0) - 1.0) * 0.5);
    while ((long)i * (i + 1) / 2 > idx) --i;
    while ((long)(i + 1) * (i + 2) / 2 <= idx) ++i;
    const int j = (int)(idx - (long)i * (i + 1) / 2);
    S[idx] = scalev(G[(size_t)i * k + j], 1.0 / (dsc[i] * dsc[j]));
  }
  __syncthreads();
  double tr = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    orig[i] = realv(S[tri(i, i)]);
    tr += orig[i];
    if (dead) dead[i] = 0;
  }
  tr = warp_sum(tr);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tr;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    sft_s = shift ? 11.0 * ((double)n * k + (double)k * (k + 1)) * DBL_EPSILON * t : 0.0;
    bad = 0;
  }
  __syncthreads();
  const double sft = sft_s;
  if (sft != 0.0)
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      if constexpr (sizeof(T) == 8) S[tri(i, i)] += sft;
      else S[tri(i, i)].x += sft;
    }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      const double d = realv(S[tri(j, j)]);
      isdead = 0;
      if (dead && (shift ? !(d - sft > fmax(1e-9 * sft, 8.0 * k * DBL_EPSILON * (orig[j] + sft)))
                         : !(d > 1e-10 * orig[j]))) {
        isdead = 1;
        piv = 1.0;
        dead[j] = 1;
      } else if (!(d > 0.0) || !isfinite(d)) {
        piv = 1.0;
        bad = 1;
      } else {
        piv = sqrt(d);
      }
    }
    __syncthreads();
    const double inv = 1.0 / piv;
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) {
      const T v = isdead ? zero_of(T()) : scalev(S[tri(i, j)], inv);
      S[tri(i, j)] = v;
      colj[i] = conjv(v);
    }
    if (threadIdx.x == 0) {
      if constexpr (sizeof(T) == 8) S[tri(j, j)] = isdead ? 1.0 : piv;
      else S[tri(j, j)] = make_double2(isdead ? 1.0 : piv, 0.0);
    }
    __syncthreads();
    if (!isdead) {
      // trailing update S(i, l) -= L(i, j) conj(L(l, j)), j < l <= i: one
      // row per warp, lanes along the row
      const int wp = threadIdx.x >> 5, ln = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int i = j + 1 + wp; i < k; i += nw) {
        const T a = S[tri(i, j)];
        T* Si = S + tri(i, 0);
        for (int l = j + 1 + ln; l <= i; l += 32) Si[l] = subv(Si[l], mulv(a, colj[l]));
      }
    }
    __syncthreads();
  }
  if (bad && threadIdx.x == 0) atomicOr(err, DEV_CHOL_PIVOT);
  for (long idx = threadIdx.x; idx < (long)k * k; idx += blockDim.x) {
    const int i = (int)(idx / k), j = (int)(idx % k);
    L[idx] = (j <= i) ? S[tri(i, j)] : zero_of(T());
  }
}

// rows r of Q: q L^H = z D^-1, i.e. q_j = (z_j / D_j - sum_{i<j} q_i conj(L_ji)) / L_jj.
// One warp per row, right-looking: lane l owns the columns l, l + 32, ...
// (R of them, in registers); at step j the owner of column j finishes
// q_j = acc_j / L_jj and broadcasts it, and every lane subtracts
// q_j conj(L_ij) from its columns i > j. Each row costs k^2 / 2 multiply-adds
// and no reductions; conj(L) is kept column by column (packed) in shared
// memory so that the lanes read consecutive entries.
template <typename T, int R>
__global__ void __launch_bounds__(1024, 1) trsm_warp_kernel(long rows, int k, const T* L,
                                                            const double* dsc, const T* Z,
                                                            T* Q) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Lc = reinterpret_cast<T*>(smem_raw);   // column j at Lc[j k - j (j - 1) / 2 + i - j]
  double* rinv = reinterpret_cast<double*>(Lc + (size_t)k * (k + 1) / 2);
  double* dinv = rinv + k;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wp; j < k; j += nw) {
    const int off = j * k - j * (j - 1) / 2;
    for (int i = j + lane; i < k; i += 32) Lc[off + i - j] = conjv(L[(size_t)i * k + j]);
    if (lane == 0) {
      rinv[j] = 1.0 / realv(L[(size_t)j * k + j]);
      dinv[j] = 1.0 / dsc[j];
    }
  }
  __syncthreads();
  // row r = wp G + b + t G nw: a partial last pass over the rows spreads
  // over all blocks (a few warps each) instead of filling a few blocks
  for (long r = (long)wp * gridDim.x + blockIdx.x; r < rows; r += (long)gridDim.x * nw) {
    const T* z = Z + r * k;
    T a[R];
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int i = lane + 32 * e;
      a[e] = i < k ? scalev(z[i], dinv[i]) : zero_of(T());
    }
#pragma unroll
    for (int e = 0; e < R; ++e) {
      for (int jj = 0; jj < 32; ++jj) {
        const int j = 32 * e + jj;
        if (j >= k) break;
        if (lane == jj) a[e] = scalev(a[e], rinv[j]);
        T q;
        if constexpr (sizeof(T) == 8) {
          q = __shfl_sync(0xffffffffu, a[e], jj);
        } else {
          q.x = __shfl_sync(0xffffffffu, a[e].x, jj);
          q.y = __shfl_sync(0xffffffffu, a[e].y, jj);
        }
        const T* Lj = Lc + (j * k - j * (j - 1) / 2) - j;
#pragma unroll
        for (int e2 = e; e2 < R; ++e2) {
          const int i = lane + 32 * e2;
          if (i > j && i < k) fnmav(a[e2], q, Lj[i]);
        }
      }
    }
    T* qo = Q + r * k;
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int i = lane + 32 * e;
      if (i < k) qo[i] = a[e];
    }
  }
}

unsigned grid_for(long n, int per = 256, long cap = 152L * 8) {
  long g = (n + per - 1) / per;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace

cudaError_t chol_inv(bool cx, int k, long n, bool shift, void* G, void* Linv,
                     int batch, int* dead, int* err, cudaStream_t s, long* launches) {
  const size_t shm = (size_t)k * sizeof(double);
  if (cx)
    chol_inv_kernel<cplx><<<batch, 256, shm, s>>>(k, n, shift, (cplx*)G, (cplx*)Linv, dead, err);
  else
    chol_inv_kernel<double><<<batch, 256, shm, s>>>(k, n, shift, (double*)G, (double*)Linv,
                                                     dead, err);
  if (launches) ++*launches;
  return cudaGetLastError();
}

size_t chol_smem_bytes(bool cx, int k) {
  return ((size_t)k * (k + 1) / 2 + k) * (cx ? 16 : 8) + (size_t)k * sizeof(double) + 16;
}

template <typename T>
cudaError_t trsm_set_smem(size_t (&configured)[5], size_t shm) {
  const void* fns[] = {(const void*)trsm_warp_kernel<T, 2>, (const void*)trsm_warp_kernel<T, 4>,
                       (const void*)trsm_warp_kernel<T, 5>, (const void*)trsm_warp_kernel<T, 6>,
                       (const void*)trsm_warp_kernel<T, 8>};
  for (int i = 0; i < 5; ++i) {
    const cudaError_t e = raise_smem(fns[i], configured[i], shm);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// one shared-memory limit per Cholesky kernel instance, raised monotonically
// (every launcher of chol_smem_kernel goes through here)
cudaError_t chol_smem_prepare(bool cx, size_t shm) {
  static size_t configured[2] = {0, 0};
  return cx ? raise_smem((const void*)chol_smem_kernel<cplx>, configured[1], shm)
            : raise_smem((const void*)chol_smem_kernel<double>, configured[0], shm);
}

// R = columns per lane: the smallest of 2, 4, 5, 6, 8 with 32 R >= k
#define CTM_TRSM_LAUNCH(T)                                                                     \
  do {                                                                                         \
    if (k <= 64)                                                                               \
      trsm_warp_kernel<T, 2><<<(unsigned)g, 1024, shm, s>>>(rows, k, (const T*)L, dsc,         \
                                                             (const T*)Z, (T*)Q);              \
    else if (k <= 128)                                                                         \
      trsm_warp_kernel<T, 4><<<(unsigned)g, 1024, shm, s>>>(rows, k, (const T*)L, dsc,         \
                                                             (const T*)Z, (T*)Q);              \
    else if (k <= 160)                                                                         \
      trsm_warp_kernel<T, 5><<<(unsigned)g, 1024, shm, s>>>(rows, k, (const T*)L, dsc,         \
                                                             (const T*)Z, (T*)Q);              \
    else if (k <= 192)                                                                         \
      trsm_warp_kernel<T, 6><<<(unsigned)g, 1024, shm, s>>>(rows, k, (const T*)L, dsc,         \
                                                             (const T*)Z, (T*)Q);              \
    else                                                                                       \
      trsm_warp_kernel<T, 8><<<(unsigned)g, 1024, shm, s>>>(rows, k, (const T*)L, dsc,         \
                                                             (const T*)Z, (T*)Q);              \
  } while (0)

cudaError_t chol_qr_pass(bool cx, int k, long rows, bool shift, bool scale, const void* G,
                         void* L, double* dsc, int* dead, const void* Z, void* Q, int* err,
                         int num_sms, cudaStream_t s, long* launches) {
  const size_t shm = chol_smem_bytes(cx, k);
  static size_t configured_trsm[2][5] = {{0}};
  {
    cudaError_t e = chol_smem_prepare(cx, shm);
    if (e == cudaSuccess) e = cx ? trsm_set_smem<cplx>(configured_trsm[1], shm)
                                 : trsm_set_smem<double>(configured_trsm[0], shm);
    if (e != cudaSuccess) return e;
  }
  // one 1024-thread block per SM (the factor fills shared memory), one warp
  // per row
  long g = (rows + 31) / 32;
  if (g > num_sms) g = num_sms;
  if (g < 1) g = 1;
  if (cx) {
    chol_smem_kernel<cplx><<<1, 256, shm, s>>>(k, rows, shift, scale, (const cplx*)G, (cplx*)L, dsc,
                                                dead, err);
    CTM_TRSM_LAUNCH(cplx);
  } else {
    chol_smem_kernel<double><<<1, 256, shm, s>>>(k, rows, shift, scale, (const double*)G, (double*)L,
                                                  dsc, dead, err);
    CTM_TRSM_LAUNCH(double);
  }
  if (launches) *launches += 2;
  return cudaGetLastError();
}

cudaError_t trsm_rows(bool cx, int k, long rows, const void* L, const double* dsc, const void* Z,
                      void* Q, int num_sms, cudaStream_t s, long* launches) {
  const size_t shm = chol_smem_bytes(cx, k);
  static size_t configured_trsm[2][5] = {{0}};
  {
    const cudaError_t e = cx ? trsm_set_smem<cplx>(configured_trsm[1], shm)
                             : trsm_set_smem<double>(configured_trsm[0], shm);
    if (e != cudaSuccess) return e;
  }
  long g = (rows + 31) / 32;
  if (g > num_sms) g = num_sms;
  if (g < 1) g = 1;
  if (cx) CTM_TRSM_LAUNCH(cplx);
  else CTM_TRSM_LAUNCH(double);
  if (launches) ++*launches;
  return cudaGetLastError();
}

// W = D^-1 L^-H from the factor of chol_smem_kernel: block c solves the
// column c of X = L^-1 by forward substitution (one warp, x in shared
// memory) and writes row c of W, W[c][i] = conj(X[i][c]) / D_c (i >= c).
template <typename T>
__global__ void __launch_bounds__(32) trinv_kernel(int k, const T* L, const double* dsc, T* W) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);
  const int c = blockIdx.x, lane = threadIdx.x;
  for (int i = c; i < k; ++i) {
    T acc = zero_of(T());
    const T* Li = L + (size_t)i * k;
    for (int l = c + lane; l < i; l += 32) fmav(acc, Li[l], xs[l]);
    acc = warp_sum(acc);
    if (lane == 0) {
      const double inv = 1.0 / realv(Li[i]);
      if (i == c) {
        if constexpr (sizeof(T) == 8) xs[i] = inv;
        else xs[i] = make_double2(inv, 0.0);
      } else {
        xs[i] = scalev(acc, -inv);
      }
    }
    __syncwarp();
  }
  const double id = 1.0 / dsc[c];
  for (int i = lane; i < k; i += 32)
    W[(size_t)c * k + i] = i >= c ? scalev(conjv(xs[i]), id) : zero_of(T());
}

cudaError_t chol_factor_inv(bool cx, int k, long rows, bool shift, bool scale, const void* G,
                            void* L, double* dsc, int* dead, void* W, int* err, cudaStream_t s,
                            long* launches) {
  const size_t shm = chol_smem_bytes(cx, k);
  const cudaError_t e = chol_smem_prepare(cx, shm);
  if (e != cudaSuccess) return e;
  if (cx) {
    chol_smem_kernel<cplx><<<1, 256, shm, s>>>(k, rows, shift, scale, (const cplx*)G, (cplx*)L,
                                                dsc, dead, err);
    trinv_kernel<cplx><<<k, 32, (size_t)k * sizeof(cplx), s>>>(k, (const cplx*)L, dsc, (cplx*)W);
  } else {
    chol_smem_kernel<double><<<1, 256, shm, s>>>(k, rows, shift, scale, (const double*)G,
                                                  (double*)L, dsc, dead, err);
    trinv_kernel<double><<<k, 32, (size_t)k * sizeof(double), s>>>(k, (const double*)L, dsc,
                                                                    (double*)W);
  }
  if (launches) *launches += 2;
  return cudaGetLastError();
}

cudaError_t repair_dead_columns(bool cx, long rows, int k, void* Q, const int* dead,
                                uint64_t seed, cudaStream_t s, long* launches) {
  if (cx) repair_kernel<cplx><<<grid_for(rows * k), 256, 0, s>>>(rows, k, (cplx*)Q, dead, seed);
  else repair_kernel<double><<<grid_for(rows * k), 256, 0, s>>>(rows, k, (double*)Q, dead, seed);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t normalize_phase(bool cx, long n, void* x, long stride, int batch, void* fac,
                            void* work, cudaStream_t s, long* launches) {
  int nblk = (int)((n + 255) / 256);
  if (nblk > 152) nblk = 152;
  if (nblk < 1) nblk = 1;
  double* ps = static_cast<double*>(work);
  double* pm = ps + (size_t)nblk * batch;
  long* pi = reinterpret_cast<long*>(pm + (size_t)nblk * batch);
  dim3 g(nblk, batch);
  if (cx) {
    normph_partial<cplx><<<g, 256, 0, s>>>(n, (const cplx*)x, stride, ps, pm, pi, nblk);
    normph_final<cplx><<<batch, 32, 0, s>>>((const cplx*)x, stride, ps, pm, pi, nblk, (cplx*)fac);
    scale_by_kernel<cplx><<<g, 256, 0, s>>>(n, (cplx*)x, stride, (const cplx*)fac);
  } else {
    normph_partial<double><<<g, 256, 0, s>>>(n, (const double*)x, stride, ps, pm, pi, nblk);
    normph_final<double><<<batch, 32, 0, s>>>((const double*)x, stride, ps, pm, pi, nblk, (double*)fac);
    scale_by_kernel<double><<<g, 256, 0, s>>>(n, (double*)x, stride, (const double*)fac);
  }
  if (launches) *launches += 3;
  return cudaGetLastError();
}

cudaError_t jacobi_svd(bool cx, int k, const void* A, long strideA, double* sv,
                       void* U, void* V, bool want_uv, void* work, int batch,
                       int max_sweeps, int* err, cudaStream_t s, long* launches) {
  const size_t shm = (size_t)k * (sizeof(double) + sizeof(int));
  if (cx)
    jacobi_kernel<cplx><<<batch, 512, shm, s>>>(k, (const cplx*)A, strideA, sv, (cplx*)U,
                                                (cplx*)V, want_uv, (cplx*)work, max_sweeps, err);
  else
    jacobi_kernel<double><<<batch, 512, shm, s>>>(k, (const double*)A, strideA, sv,
                                                  (double*)U, (double*)V, want_uv,
                                                  (double*)work, max_sweeps, err);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t column_phase(bool cx, long n, int ncol, long ld, const void* Z, void* ph,
                         int batch, long strideZ, cudaStream_t s, long* launches) {
  dim3 grid(ncol, batch);
  if (cx) colphase_kernel<cplx><<<grid, 256, 0, s>>>(n, ncol, ld, (const cplx*)Z, strideZ, (cplx*)ph);
  else colphase_kernel<double><<<grid, 256, 0, s>>>(n, ncol, ld, (const double*)Z, strideZ, (double*)ph);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t scale_columns_conj(bool cx, long rows, int ncol, long ld, void* Z,
                               const void* ph, cudaStream_t s, long* launches) {
  if (cx) scale_cols_kernel<cplx><<<grid_for(rows * ncol), 256, 0, s>>>(rows, ncol, ld, (cplx*)Z, (const cplx*)ph);
  else scale_cols_kernel<double><<<grid_for(rows * ncol), 256, 0, s>>>(rows, ncol, ld, (double*)Z, (const double*)ph);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t scale_by_inv_sqrt(bool cx, int k, int c, const void* V, const double* sv,
                              double cutoff, void* Vs, cudaStream_t s, long* launches) {
  if (cx) inv_sqrt_kernel<cplx><<<grid_for((long)k * c), 256, 0, s>>>(k, c, (const cplx*)V, sv, cutoff, (cplx*)Vs);
  else inv_sqrt_kernel<double><<<grid_for((long)k * c), 256, 0, s>>>(k, c, (const double*)V, sv, cutoff, (double*)Vs);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t normalize(bool cx, long n, void* x, long stride, int batch, double* nrm,
                      bool scale, void* work, cudaStream_t s, long* launches) {
  int nblk = (int)((n + 255) / 256);
  if (nblk > 152) nblk = 152;
  if (nblk < 1) nblk = 1;
  dim3 g(nblk, batch);
  if (cx) sumsq_partial<cplx><<<g, 256, 0, s>>>(n, (const cplx*)x, stride, (double*)work, nblk);
  else sumsq_partial<double><<<g, 256, 0, s>>>(n, (const double*)x, stride, (double*)work, nblk);
  sumsq_final<<<batch, 256, 0, s>>>((const double*)work, nblk, nrm);
  if (launches) *launches += 2;
  if (scale) {
    if (cx) scale_kernel<cplx><<<g, 256, 0, s>>>(n, (cplx*)x, stride, nrm);
    else scale_kernel<double><<<g, 256, 0, s>>>(n, (double*)x, stride, nrm);
    if (launches) ++*launches;
  }
  return cudaGetLastError();
}

cudaError_t spectra_delta(int c, int batch, double* snew, double* sold, double* delta,
                          cudaStream_t s, long* launches) {
  spectra_delta_kernel<<<1, 256, 0, s>>>(c, batch, snew, sold, delta);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t add_identity(bool cx, int k, void* G, double alpha, int batch, cudaStream_t s,
                         long* launches) {
  if (cx) add_identity_kernel<cplx><<<grid_for((long)k * batch), 256, 0, s>>>(k, (cplx*)G, alpha, batch);
  else add_identity_kernel<double><<<grid_for((long)k * batch), 256, 0, s>>>(k, (double*)G, alpha, batch);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t trace_products(bool cx, int d2, const void* O, const void* R, double* out4,
                           cudaStream_t s, long* launches) {
  if (cx) trace_products_kernel<cplx><<<1, 32, 0, s>>>(d2, (const cplx*)O, (const cplx*)R, out4);
  else trace_products_kernel<double><<<1, 32, 0, s>>>(d2, (const double*)O, (const double*)R, out4);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace ctm

namespace ctm {
namespace {

// out = 1 - ||M[:c, :c]||_F^2 / c for a k x k row-major M (one block)
template <typename T>
__global__ void mean_sin2_kernel(int k, int c, const T* M, double* out) {
  __shared__ double part[32];
  double acc = 0.0;
  for (long idx = threadIdx.x; idx < (long)c * c; idx += blockDim.x) {
    const long i = idx / c, j = idx % c;
    acc += absq(M[i * k + j]);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *out = 1.0 - v / (double)c;
  }
}

}  // namespace

cudaError_t mean_sin2(bool cx, int k, int c, const void* M, double* out, cudaStream_t s,
                      long* launches) {
  if (cx) mean_sin2_kernel<cplx><<<1, 256, 0, s>>>(k, c, (const cplx*)M, out);
  else mean_sin2_kernel<double><<<1, 256, 0, s>>>(k, c, (const double*)M, out);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace ctm

#include "small_eig.cuh"

namespace ctm {
namespace {

// counter-based pseudo-random fill (splitmix64 of seed and index), uniform
// in [-1, 1): a deterministic start block
__global__ void hash_fill_kernel(long n, uint64_t seed, double* x) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    uint64_t z = seed * 0x9E3779B97F4A7C15ull + (uint64_t)i * 0xBF58476D1CE4E5B9ull + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

// eigenvalues of one m x m (real or complex) row-major matrix, sorted by
// descending modulus (stable), as (re, im) pairs; status[0] = iterations
// or -1
template <typename T>
__global__ void small_eig_kernel(int m, const T* H, double* ev, int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  zc A[32 * 32], e[32];
  for (int i = 0; i < m * m; ++i) {
    if constexpr (sizeof(T) == 16) A[i] = zmk(reinterpret_cast<const double2*>(H)[i].x,
                                              reinterpret_cast<const double2*>(H)[i].y);
    else A[i] = zmk(reinterpret_cast<const double*>(H)[i], 0.0);
  }
  const int it = small_eigvals(m, A, e);
  for (int i = 1; i < m; ++i) {
    const zc v = e[i];
    const double a = zabs(v);
    int j = i - 1;
    while (j >= 0 && zabs(e[j]) < a) {
      e[j + 1] = e[j];
      --j;
    }
    e[j + 1] = v;
  }
  for (int i = 0; i < m; ++i) {
    ev[2 * i] = e[i].re;
    ev[2 * i + 1] = e[i].im;
  }
  status[0] = it;
}

}  // namespace

cudaError_t hash_fill(long n, uint64_t seed, double* x, cudaStream_t s, long* launches) {
  long b = (n + 255) / 256;
  if (b > 152L * 8) b = 152L * 8;
  hash_fill_kernel<<<(unsigned)(b < 1 ? 1 : b), 256, 0, s>>>(n, seed, x);
  if (launches) ++*launches;
  return cudaGetLastError();
}

cudaError_t small_eig(bool cx, int m, const void* H, double* ev, int* status, cudaStream_t s,
                      long* launches) {
  if (m < 1 || m > 32) return cudaErrorInvalidValue;
  if (cx) small_eig_kernel<cplx><<<1, 1, 0, s>>>(m, (const cplx*)H, ev, status);
  else small_eig_kernel<double><<<1, 1, 0, s>>>(m, (const double*)H, ev, status);
  if (launches) ++*launches;
  return cudaGetLastError();
}

}  // namespace ctm
