// Standard truncated-SVD projectors (paper Eq. svd_projectors_diag), the
// comparison baseline of SI-CTMRG: the full SVD of the N x N matrix
// M = H_L H_R. The dense SVD is cuSOLVER's gesvd, the library routine the
// standard method rests on; everything around it (forming M, the sign fix,
// s^-1/2, the projector products) runs in this library's kernels.
//
// M is row-major; cuSOLVER reads the buffer as the column-major M^T, whose
// SVD is M^T = conj(V) S U^T. So the returned column-major U' holds conj(V)
// and the column-major VT' holds U^T, i.e. read row-major it is U itself.
//
// cuSOLVER is opened with dlopen on first use, so that the SI path never
// depends on it.
#include <cusolverDn.h>
#include <dlfcn.h>

#include <cstring>
#include <string>

#include "common.cuh"
#include "kernels.h"
#include "svd_proj.h"

namespace ctm {

struct SvdCtx {
  bool cx = false;
  int N = 0;
  cusolverDnHandle_t h = nullptr;
  void* Up = nullptr;       // column-major U' = conj(V), N x N
  void* VTp = nullptr;      // column-major VT' = U^T, N x N
  double* s = nullptr;      // N singular values, descending
  void* work = nullptr;
  int lwork = 0;
  double* rwork = nullptr;  // complex gesvd: N - 1 doubles
  int* info = nullptr;
  void* ph = nullptr;       // chi phases
  std::string msg;
};

namespace {

struct Solver {
  bool tried = false, ok = false;
  cusolverStatus_t (*create)(cusolverDnHandle_t*) = nullptr;
  cusolverStatus_t (*destroy)(cusolverDnHandle_t) = nullptr;
  cusolverStatus_t (*set_stream)(cusolverDnHandle_t, cudaStream_t) = nullptr;
  cusolverStatus_t (*zbuf)(cusolverDnHandle_t, int, int, int*) = nullptr;
  cusolverStatus_t (*dbuf)(cusolverDnHandle_t, int, int, int*) = nullptr;
  cusolverStatus_t (*zgesvd)(cusolverDnHandle_t, signed char, signed char, int, int,
                             cuDoubleComplex*, int, double*, cuDoubleComplex*, int,
                             cuDoubleComplex*, int, cuDoubleComplex*, int, double*, int*) = nullptr;
  cusolverStatus_t (*dgesvd)(cusolverDnHandle_t, signed char, signed char, int, int, double*, int,
                             double*, double*, int, double*, int, double*, int, double*,
                             int*) = nullptr;
};

Solver load_solver() {
  Solver sv;
  sv.tried = true;
  void* lib = nullptr;
  for (const char* name : {"libcusolver.so", "libcusolver.so.12", "libcusolver.so.13",
                           "libcusolver.so.11"})
    if ((lib = dlopen(name, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
  if (!lib) return sv;
  sv.create = reinterpret_cast<decltype(sv.create)>(dlsym(lib, "cusolverDnCreate"));
  sv.destroy = reinterpret_cast<decltype(sv.destroy)>(dlsym(lib, "cusolverDnDestroy"));
  sv.set_stream = reinterpret_cast<decltype(sv.set_stream)>(dlsym(lib, "cusolverDnSetStream"));
  sv.zbuf = reinterpret_cast<decltype(sv.zbuf)>(dlsym(lib, "cusolverDnZgesvd_bufferSize"));
  sv.dbuf = reinterpret_cast<decltype(sv.dbuf)>(dlsym(lib, "cusolverDnDgesvd_bufferSize"));
  sv.zgesvd = reinterpret_cast<decltype(sv.zgesvd)>(dlsym(lib, "cusolverDnZgesvd"));
  sv.dgesvd = reinterpret_cast<decltype(sv.dgesvd)>(dlsym(lib, "cusolverDnDgesvd"));
  sv.ok = sv.create && sv.destroy && sv.set_stream && sv.zbuf && sv.dbuf && sv.zgesvd &&
          sv.dgesvd;
  return sv;
}

// opened once (thread-safe initialisation of a function-local static)
Solver& solver() {
  static Solver sv = load_solver();
  return sv;
}

ctm_status svfail(SvdCtx* sc, ctm_status st, const char* m) {
  sc->msg = m;
  return st;
}

// ph[j] = phase of the largest-modulus entry of column j of U (row-major,
// U[i][j] = VT'[i * N + j]; lowest row on a tie), 1 for a zero column
template <typename T>
__global__ void svd_pivot_phase(int N, const T* VTp, T* ph) {
  const int j = blockIdx.x;
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double a = absq(VTp[(size_t)i * N + j]);
    if (a > best || (a == best && i < bi)) { best = a; bi = i; }
  }
  __shared__ double sb[256];
  __shared__ int si[256];
  sb[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const double b2 = sb[threadIdx.x + o];
      const int i2 = si[threadIdx.x + o];
      if (b2 > sb[threadIdx.x] || (b2 == sb[threadIdx.x] && i2 < si[threadIdx.x])) {
        sb[threadIdx.x] = b2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const T v = VTp[(size_t)si[0] * N + j];
    const double m = sqrt(absq(v));
    if constexpr (sizeof(T) == 8) ph[j] = m > 0.0 ? v / m : 1.0;
    else ph[j] = m > 0.0 ? make_double2(v.x / m, v.y / m) : make_double2(1.0, 0.0);
  }
}

// Us[i][j] = U[i][j] conj(ph_j) s_j^-1/2, Vs[i][j] = V[i][j] conj(ph_j) s_j^-1/2
// (N x chi row-major), s_j^-1/2 := 0 for s_j <= cutoff s_0
template <typename T>
__global__ void svd_scale_uv(int N, int chi, const T* Up, const T* VTp, const double* s,
                             const T* ph, double cutoff, T* Us, T* Vs) {
  const long n = (long)N * chi;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / chi), j = (int)(idx % chi);
    const double isq = (s[0] > 0.0 && s[j] > cutoff * s[0]) ? 1.0 / sqrt(s[j]) : 0.0;
    const T f = scalev(conjv(ph[j]), isq);
    Us[idx] = mulv(VTp[(size_t)i * N + j], f);
    Vs[idx] = mulv(conjv(Up[(size_t)j * N + i]), f);
  }
}

template <typename T>
__global__ void svd_unit_phase(int chi, T* ph) {
  for (int j = threadIdx.x; j < chi; j += blockDim.x) {
    if constexpr (sizeof(T) == 8) ph[j] = 1.0;
    else ph[j] = make_double2(1.0, 0.0);
  }
}

__global__ void svd_info_to_err(const int* info, int* err) {
  if (*info != 0) atomicOr(err, DEV_NONFINITE);
}

}  // namespace

ctm_status svd_create(SvdCtx** out, bool cx, int N, int chi) {
  SvdCtx* sc = new SvdCtx;
  sc->cx = cx;
  sc->N = N;
  *out = sc;
  const size_t es = cx ? 16 : 8;
  Solver& sv = solver();
  if (!sv.ok) return svfail(sc, CTM_EUNSUPPORTED, "cuSOLVER (libcusolver.so) not found");
  if (sv.create(&sc->h) != CUSOLVER_STATUS_SUCCESS) {
    sc->h = nullptr;
    return svfail(sc, CTM_ECUDA, "cusolverDnCreate failed");
  }
  if ((cx ? sv.zbuf : sv.dbuf)(sc->h, N, N, &sc->lwork) != CUSOLVER_STATUS_SUCCESS)
    return svfail(sc, CTM_ECUDA, "gesvd workspace query failed");
  if (cudaMalloc(&sc->Up, (size_t)N * N * es) != cudaSuccess ||
      cudaMalloc(&sc->VTp, (size_t)N * N * es) != cudaSuccess ||
      cudaMalloc(&sc->s, (size_t)N * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&sc->work, (size_t)sc->lwork * es) != cudaSuccess ||
      cudaMalloc(&sc->rwork, (size_t)(N > 1 ? N : 2) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&sc->info, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&sc->ph, (size_t)(chi > 0 ? chi : 1) * es) != cudaSuccess)
    return svfail(sc, CTM_ENOMEM, "device allocation for the dense SVD failed");
  return CTM_OK;
}

void svd_destroy(SvdCtx* sc) {
  if (!sc) return;
  if (sc->h) solver().destroy(sc->h);
  cudaFree(sc->Up);
  cudaFree(sc->VTp);
  cudaFree(sc->s);
  cudaFree(sc->work);
  cudaFree(sc->rwork);
  cudaFree(sc->info);
  cudaFree(sc->ph);
  delete sc;
}

ctm_status svd_truncated(SvdCtx* sc, void* M, int chi, double cutoff, bool sign_fix, void* Us,
                         void* Vs, int* err, cudaStream_t s, long* launches) {
  const int N = sc->N;
  if (chi < 1 || chi > N) return svfail(sc, CTM_EINVAL, "chi out of range for the dense SVD");
  Solver& sv = solver();
  if (sv.set_stream(sc->h, s) != CUSOLVER_STATUS_SUCCESS)
    return svfail(sc, CTM_ECUDA, "cusolverDnSetStream failed");
  cusolverStatus_t st;
  if (sc->cx)
    st = sv.zgesvd(sc->h, 'S', 'S', N, N, static_cast<cuDoubleComplex*>(M), N, sc->s,
                          static_cast<cuDoubleComplex*>(sc->Up), N,
                          static_cast<cuDoubleComplex*>(sc->VTp), N,
                          static_cast<cuDoubleComplex*>(sc->work), sc->lwork, sc->rwork,
                          sc->info);
  else
    st = sv.dgesvd(sc->h, 'S', 'S', N, N, static_cast<double*>(M), N, sc->s,
                          static_cast<double*>(sc->Up), N, static_cast<double*>(sc->VTp), N,
                          static_cast<double*>(sc->work), sc->lwork, nullptr, sc->info);
  if (st != CUSOLVER_STATUS_SUCCESS) return svfail(sc, CTM_ECUDA, "gesvd failed");
  svd_info_to_err<<<1, 1, 0, s>>>(sc->info, err);
  const long n = (long)N * chi;
  long g = (n + 255) / 256;
  if (g > 152L * 8) g = 152L * 8;
  if (sc->cx) {
    if (sign_fix) {
      svd_pivot_phase<cplx><<<chi, 256, 0, s>>>(N, (const cplx*)sc->VTp, (cplx*)sc->ph);
    } else {
      svd_unit_phase<cplx><<<1, 256, 0, s>>>(chi, (cplx*)sc->ph);
    }
    svd_scale_uv<cplx><<<(unsigned)g, 256, 0, s>>>(N, chi, (const cplx*)sc->Up,
                                                     (const cplx*)sc->VTp, sc->s,
                                                     (const cplx*)sc->ph, cutoff, (cplx*)Us,
                                                     (cplx*)Vs);
  } else {
    if (sign_fix) {
      svd_pivot_phase<double><<<chi, 256, 0, s>>>(N, (const double*)sc->VTp, (double*)sc->ph);
    } else {
      svd_unit_phase<double><<<1, 256, 0, s>>>(chi, (double*)sc->ph);
    }
    svd_scale_uv<double><<<(unsigned)g, 256, 0, s>>>(N, chi, (const double*)sc->Up,
                                                       (const double*)sc->VTp, sc->s,
                                                       (const double*)sc->ph, cutoff,
                                                       (double*)Us, (double*)Vs);
  }
  if (launches) *launches += 3;
  return cudaGetLastError() == cudaSuccess ? CTM_OK
                                           : svfail(sc, CTM_ECUDA, "projector scaling failed");
}

const char* svd_last_error(const SvdCtx* sc) { return sc ? sc->msg.c_str() : ""; }

}  // namespace ctm
