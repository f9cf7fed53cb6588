// Host launchers of the libctm kernels (all asynchronous on the given stream).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

namespace ctm {

// Raises the dynamic shared-memory limit of kernel fn to at least bytes;
// configured remembers the largest size set so far. Serialised, so that
// several host threads (the serving runtime) may launch concurrently.
inline cudaError_t raise_smem(const void* fn, size_t& configured, size_t bytes) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (bytes <= configured) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) configured = bytes;
  return e;
}

// ------------------------------------------------------------- permute.cu
// out = in with axes reordered: output axis j is input axis perm[j]; both
// row-major and contiguous. conj conjugates complex elements on the way.
cudaError_t permute(const void* in, void* out, int rank, const long* in_dims,
                    const int* perm, bool cx, bool conj, cudaStream_t s,
                    long* launches);

// ------------------------------------------------------------- gemm64.cu
enum Op { OP_N = 0, OP_T = 1, OP_C = 2, OP_R = 3 };  // R = conj, no transpose

struct GemmDesc {
  bool cx = false;
  int opA = OP_N, opB = OP_N;
  long M = 0, N = 0, K = 0;
  const void* A = nullptr; long lda = 0, strideA = 0;
  const void* B = nullptr; long ldb = 0, strideB = 0;
  void* C = nullptr; long ldc = 0, strideC = 0;
  double alpha[2] = {1.0, 0.0};
  double beta[2] = {0.0, 0.0};
  int batch = 1;
  bool lower_only = false;   // compute only output tiles on or below the diagonal
};
// C = alpha op(A) op(B) + beta C in fp64, row-major; op(A) is M x K, op(B)
// K x N. Split-K partials (deterministic reduction) use work.
cudaError_t gemm64(const GemmDesc& g, void* work, size_t work_bytes,
                   cudaStream_t s, long* launches);
size_t gemm64_work_bytes(const GemmDesc& g);

// out[b] = sum_i conj?(x[b][i]) y[b][i] (n elements, batch b), fp64.
cudaError_t dot64(bool cx, bool conj_x, long n, const void* x, long sx,
                  const void* y, long sy, void* out, int batch, void* work,
                  size_t work_bytes, cudaStream_t s, long* launches);

// ------------------------------------------------------------- linalg.cu
// Lower Cholesky factor of G (+ shift I) and its inverse, one block per
// matrix: G is k x k (ld k), overwritten by L; Linv receives L^-1. With
// shift != 0 the shift is 11 (n k + k (k + 1)) u trace(G) (shifted
// CholeskyQR, Fukaya et al. 2020); n is the row count of the factored block.
// With dead != NULL a column that lies numerically in the span of the
// previous ones (shifted pass: residual below 1e-9 of the shift; plain pass:
// pivot below 1e-10 of its squared norm) is marked dead[j] = 1 and excluded
// (unit column of L); repair_dead_columns then refills it.
cudaError_t chol_inv(bool cx, int k, long n, bool shift, void* G, void* Linv,
                     int batch, int* dead, int* err, cudaStream_t s, long* launches);

// One CholeskyQR pass with the factor in shared memory: L = chol(D^-1 G D^-1
// (+ shift I)) (D = sqrt(diag G) with scale, else I; dead-column detection as
// in chol_inv), then Q = Z D^-1 L^-H row by row on all SMs. Needs
// chol_smem_bytes(cx, k) <= the shared memory of one block (k <= ~166
// complex, ~235 real); dsc receives D (k doubles).
size_t chol_smem_bytes(bool cx, int k);
cudaError_t chol_qr_pass(bool cx, int k, long rows, bool shift, bool scale, const void* G,
                         void* L, double* dsc, int* dead, const void* Z, void* Q, int* err,
                         int num_sms, cudaStream_t s, long* launches);

// ------------------------------------------------------------- absorb.cu
// Out[t,d,D,n,e,E] = sum A[s,u,l,d,e] B[s,v,w,D,E] In[t,l,w,n,u,v] with In,
// Out [chi, Dk, Db, chi, Dk, Db] (single-layer absorption of the ket and bra
// tensors into an enlarged corner or edge); fp32 arithmetic when fp32.
// Supported for Dk, Db <= 8 when A, B and the per-pair tiles fit in one
// block's shared memory (absorb_ab_supported; e.g. D <= 6 for any
// precision at d = 2, D = 7, 8 at d = 2 in fp32 or real fp64).
bool absorb_ab_supported(bool cx, bool fp32, int Dk, int Db, int d);
cudaError_t absorb_ab(bool cx, bool fp32, int chi, int Dk, int Db, int d, const void* In,
                      const void* A, const void* B, void* Out, int num_sms, cudaStream_t s,
                      long* launches);

// ------------------------------------------------------- cholqr_mixed.cu
// B = F^H with F = tril(G - I, -1) + diag(G - I) / 2 from the lower triangle
// of an fp64 Gram G of a nearly orthonormal block (first-order Cholesky
// factor of G = (I + F)(I + F)^H).
cudaError_t orth_correction(bool cx, int k, const void* G, void* B, cudaStream_t s,
                            long* launches);
// z -= d elementwise (n elements).
cudaError_t sub_inplace(bool cx, long n, void* z, const void* d, cudaStream_t s,
                        long* launches);

// The factor of chol_qr_pass (same options) and, instead of the row solve,
// W = D^-1 L^-H (k x k, row-major, upper triangular) so that the caller
// forms Q = Z W with a GEMM. L receives the factor.
cudaError_t chol_factor_inv(bool cx, int k, long rows, bool shift, bool scale, const void* G,
                            void* L, double* dsc, int* dead, void* W, int* err, cudaStream_t s,
                            long* launches);

// The row solve of chol_qr_pass alone: Q = Z D^-1 L^-H for a factor L and
// scales D already computed (chol_cluster).
cudaError_t trsm_rows(bool cx, int k, long rows, const void* L, const double* dsc, const void* Z,
                      void* Q, int num_sms, cudaStream_t s, long* launches);

// ------------------------------------------------------- chol_cluster.cu
// The factor of chol_qr_pass / chol_factor_inv (same options and outputs:
// L, dsc, dead; with W != null also W = D^-1 L^-H) computed by a cluster of
// eight CTAs (rows dealt cyclically, one cluster barrier per column). W may
// alias G. Where the packed factor fits one CTA's shared memory (k <= 156
// complex, 225 real) every CTA gathers it for the inverse; above that the
// CTAs keep only their own rows and read the others through distributed
// shared memory (chol_cluster_supported: up to k ~ 390 complex).
bool chol_cluster_supported(bool cx, int k);
cudaError_t chol_cluster(bool cx, int k, long rows, bool shift, bool scale, const void* G,
                         void* L, double* dsc, int* dead, void* W, int* err, cudaStream_t s,
                         long* launches);

// Overwrite the dead columns of a rows x k matrix with deterministic
// pseudo-random entries (a counter-based hash of seed, column, row).
cudaError_t repair_dead_columns(bool cx, long rows, int k, void* Q, const int* dead,
                                uint64_t seed, cudaStream_t s, long* launches);

// Per tensor (batch, stride): x <- x * conj(phase of its largest-modulus
// entry, lowest index on ties) / ||x||_F. work: 3 * 152 * batch doubles;
// fac: batch elements.
cudaError_t normalize_phase(bool cx, long n, void* x, long stride, int batch, void* fac,
                            void* work, cudaStream_t s, long* launches);

// One-sided Jacobi SVD (Hestenes) of k x k row-major matrices, one block per
// matrix: A = U diag(s) V^H with s descending; U, V row-major k x k. work
// holds 2 k^2 elements per matrix. want_uv = false computes s only.
cudaError_t jacobi_svd(bool cx, int k, const void* A, long strideA,
                       double* s, void* U, void* V, bool want_uv, void* work,
                       int batch, int max_sweeps, int* err, cudaStream_t s_,
                       long* launches);

// The same SVD with each matrix spread over several blocks of one
// cooperative grid (jacobi.cu); max_blocks caps the grid (SM count). work:
// jacobi_coop_work_bytes(cx, k, batch). With Vinit (row-major k x k per
// matrix, unitary) the accumulated V starts from Vinit instead of the
// identity: the SVD of A Vinit then returns V = Vinit J, the right singular
// vectors of A (used after the fp32 pre-solve, jacobi32_presolve). Vinit may
// alias V and A may alias U (both are read before anything is written).
cudaError_t jacobi_svd_coop(bool cx, int k, const void* A, long strideA, double* s, void* U,
                            void* V, bool want_uv, void* work, int batch, int max_sweeps,
                            int* err, int max_blocks, cudaStream_t s_, long* launches,
                            const void* Vinit = nullptr);

// ------------------------------------------------------------ jacobi32.cu
// fp32 one-sided Jacobi of a batch of k x k matrices (fp64 in, row-major,
// stride strideA elements) on clusters of two CTAs, to the fp32 threshold or
// max_sweeps: V0 receives the accumulated right rotations in fp64 (row-major
// k x k per matrix; unitary to ~1e-6), sweeps (optional) the sweeps used.
// Supported when jacobi32_supported(cx, k) (A and V each fit one CTA's
// shared memory in fp32: k <= 169 complex, 238 real).
bool jacobi32_supported(bool cx, int k);
cudaError_t jacobi32_presolve(bool cx, int k, const void* A, long strideA, void* V0, int batch,
                              int max_sweeps, int* sweeps, cudaStream_t s, long* launches);
size_t jacobi_coop_work_bytes(bool cx, int k, int batch);

// chol_inv on a cooperative grid (blocked, jacobi.cu); with scale the Gram
// is first scaled to unit diagonal (D^-1 G D^-1) and Linv returns
// L_s^-1 D^-1, so that Z Linv^H is still the orthonormalised block. work:
// chol_coop_work_bytes(k, batch).
cudaError_t chol_inv_coop(bool cx, int k, long n, bool shift, bool scale, void* G, void* Linv,
                          int batch, int* dead, void* work, int* err, int max_blocks,
                          cudaStream_t s, long* launches);
size_t chol_coop_work_bytes(int k, int batch);

// Phase of the largest-modulus entry (lowest row on ties) of each of the
// first ncol columns of an n x ld row-major matrix; ph gets the phase.
cudaError_t column_phase(bool cx, long n, int ncol, long ld, const void* Z,
                         void* ph, int batch, long strideZ, cudaStream_t s,
                         long* launches);

// Multiply column j of each listed row-major matrix by conj(ph[j]).
cudaError_t scale_columns_conj(bool cx, long rows, int ncol, long ld,
                               void* Z, const void* ph, cudaStream_t s,
                               long* launches);

// Vs[i][j] = V[i][j] * s_j^-1/2 (j < c, s_j > cutoff * s_0, else 0) for a
// k x k matrix V, output k x c.
cudaError_t scale_by_inv_sqrt(bool cx, int k, int c, const void* V,
                              const double* s, double cutoff, void* Vs,
                              cudaStream_t s_, long* launches);

// Frobenius norm of each of batch tensors (n elements) into nrm[b], then
// x /= nrm (when scale). Deterministic two-level reduction.
cudaError_t normalize(bool cx, long n, void* x, long stride, int batch,
                      double* nrm, bool scale, void* work, cudaStream_t s,
                      long* launches);

// spectra (batch x c, descending) -> unit 2-norm rows; delta[0] = max over
// rows of ||new - old||_2; old <- new.
cudaError_t spectra_delta(int c, int batch, double* snew, double* sold,
                          double* delta, cudaStream_t s, long* launches);

// out = 1 - ||M[:c, :c]||_F^2 / c for a k x k row-major M: the mean sin^2
// of the principal angles between two c-dimensional subspaces whose
// orthonormal bases have overlap matrix M[:c, :c].
cudaError_t mean_sin2(bool cx, int k, int c, const void* M, double* out, cudaStream_t s,
                      long* launches);

// x[i] = uniform [-1, 1) pseudo-random numbers of a counter-based hash of
// (seed, i) (n doubles).
cudaError_t hash_fill(long n, uint64_t seed, double* x, cudaStream_t s, long* launches);

// Eigenvalues of one m x m row-major matrix (m <= 32; real or complex), by
// Hessenberg reduction and shifted QR on one thread, sorted by descending
// modulus, into ev[2 m] (re, im); status[0] = QR iterations or -1.
cudaError_t small_eig(bool cx, int m, const void* H, double* ev, int* status, cudaStream_t s,
                      long* launches);

// G += alpha * I for batch k x k matrices
cudaError_t add_identity(bool cx, int k, void* G, double alpha, int batch,
                         cudaStream_t s, long* launches);

// y = sum_i O[i] * R[perm(i)] trace product Tr(O R) and Tr(R) for d2 x d2.
cudaError_t trace_products(bool cx, int d2, const void* O, const void* R,
                           double* out4, cudaStream_t s, long* launches);

}  // namespace ctm
