// Internal interface of libctm: the context and the contraction helpers that
// the move (ctm.cu) and the reverse-mode pass (grad.cu) share. Not part of the
// C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <initializer_list>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "common.cuh"
#include "ctm.h"
#include "kernels.h"
#include "split_gemm.h"
#include "svd_proj.h"

namespace ctmi {

struct Tn {
  void* p = nullptr;
  int r = 0;
  long d[8] = {0};
  long size() const {
    long s = 1;
    for (int i = 0; i < r; ++i) s *= d[i];
    return s;
  }
};

inline Tn tn(void* p, std::initializer_list<long> dims) {
  Tn t;
  t.p = p;
  for (long x : dims) t.d[t.r++] = x;
  return t;
}

struct GradState;   // recorded moves for the reverse-mode pass (grad.cu)
using ctm::SplitCtx;
using ctm::SvdCtx;

}  // namespace ctmi

using ctm::SplitCtx;
using ctm::SvdCtx;

struct ctm_ctx {
  int Lx = 0, Ly = 0, S = 0, d = 0, Dk = 0, Db = 0, chi = 0, N = 0, k = 0;
  bool cx = false;
  size_t es = 8;
  ctm_opts opts{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<void*> allocs;
  // tensors
  void* ket[4] = {nullptr};  // [S][d Dk^4] per rotation
  void* bra[4] = {nullptr};  // [S][d Db^4]
  void* C = nullptr;         // [4][S][chi^2]
  void* T = nullptr;         // [4][S][chi^2 Dk Db]
  void* X = nullptr;         // [4][S][N k]
  void* W = nullptr;
  std::vector<char> rf_ready;
  // workspace
  void* Q[4] = {nullptr};
  void* pipe[2] = {nullptr};
  size_t pipe_elems = 0;
  char* scratch = nullptr;
  size_t scratch_bytes = 0, scratch_off = 0;
  void* Pl = nullptr;        // [Lmax][N chi] current column
  void* PrH = nullptr;
  void* lastPl = nullptr;    // [S][N chi] of the last move
  void* lastPrH = nullptr;
  int last_dir = -1;
  void* Z[4] = {nullptr};    // N x k blocks
  void* ZR = nullptr;        // [Lmax][N k] Z_R, Z_L of the cuts of a column
  void* ZL = nullptr;
  void* Xn = nullptr;
  void* Wn = nullptr;
  void* G = nullptr;         // k x k
  void* Linv = nullptr;
  void* rho = nullptr;       // [Lmax][k k]
  void* u = nullptr;         // [Lmax][k k]
  void* v = nullptr;
  void* jv0 = nullptr;       // fp32 pre-solve of the small SVDs: V0 (two buffers),
  void* jv1 = nullptr;       // Newton-Schulz temporary and A V0, each
  void* jT = nullptr;        // max(Lmax k^2, 4 S chi^2) elements
  void* jB = nullptr;
  void* jw = nullptr;        // Jacobi work, max(2 Lmax k^2, 8 S chi^2) elements
  void* ph = nullptr;
  void* Vs = nullptr;        // k x chi
  void* Us = nullptr;
  double* sv = nullptr;      // max(Lmax k, 4 S chi)
  void* stC1 = nullptr;      // staging [Lmax][chi^2]
  void* stC4 = nullptr;
  void* stT4 = nullptr;      // [Lmax][chi^2 Dk Db]
  double* spec_old = nullptr;  // [4 S][chi]
  double* spec_new = nullptr;
  double* dscal = nullptr;     // small device scalars
  void* op = nullptr;          // d^4 operator
  void* rho2 = nullptr;        // d^4 two-site density matrix
  void* imp[2] = {nullptr};    // impurity kets
  int* err = nullptr;
  int* dead = nullptr;         // k flags of the CholeskyQR repair
  void* chol_work = nullptr;   // cooperative Cholesky scratch
  double* dsc = nullptr;       // column scales of the Jacobi-scaled Gram
  void* fac = nullptr;         // per-tensor normalisation factors
  uint64_t qr_calls = 0;       // counter of the repair directions
  // recycling policy (opts.recycle_sin2): per direction and cut, the number of
  // subspace-iteration updates made and whether the next move only recycles
  std::vector<int> si_updates;
  std::vector<char> si_skip;
  std::vector<char> si_rounds_used;   // rounds > 0 in the last move of (r, cut)
  double* dsin2 = nullptr;     // [4 S] mean sin^2 of the last move of each cut
  void* sinG = nullptr;        // [Lmax][k k] X_old^H X_upd of the cuts of a column
  void* Xraw = nullptr;        // initial raw blocks (randomized-SVD warm-up)
  void* Wraw = nullptr;
  long n_updates = 0, n_skipped = 0;
  int moves_done[4] = {0, 0, 0, 0};
  int num_sms = 1;
  bool spectra_init = false;
  // spec_old holds the normalised spectra of the current C (set by the
  // convergence measure, cleared by anything that changes C)
  bool spectra_fresh = false;
  // split-precision state
  SplitCtx* split = nullptr;
  // refinement (opts.split_refine): every large product exact-digit fp64-accurate
  bool exact = false;
  // lanes: the cuts of a column are independent until their small SVDs, so
  // they run concurrently, each on its own stream with its own corners and
  // workspace; use_lane() points the fields above at lane i
  struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    void* Q[4] = {nullptr};
    void* pipe[2] = {nullptr};
    char* scratch = nullptr;
    size_t scratch_bytes = 0;
    SplitCtx* split = nullptr;
    void* Z[4] = {nullptr};
    void* G = nullptr;
    void* Linv = nullptr;
    double* dsc = nullptr;
    int* dead = nullptr;
    void* chol_work = nullptr;   // cooperative Cholesky scratch (large k)
    // projector step of a cut (si_finish): recycled bases, scaled v / u, phases
    void* Xn = nullptr;
    void* Wn = nullptr;
    void* Vs = nullptr;
    void* Us = nullptr;
    void* ph = nullptr;
  };
  std::vector<Lane> lanes;   // lane 0 = the context's own buffers and stream
  int cur_lane = 0;
  // standard truncated-SVD projectors (CTM_PROJ_SVD)
  SvdCtx* svd = nullptr;
  void* svdM = nullptr;      // N x N
  void* svdUs = nullptr;     // N x chi
  void* svdVs = nullptr;
  // phase timing (profiling)
  bool prof = false;
  std::vector<cudaEvent_t> pev;
  std::vector<int> pph;
  size_t pev_used = 0;
  double phase_ms[CTM_NPHASES] = {0};
  // bookkeeping
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double last_ms = 0.0;
  long launches = 0, last_launches = 0;
  std::string msg;
  // reverse-mode differentiation: checkpoints of recorded moves
  ctmi::GradState* grad = nullptr;
  bool bra_is_conj = false;   // iPEPS context with bra = conj(A)
};

namespace ctm {
ctm_status cuda_fail(cudaError_t e, const char* expr, const char* file, int line);
}

#define CK(expr)                                \
  do {                                          \
    ctm_status st__ = (expr);                   \
    if (st__ != CTM_OK) return st__;            \
  } while (0)

namespace ctmi {

extern thread_local std::string g_create_error;
extern thread_local ctm_ctx* g_cur;

struct Guard {
  explicit Guard(ctm_ctx* c) { g_cur = c; }
  ~Guard() { g_cur = nullptr; }
};

ctm_status fail(ctm_ctx* c, ctm_status st, const std::string& m);
size_t elems_C(const ctm_ctx* c);
size_t elems_T(const ctm_ctx* c);
size_t elems_ket(const ctm_ctx* c);
size_t elems_bra(const ctm_ctx* c);
char* at(void* base, size_t elems, const ctm_ctx* c);
ctm_status dalloc(ctm_ctx* c, void** p, size_t bytes);
int frame_site(const ctm_ctx* c, int r, int x, int y);
int frame_label(int r, int i);
void* Cp(ctm_ctx* c, int label, int site);
void* Tp(ctm_ctx* c, int label, int site);
void* KETp(ctm_ctx* c, int rot, int site);
void* BRAp(ctm_ctx* c, int rot, int site);
void use_lane(ctm_ctx* c, int i);
void* scratch_alloc(ctm_ctx* c, size_t bytes);
// out = contraction of A and B given as an einsum spec (no batch or traced
// labels): at most one permute per operand, one GEMM, one permute of out
ctm_status ein(ctm_ctx* c, const char* spec, const Tn& A, bool cA, const Tn& B, bool cB,
               const Tn& out);
ctm_status qr_inplace(ctm_ctx* c, void* Zm, void* tmp, bool split_mode);
ctm_status mm_small(ctm_ctx* c, int opA, int opB, long M, long Nn, long K, const void* A,
                    long lda, const void* B, long ldb, void* Cm, long ldc);
ctm_status check_err(ctm_ctx* c);
// recorded moves (grad.cu): called at the start of every move while recording
ctm_status grad_checkpoint(ctm_ctx* c, int r);
void grad_destroy(ctm_ctx* c);

}  // namespace ctmi
