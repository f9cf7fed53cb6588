// libctm: SI-CTMRG on one GB300 -- context, move orchestration and C ABI.
//
// Paper: Zhang & Corboz, "Fast two-dimensional tensor-network contraction via
// subspace iteration" (arXiv 2607.15158). Every step runs in this library's
// kernels (permute.cu, gemm64.cu, linalg.cu, split_gemm.cu) on one stream;
// the host only sequences them.
//
// Layout in HBM (one allocation per array, all row-major):
//   ket / bra tensors, 4 rotations x sites      A[r][site][s][u][l][d][r]
//   corners  C[label][site][chi][chi]
//   edges    T[label][site][chi][chi][Dk][Db]
//   rangefinders X, W[direction][cut][N][k]
//   workspace: four enlarged corners Q[4][N][N], two pipeline buffers and a
//   scratch arena for the permutes of the pairwise contractions, the N x k
//   blocks of the subspace iteration and the k x k small problem.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

using namespace ctm;
using namespace ctmi;

namespace ctmi {

thread_local std::string g_create_error;
thread_local ctm_ctx* g_cur = nullptr;

ctm_status fail(ctm_ctx* c, ctm_status st, const std::string& m) {
  if (c) c->msg = m;
  else g_create_error = m;
  return st;
}

}  // namespace ctmi

namespace ctm {
ctm_status cuda_fail(cudaError_t e, const char* expr, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof buf, "CUDA error %s (%s) at %s:%d in %s", cudaGetErrorName(e),
           cudaGetErrorString(e), file, line, expr);
  if (ctmi::g_cur) ctmi::g_cur->msg = buf;
  else ctmi::g_create_error = buf;
  return e == cudaErrorMemoryAllocation ? CTM_ENOMEM : CTM_ECUDA;
}
}  // namespace ctm


namespace ctmi {

enum Phase { PH_CORNER = 0, PH_SLICE, PH_PROD, PH_QR, PH_SMALL, PH_ABSORB, PH_NORM, PH_SPECTRA };

// non-overlapping timed intervals of the move (only while profiling)
struct PhaseScope {
  ctm_ctx* c;
  int ph;
  bool on;
  PhaseScope(ctm_ctx* c_, int ph_) : c(c_), ph(ph_) {
    if (c->prof && c->pev_used + 2 > c->pev.size()) {
      // the whole profiled region is timed: the event pool grows
      const size_t old = c->pev.size();
      c->pev.resize(old + 16384);
      for (size_t i = old; i < c->pev.size(); ++i)
        if (cudaEventCreate(&c->pev[i]) != cudaSuccess) {
          c->pev.resize(i);
          break;
        }
      c->pph.resize(c->pev.size() / 2);
    }
    on = c->prof && c->pev_used + 2 <= c->pev.size();
    if (on) {
      cudaEventRecord(c->pev[c->pev_used], c->stream);
    }
  }
  ~PhaseScope() {
    if (on) {
      cudaEventRecord(c->pev[c->pev_used + 1], c->stream);
      c->pph[c->pev_used / 2] = ph;
      c->pev_used += 2;
    }
  }
};

void phases_fold(ctm_ctx* c) {
  for (size_t i = 0; i + 1 < c->pev_used; i += 2) {
    cudaEventSynchronize(c->pev[i + 1]);
    float t = 0.f;
    cudaEventElapsedTime(&t, c->pev[i], c->pev[i + 1]);
    c->phase_ms[c->pph[i / 2]] += t;
  }
  c->pev_used = 0;
}

// ------------------------------------------------------------ helpers
// number of lanes for an Lx x Ly cell: lane 0 runs the column-level work
// (small SVDs, projectors, absorption), lanes 1 .. 3 the cuts
int lanes_for(int Lx, int Ly) {
  const int L = std::max(Lx, Ly);
  return L >= 2 ? std::min(3, L) + 1 : 1;
}

size_t elems_C(const ctm_ctx* c) { return (size_t)c->chi * c->chi; }
size_t elems_T(const ctm_ctx* c) { return (size_t)c->chi * c->chi * c->Dk * c->Db; }
size_t elems_ket(const ctm_ctx* c) { return (size_t)c->d * c->Dk * c->Dk * c->Dk * c->Dk; }
size_t elems_bra(const ctm_ctx* c) { return (size_t)c->d * c->Db * c->Db * c->Db * c->Db; }

char* at(void* base, size_t elems, const ctm_ctx* c) {
  return static_cast<char*>(base) + elems * c->es;
}

// remaining successful allocations before an injected failure (< 0: off)
std::atomic<int> g_fail_alloc_after{-1};

ctm_status dalloc(ctm_ctx* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  {
    int left = g_fail_alloc_after.load();
    while (left >= 0) {
      if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {
        if (left == 0) {
          *p = nullptr;
          return fail(c, CTM_ENOMEM, "device allocation failed (injected by ctm_debug_fail_alloc)");
        }
        break;
      }
    }
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[256];
    snprintf(buf, sizeof buf, "device allocation of %zu bytes failed (%s)", bytes,
             cudaGetErrorString(e));
    return fail(c, CTM_ENOMEM, buf);
  }
  c->allocs.push_back(*p);
  return CTM_OK;
}

// Frame of the cell after r counter-clockwise quarter turns: frame position
// (x, y) -> original site; one turn sends site (x, y) to (y, -x mod Lx).
int frame_site(const ctm_ctx* c, int r, int x, int y) {
  const int Lxf = (r & 1) ? c->Ly : c->Lx, Lyf = (r & 1) ? c->Lx : c->Ly;
  x = ((x % Lxf) + Lxf) % Lxf;
  y = ((y % Lyf) + Lyf) % Lyf;
  for (int k = r; k > 0; --k) {
    const int lx_prev = ((k - 1) & 1) ? c->Ly : c->Lx;
    const int nx = (((-y) % lx_prev) + lx_prev) % lx_prev;
    y = x;
    x = nx;
  }
  return y * c->Lx + x;
}
int frame_label(int r, int i) { return (i + r) & 3; }

void* Cp(ctm_ctx* c, int label, int site) { return at(c->C, (size_t)(label * c->S + site) * elems_C(c), c); }
void* Tp(ctm_ctx* c, int label, int site) { return at(c->T, (size_t)(label * c->S + site) * elems_T(c), c); }
void* KETp(ctm_ctx* c, int rot, int site) { return at(c->ket[rot & 3], (size_t)site * elems_ket(c), c); }
void* BRAp(ctm_ctx* c, int rot, int site) { return at(c->bra[rot & 3], (size_t)site * elems_bra(c), c); }

// frame accessors
void* fC(ctm_ctx* c, int r, int i, int x, int y) { return Cp(c, frame_label(r, i), frame_site(c, r, x, y)); }
void* fT(ctm_ctx* c, int r, int i, int x, int y) { return Tp(c, frame_label(r, i), frame_site(c, r, x, y)); }

// Point the per-cut workspace fields of c at lane i (see ctm_ctx::Lane).
void use_lane(ctm_ctx* c, int i) {
  if (c->lanes.empty() || i == c->cur_lane) return;
  const ctm_ctx::Lane& L = c->lanes[i];
  c->stream = L.stream;
  for (int q = 0; q < 4; ++q) c->Q[q] = L.Q[q];
  c->pipe[0] = L.pipe[0];
  c->pipe[1] = L.pipe[1];
  c->scratch = L.scratch;
  c->scratch_bytes = L.scratch_bytes;
  c->scratch_off = 0;
  c->split = L.split;
  for (int q = 0; q < 4; ++q) c->Z[q] = L.Z[q];
  c->G = L.G;
  c->Linv = L.Linv;
  c->dsc = L.dsc;
  c->dead = L.dead;
  c->chol_work = L.chol_work;
  c->Xn = L.Xn;
  c->Wn = L.Wn;
  c->Vs = L.Vs;
  c->Us = L.Us;
  c->ph = L.ph;
  c->cur_lane = i;
}

// returns c to lane 0 when a move leaves early
struct LaneReset {
  ctm_ctx* c;
  ~LaneReset() { use_lane(c, 0); }
};

void* scratch_alloc(ctm_ctx* c, size_t bytes) {
  size_t off = (c->scratch_off + 255) & ~(size_t)255;
  if (off + bytes > c->scratch_bytes) return nullptr;
  c->scratch_off = off + bytes;
  return c->scratch + off;
}

ctm_status gemm(ctm_ctx* c, GemmDesc& g) {
  g.cx = c->cx;
  const size_t wb = gemm64_work_bytes(g);
  void* work = nullptr;
  const size_t mark = c->scratch_off;
  if (wb) {
    work = scratch_alloc(c, wb);
    if (!work) return fail(c, CTM_ENOMEM, "scratch arena too small for split-K partials");
  }
  CTM_CUDA_OK(gemm64(g, work, wb, c->stream, &c->launches));
  c->scratch_off = mark;
  return CTM_OK;
}

// Products whose result must stay fp64-accurate (CholeskyQR Grams, rho, the
// projectors): in split contexts with opts.fp64_tc as exact fixed-point
// digit products on the tensor cores (oz_gemm), else the fp64 GEMM.
constexpr double FP64TC_MIN_MNK = 1 << 16;
ctm_status gemm_exact(ctm_ctx* c, GemmDesc& g) {
  if (c->split && c->opts.fp64_tc && g.batch == 1 && g.opB == OP_N && g.alpha[0] == 1.0 &&
      g.alpha[1] == 0.0 && g.beta[0] == 0.0 && g.beta[1] == 0.0 &&
      (double)g.M * g.N * g.K >= FP64TC_MIN_MNK) {
    const ctm_status st = oz_gemm(c->split, g.opA, g.A, g.lda, g.opB, g.B, g.ldb, (int)g.M,
                                  (int)g.N, (int)g.K, g.C, g.ldc, c->stream, &c->launches);
    if (st != CTM_OK) return fail(c, st, split_last_error(c->split));
    return CTM_OK;
  }
  return gemm(c, g);
}

// The A / conj(A) absorption runs as one fused kernel (fp32 arithmetic in
// split contexts) where it fits, unless a split context asks for it on the
// tensor cores (opts.absorb_tc): then it is two split-precision GEMMs with
// permutes, as accurate as the other products.
bool use_fused_absorb(bool cx, bool split, const ctm_opts& o, int Dk, int Db, int d) {
  if (split && o.absorb_tc) return false;
  return absorb_ab_supported(cx, split, Dk, Db, d);
}

// contractions with at least this many multiply-adds go to the split-precision
// tensor-core GEMM when the context runs in CTM_PREC_SPLIT_BF16
constexpr double SPLIT_MIN_MNK = 1 << 22;

// ------------------------------------------------ pairwise contractions
// out[lo] = sum over shared labels of A[la] B[lb] (conj on request): at most
// one permute of each operand into a matrix view, one fp64 GEMM (or a dot
// product for a scalar result), one permute of the result.
ctm_status ein(ctm_ctx* c, const char* spec, const Tn& A, bool cA, const Tn& B, bool cB,
               const Tn& out) {
  std::string s(spec);
  const size_t comma = s.find(','), arrow = s.find("->");
  if (comma == std::string::npos || arrow == std::string::npos)
    return fail(c, CTM_EINVAL, std::string("bad contraction spec ") + spec);
  const std::string la = s.substr(0, comma), lb = s.substr(comma + 1, arrow - comma - 1),
                    lo = s.substr(arrow + 2);
  if ((int)la.size() != A.r || (int)lb.size() != B.r || (int)lo.size() != out.r)
    return fail(c, CTM_EINVAL, std::string("rank mismatch in ") + spec);
  long dim[128] = {0};
  auto setdim = [&](char ch, long v) -> bool {
    if (dim[(int)ch] && dim[(int)ch] != v) return false;
    dim[(int)ch] = v;
    return true;
  };
  for (int i = 0; i < A.r; ++i)
    if (!setdim(la[i], A.d[i])) return fail(c, CTM_EINVAL, std::string("dim mismatch in ") + spec);
  for (int i = 0; i < B.r; ++i)
    if (!setdim(lb[i], B.d[i])) return fail(c, CTM_EINVAL, std::string("dim mismatch in ") + spec);
  for (int i = 0; i < out.r; ++i)
    if (!setdim(lo[i], out.d[i])) return fail(c, CTM_EINVAL, std::string("dim mismatch in ") + spec);
  std::string fa, fb, ca, cb;
  for (char ch : lo) {
    const bool ia = la.find(ch) != std::string::npos, ib = lb.find(ch) != std::string::npos;
    if (ia && ib) return fail(c, CTM_EINVAL, std::string("batch labels unsupported: ") + spec);
    if (ia) fa += ch;
    else if (ib) fb += ch;
    else return fail(c, CTM_EINVAL, std::string("unknown output label in ") + spec);
  }
  for (char ch : la)
    if (lb.find(ch) != std::string::npos && lo.find(ch) == std::string::npos) ca += ch;
  for (char ch : lb)
    if (la.find(ch) != std::string::npos && lo.find(ch) == std::string::npos) cb += ch;
  for (char ch : la)
    if (lo.find(ch) == std::string::npos && lb.find(ch) == std::string::npos)
      return fail(c, CTM_EINVAL, std::string("traced label unsupported: ") + spec);
  for (char ch : lb)
    if (lo.find(ch) == std::string::npos && la.find(ch) == std::string::npos)
      return fail(c, CTM_EINVAL, std::string("traced label unsupported: ") + spec);
  long M = 1, Nn = 1, K = 1;
  for (char ch : fa) M *= dim[(int)ch];
  for (char ch : fb) Nn *= dim[(int)ch];
  for (char ch : ca) K *= dim[(int)ch];
  // layout options for a given contraction order
  struct Plan { int opA, opB; bool permA, permB; std::string ordA, ordB; long cost; };
  auto plan_for = [&](const std::string& co) {
    Plan p{};
    if (la == fa + co) { p.opA = OP_N; p.permA = false; }
    else if (la == co + fa) { p.opA = OP_T; p.permA = false; }
    else { p.opA = OP_N; p.permA = true; p.ordA = fa + co; }
    if (lb == co + fb) { p.opB = OP_N; p.permB = false; }
    else if (lb == fb + co) { p.opB = OP_T; p.permB = false; }
    else { p.opB = OP_N; p.permB = true; p.ordB = co + fb; }
    p.cost = (p.permA ? A.size() : 0) + (p.permB ? B.size() : 0);
    return p;
  };
  Plan p1 = plan_for(ca), p2 = plan_for(cb);
  Plan p = p2.cost < p1.cost ? p2 : p1;
  const size_t mark = c->scratch_off;
  const void* Am = A.p;
  const void* Bm = B.p;
  auto do_perm = [&](const Tn& X, const std::string& lx, const std::string& ord, bool conj,
                     const void** dst) -> ctm_status {
    void* buf = scratch_alloc(c, X.size() * c->es);
    if (!buf) return fail(c, CTM_ENOMEM, std::string("scratch arena too small in ") + spec);
    int perm[8];
    for (int j = 0; j < X.r; ++j) perm[j] = (int)lx.find(ord[j]);
    CTM_CUDA_OK(permute(X.p, buf, X.r, X.d, perm, c->cx, conj && c->cx, c->stream, &c->launches));
    *dst = buf;
    return CTM_OK;
  };
  bool conjA_in_gemm = false, conjB_in_gemm = false;
  if (p.permA) CK(do_perm(A, la, p.ordA, cA, &Am));
  else conjA_in_gemm = cA;
  if (p.permB) CK(do_perm(B, lb, p.ordB, cB, &Bm));
  else conjB_in_gemm = cB;
  if (c->cx) {
    if (conjA_in_gemm) p.opA = (p.opA == OP_T) ? OP_C : OP_R;
    if (conjB_in_gemm) p.opB = (p.opB == OP_T) ? OP_C : OP_R;
  }
  const std::string want = fa + fb;
  const bool final_perm = (want != lo);
  void* Cm = out.p;
  if (final_perm) {
    Cm = scratch_alloc(c, (size_t)M * Nn * c->es);
    if (!Cm) return fail(c, CTM_ENOMEM, std::string("scratch arena too small in ") + spec);
  }
  if (M == 1 && Nn == 1) {
    // scalar: a dot product; both operands are in contraction order
    if (p.opA == OP_R || p.opA == OP_C || p.opB == OP_R || p.opB == OP_C) {
      // conjugation outside a permute: materialise it
      if (p.opA == OP_R || p.opA == OP_C) CK(do_perm(tn((void*)Am, {K}), "k", "k", true, &Am));
      if (p.opB == OP_R || p.opB == OP_C) CK(do_perm(tn((void*)Bm, {K}), "k", "k", true, &Bm));
    }
    const size_t wb = (size_t)304 * c->es;
    void* w = scratch_alloc(c, wb);
    if (!w) return fail(c, CTM_ENOMEM, "scratch arena too small for a dot product");
    CTM_CUDA_OK(dot64(c->cx, false, K, Am, 0, Bm, 0, Cm, 1, w, wb, c->stream, &c->launches));
  } else {
    const long lda = (p.opA == OP_N || p.opA == OP_R) ? K : M;
    const long ldb = (p.opB == OP_N || p.opB == OP_R) ? Nn : K;
    if (c->split && (double)M * Nn * K >= SPLIT_MIN_MNK) {
      // large contraction (enlarged corners, absorption): split precision on
      // the tensor cores (exact digits during the refinement)
      const ctm_status st =
          c->exact ? oz_gemm(c->split, p.opA, Am, lda, p.opB, Bm, ldb, (int)M, (int)Nn, (int)K,
                             Cm, Nn, c->stream, &c->launches)
                   : split_gemm(c->split, p.opA, Am, lda, p.opB, Bm, ldb, (int)M, (int)Nn,
                                       (int)K, Cm, Nn, c->stream, &c->launches);
      if (st != CTM_OK) return fail(c, st, split_last_error(c->split));
    } else {
      GemmDesc g;
      g.opA = p.opA;
      g.opB = p.opB;
      g.M = M; g.N = Nn; g.K = K;
      g.A = Am; g.lda = lda;
      g.B = Bm; g.ldb = ldb;
      g.C = Cm; g.ldc = Nn;
      CK(gemm(c, g));
    }
  }
  if (final_perm) {
    Tn tmp;
    tmp.p = Cm;
    tmp.r = (int)want.size();
    for (int j = 0; j < tmp.r; ++j) tmp.d[j] = dim[(int)want[j]];
    int perm[8];
    for (int j = 0; j < out.r; ++j) perm[j] = (int)want.find(lo[j]);
    CTM_CUDA_OK(permute(Cm, out.p, tmp.r, tmp.d, perm, c->cx, false, c->stream, &c->launches));
  }
  c->scratch_off = mark;
  return CTM_OK;
}

// ------------------------------------------------------ enlarged corners
// Q[(t,d,d'),(n,r,r')] = sum C[p,m] Ta[m,n,u,u'] Tb[t,p,l,l'] A[s,u,l,d,r]
// B[s,u',l',d',r'] (paper Eq. rho_M_diag): corner i of the cut whose
// upper-left frame position is (x, y) is this upper-left form applied to the
// tensors turned by i more quarter turns.
ctm_status enlarged_corner(ctm_ctx* c, int r, int i, int x, int y, void* Qout) {
  const long chi = c->chi, Dk = c->Dk, Db = c->Db, d = c->d;
  static const int dx[4] = {0, 1, 1, 0}, dy[4] = {0, 0, 1, 1};
  const int sx = x + dx[i], sy = y + dy[i];
  const int site = frame_site(c, r, sx, sy);
  void* Cc = fC(c, r, i, sx, sy);
  void* Tb = fT(c, r, (i + 3) & 3, sx, sy);
  void* Ta = fT(c, r, i, sx, sy);
  void* A = KETp(c, r + i, site);
  void* B = BRAp(c, r + i, site);
  Tn CT = tn(c->pipe[0], {chi, chi, Dk, Db});
  CK(ein(c, "pm,mnuv->pnuv", tn(Cc, {chi, chi}), false, tn(Ta, {chi, chi, Dk, Db}), false, CT));
  Tn CTT = tn(c->pipe[1], {chi, Dk, Db, chi, Dk, Db});
  CK(ein(c, "tplw,pnuv->tlwnuv", tn(Tb, {chi, chi, Dk, Db}), false, CT, false, CTT));
  if (!c->exact && use_fused_absorb(c->cx, c->split != nullptr, c->opts, (int)Dk, (int)Db, (int)d)) {
    // A and B in one pass over the block (fp32 arithmetic in split contexts)
    CTM_CUDA_OK(absorb_ab(c->cx, c->split != nullptr, (int)chi, (int)Dk, (int)Db, (int)d, CTT.p,
                          A, B, Qout, c->num_sms, c->stream, &c->launches));
    return CTM_OK;
  }
  Tn R1 = tn(c->pipe[0], {chi, Db, chi, Db, d, Dk, Dk});
  CK(ein(c, "tlwnuv,sulde->twnvsde", CTT, false, tn(A, {d, Dk, Dk, Dk, Dk}), false, R1));
  CK(ein(c, "twnvsde,svwDE->tdDneE", R1, false, tn(B, {d, Db, Db, Db, Db}), false,
         tn(Qout, {chi, Dk, Db, chi, Dk, Db})));
  return CTM_OK;
}

// ------------------------------------------------- subspace iteration
// Y = op(Q) Z for an N x N corner and an N x k block.
ctm_status apply_corner(ctm_ctx* c, const void* Qm, bool herm, const void* Zin, void* Zout) {
  PhaseScope ps(c, PH_PROD);
  if (c->split) {
    const int opQ = herm ? (c->cx ? OP_C : OP_T) : OP_N;
    const ctm_status st =
        c->exact ? oz_gemm(c->split, opQ, Qm, c->N, OP_N, Zin, c->k, c->N, c->k, c->N, Zout,
                           c->k, c->stream, &c->launches)
                 : split_apply(c->split, Qm, herm, Zin, Zout, c->N, c->k, c->stream,
                               &c->launches);
    if (st != CTM_OK) return fail(c, st, split_last_error(c->split));
    return CTM_OK;
  }
  GemmDesc g;
  g.opA = herm ? OP_C : OP_N;
  g.opB = OP_N;
  g.M = c->N; g.N = c->k; g.K = c->N;
  g.A = Qm; g.lda = c->N;
  g.B = Zin; g.ldb = c->k;
  g.C = Zout; g.ldc = c->k;
  return gemm(c, g);
}

ctm_status mm_exact(ctm_ctx* c, int opA, int opB, long M, long Nn, long K, const void* A,
                    long lda, const void* B, long ldb, void* Cm, long ldc);

// Orthonormal basis of span(Z) in place (N x k): shifted CholeskyQR followed
// by two CholeskyQR passes (CholeskyQR3, Fukaya et al. 2020). Only the span
// enters the projectors (paper step 1), so R is not kept.
ctm_status qr_inplace(ctm_ctx* c, void* Zm, void* tmp, bool split_mode) {
  PhaseScope ps(c, PH_QR);
  // every pass also finds columns that are numerically in the span of the
  // previous ones (rank-deficient block: D = 1 states, fast decaying
  // spectra) and refills them with pseudo-random directions; such columns
  // carry no information of the block, and the next QR orthonormalises them.
  // Three passes (shifted CholeskyQR3) on the Jacobi-scaled Gram (columns of
  // unit norm; much of the ill-conditioning of M^H M X is column scaling):
  // fp64-accurate Gram (an exact-digit tensor-core product in split
  // contexts), the k x k Cholesky factor on a cluster of eight CTAs, and
  // Q = Z D^-1 L^-H by the fp64 row solve or, in split contexts, as Z times
  // the explicit D^-1 L^-H.
  ++c->qr_calls;
  const bool split = split_mode && c->split != nullptr && !c->exact;
  const int passes = 3;
  const bool smem_chol = chol_smem_bytes(c->cx, c->k) <= (size_t)(226 * 1024);
  for (int pass = 0; pass < passes; ++pass) {
    const int opH = c->cx ? OP_C : OP_T;
    if (split && pass == passes - 1) {
      // last pass of a split context: the block is orthonormal to ~1e-7, so
      // Q <- Q L^-H with L = chol(Q^H Q) = I + F is applied to first order,
      // Q <- Q - Q F^H: the fp64 Gram fixes F, and the small correction
      // Q F^H runs on the tensor cores (its ~1e-7 relative error is ~1e-15
      // of Q)
      GemmDesc g;
      g.opA = opH;
      g.opB = OP_N;
      g.M = c->k; g.N = c->k; g.K = c->N;
      g.A = Zm; g.lda = c->k;
      g.B = Zm; g.ldb = c->k;
      g.C = c->G; g.ldc = c->k;
      g.lower_only = true;
      CK(gemm_exact(c, g));
      CTM_CUDA_OK(orth_correction(c->cx, c->k, c->G, c->Linv, c->stream, &c->launches));
      const ctm_status st = split_gemm(c->split, OP_N, Zm, c->k, OP_N, c->Linv, c->k, c->N, c->k,
                                       c->k, tmp, c->k, c->stream, &c->launches);
      if (st != CTM_OK) return fail(c, st, split_last_error(c->split));
      CTM_CUDA_OK(sub_inplace(c->cx, c->N * c->k, Zm, tmp, c->stream, &c->launches));
      break;
    }
    {
      // the Gram stays fp64: from unsettled rangefinders its columns are
      // nearly parallel and a ~1e-7-accurate Gram would lose the subspace
      GemmDesc g;
      g.opA = opH;
      g.opB = OP_N;
      g.M = c->k; g.N = c->k; g.K = c->N;
      g.A = Zm; g.lda = c->k;
      g.B = Zm; g.ldb = c->k;
      g.C = c->G; g.ldc = c->k;
      g.lower_only = smem_chol;
      CK(gemm_exact(c, g));
    }
    int* dead = c->dead;   // every pass finds and refills dependent columns
    // the k x k factor on a cluster of eight SMs where it fits (chol_cluster.cu),
    // else on one SM (the fp64 pipe of one SM bounds it)
    const bool cl_chol = chol_cluster_supported(c->cx, c->k);
    if (split && smem_chol && pass == 1) {
      // second pass of a split context: the block is already conditioned by
      // the shifted pass, so Q = Z D^-1 L^-H runs on the tensor cores (the
      // explicit k x k inverse replaces the fp64 row solve; its ~1e-7 error
      // is removed by the correction pass that follows)
      if (cl_chol)
        CTM_CUDA_OK(chol_cluster(c->cx, c->k, c->N, false, true, c->G, c->Linv, c->dsc, dead,
                                 c->G, c->err, c->stream, &c->launches));
      else
        CTM_CUDA_OK(chol_factor_inv(c->cx, c->k, c->N, false, true, c->G, c->Linv, c->dsc, dead,
                                    c->G, c->err, c->stream, &c->launches));
      const ctm_status st = split_gemm(c->split, OP_N, Zm, c->k, OP_N, c->G, c->k, c->N, c->k,
                                       c->k, tmp, c->k, c->stream, &c->launches);
      if (st != CTM_OK) return fail(c, st, split_last_error(c->split));
    } else if (smem_chol) {
      // L = chol(D^-1 G D^-1) in shared memory, Q = Z D^-1 L^-H row by row
      if (cl_chol && c->split && c->opts.fp64_tc) {
        // split contexts: the explicit W = D^-1 L^-H (its norm is at most
        // ~shift^-1/2 in the shifted pass) and Q = Z W as an fp64-accurate
        // tensor-core product instead of the fp64 row solve
        CTM_CUDA_OK(chol_cluster(c->cx, c->k, c->N, pass == 0, true, c->G, c->Linv, c->dsc, dead,
                                 c->G, c->err, c->stream, &c->launches));
        CK(mm_exact(c, OP_N, OP_N, c->N, c->k, c->k, Zm, c->k, c->G, c->k, tmp, c->k));
      } else if (cl_chol) {
        CTM_CUDA_OK(chol_cluster(c->cx, c->k, c->N, pass == 0, true, c->G, c->Linv, c->dsc, dead,
                                 nullptr, c->err, c->stream, &c->launches));
        CTM_CUDA_OK(trsm_rows(c->cx, c->k, c->N, c->Linv, c->dsc, Zm, tmp, c->num_sms, c->stream,
                              &c->launches));
      } else {
        CTM_CUDA_OK(chol_qr_pass(c->cx, c->k, c->N, pass == 0, true, c->G, c->Linv, c->dsc, dead,
                                 Zm, tmp, c->err, c->num_sms, c->stream, &c->launches));
      }
    } else if (cl_chol) {
      // the packed factor exceeds one CTA: the row-distributed cluster factor
      // forms W = D^-1 L^-H; Q = Z W (fp64-accurate in the shifted first
      // pass, whose W has norm up to shift^-1/2; split in the second)
      CTM_CUDA_OK(chol_cluster(c->cx, c->k, c->N, pass == 0, true, c->G, c->Linv, c->dsc, dead,
                               c->G, c->err, c->stream, &c->launches));
      if (split && pass > 0) {
        const ctm_status st = split_gemm(c->split, OP_N, Zm, c->k, OP_N, c->G, c->k, c->N, c->k,
                                         c->k, tmp, c->k, c->stream, &c->launches);
        if (st != CTM_OK) return fail(c, st, split_last_error(c->split));
      } else {
        CK(mm_exact(c, OP_N, OP_N, c->N, c->k, c->k, Zm, c->k, c->G, c->k, tmp, c->k));
      }
    } else {
      CTM_CUDA_OK(chol_inv_coop(c->cx, c->k, c->N, pass == 0, true, c->G, c->Linv, 1, dead,
                                c->chol_work, c->err, c->num_sms, c->stream, &c->launches));
      // the shifted first pass multiplies by an inverse of norm up to
      // shift^-1/2 (~1e4): it stays fp64; the conditioned second pass may
      // run on the tensor cores
      if (split && pass > 0) {
        const ctm_status st = split_gemm(c->split, OP_N, Zm, c->k, opH, c->Linv, c->k, c->N, c->k,
                                         c->k, tmp, c->k, c->stream, &c->launches);
        if (st != CTM_OK) return fail(c, st, split_last_error(c->split));
      } else {
        GemmDesc h;
        h.opA = OP_N;
        h.opB = opH;
        h.M = c->N; h.N = c->k; h.K = c->k;
        h.A = Zm; h.lda = c->k;
        h.B = c->Linv; h.ldb = c->k;
        h.C = tmp; h.ldc = c->k;
        CK(gemm(c, h));
      }
    }
    CTM_CUDA_OK(repair_dead_columns(c->cx, c->N, c->k, tmp, c->dead,
                                    (c->opts.seed * 1000003ull + c->qr_calls) * 4 + pass,
                                    c->stream, &c->launches));
    CTM_CUDA_OK(cudaMemcpyAsync(Zm, tmp, (size_t)c->N * c->k * c->es, cudaMemcpyDeviceToDevice,
                                c->stream));
  }
  return CTM_OK;
}

ctm_status mm_small(ctm_ctx* c, int opA, int opB, long M, long Nn, long K, const void* A,
                    long lda, const void* B, long ldb, void* Cm, long ldc) {
  GemmDesc g;
  g.opA = opA; g.opB = opB;
  g.M = M; g.N = Nn; g.K = K;
  g.A = A; g.lda = lda;
  g.B = B; g.ldb = ldb;
  g.C = Cm; g.ldc = ldc;
  return gemm(c, g);
}

ctm_status mm_exact(ctm_ctx* c, int opA, int opB, long M, long Nn, long K, const void* A,
                    long lda, const void* B, long ldb, void* Cm, long ldc) {
  GemmDesc g;
  g.opA = opA; g.opB = opB;
  g.M = M; g.N = Nn; g.K = K;
  g.A = A; g.lda = lda;
  g.B = B; g.ldb = ldb;
  g.C = Cm; g.ldc = ldc;
  return gemm_exact(c, g);
}

// SI projectors of one cut (paper "QR-based projector", steps 1-4), first
// half: rounds of X <- qr(M^H M X), W <- qr(M M^H W) with M = Q3 Q4 Q1 Q2
// applied one corner at a time; Z_R = Q1 Q2 X and Z_L = (Q3 Q4)^H W into
// slot y, rho = Z_L^H Z_R (Eq. rho_hat_diag) into slot y. The small SVDs of
// all cuts of a column then run as one batched launch (si_small_svd), and
// si_finish builds the projectors.
ctm_status si_rho(ctm_ctx* c, int r, int cut, int y) {
  const size_t Nk = (size_t)c->N * c->k;
  void* X = at(c->X, (size_t)(r * c->S + cut) * Nk, c);
  void* W = at(c->W, (size_t)(r * c->S + cut) * Nk, c);
  void** Q = c->Q;
  void** Z = c->Z;
  char& ready = c->rf_ready[r * c->S + cut];
  const bool warm = c->moves_done[r] < c->opts.warmup_iters;
  if (warm && c->opts.warmup_rsvd) {
    // randomized-SVD warm-up: every warm-up move starts from the initial
    // random blocks, not from the recycled bases
    CTM_CUDA_OK(cudaMemcpyAsync(X, at(c->Xraw, (size_t)(r * c->S + cut) * Nk, c), Nk * c->es,
                                cudaMemcpyDeviceToDevice, c->stream));
    CTM_CUDA_OK(cudaMemcpyAsync(W, at(c->Wraw, (size_t)(r * c->S + cut) * Nk, c), Nk * c->es,
                                cudaMemcpyDeviceToDevice, c->stream));
    ready = 0;
  }
  if (!ready) {
    CK(qr_inplace(c, X, Z[0], false));
    CK(qr_inplace(c, W, Z[0], false));
    ready = 1;
  }
  const int rc = r * c->S + cut;
  // recycling policy (paper step 4): a cut whose leading subspace stopped
  // moving only recycles its bases, with no update round
  const int rounds = warm ? c->opts.warmup_rounds
                          : (c->si_skip[rc] ? 0 : c->opts.si_rounds);
  c->si_rounds_used[rc] = rounds > 0;
  if (rounds > 0) {
    ++c->si_updates[rc];
    ++c->n_updates;
  } else {
    ++c->n_skipped;
  }
  const bool track = c->opts.recycle_sin2 > 0.0;
  if (track && rounds > 0)
    CTM_CUDA_OK(cudaMemcpyAsync(Z[3], X, Nk * c->es, cudaMemcpyDeviceToDevice, c->stream));
  // fp64 QR schedule in fp64 contexts and during warm-up, split afterwards
  const bool split_qr = c->split != nullptr && !c->exact && !warm;
  // fp64: a QR after each application of M or M^H (the span of M^H M X
  // without squaring cond(M)); split: one QR per update on the Jacobi-scaled
  // block (the products themselves carry ~1e-7 errors)
  const bool qr_each = !split_qr;
  for (int round = 0; round < rounds && c->opts.si_coupled; ++round) {
    // coupled (Halko) round: W <- qr(M X), X <- qr(M^H W)
    CK(apply_corner(c, Q[1], false, X, Z[0]));
    CK(apply_corner(c, Q[0], false, Z[0], Z[1]));
    CK(apply_corner(c, Q[3], false, Z[1], Z[0]));
    CK(apply_corner(c, Q[2], false, Z[0], W));
    CK(qr_inplace(c, W, Z[0], split_qr));
    CK(apply_corner(c, Q[2], true, W, Z[0]));
    CK(apply_corner(c, Q[3], true, Z[0], Z[1]));
    CK(apply_corner(c, Q[0], true, Z[1], Z[0]));
    CK(apply_corner(c, Q[1], true, Z[0], X));
    CK(qr_inplace(c, X, Z[0], split_qr));
  }
  for (int round = 0; round < rounds && !c->opts.si_coupled; ++round) {
    // X <- qr(M^H M X)
    CK(apply_corner(c, Q[1], false, X, Z[0]));
    CK(apply_corner(c, Q[0], false, Z[0], Z[1]));
    CK(apply_corner(c, Q[3], false, Z[1], Z[0]));
    CK(apply_corner(c, Q[2], false, Z[0], Z[1]));
    if (qr_each) CK(qr_inplace(c, Z[1], Z[0], false));
    CK(apply_corner(c, Q[2], true, Z[1], Z[0]));
    CK(apply_corner(c, Q[3], true, Z[0], Z[2]));
    CK(apply_corner(c, Q[0], true, Z[2], Z[0]));
    CK(apply_corner(c, Q[1], true, Z[0], X));
    CK(qr_inplace(c, X, Z[0], split_qr));
    // W <- qr(M qr(M^H W))
    CK(apply_corner(c, Q[2], true, W, Z[0]));
    CK(apply_corner(c, Q[3], true, Z[0], Z[1]));
    CK(apply_corner(c, Q[0], true, Z[1], Z[0]));
    CK(apply_corner(c, Q[1], true, Z[0], Z[1]));
    if (qr_each) CK(qr_inplace(c, Z[1], Z[0], false));
    CK(apply_corner(c, Q[1], false, Z[1], Z[0]));
    CK(apply_corner(c, Q[0], false, Z[0], Z[2]));
    CK(apply_corner(c, Q[3], false, Z[2], Z[0]));
    CK(apply_corner(c, Q[2], false, Z[0], W));
    CK(qr_inplace(c, W, Z[0], split_qr));
  }
  if (track && rounds > 0) {
    // overlap of the bases before and after the update, for the principal
    // angles of the recycling policy
    const int opH0 = c->cx ? OP_C : OP_T;
    CK(mm_small(c, opH0, OP_N, c->k, c->k, c->N, Z[3], c->k, X, c->k,
                at(c->sinG, (size_t)y * c->k * c->k, c), c->k));
  }
  // Z_R = Q1 (Q2 X), Z_L = Q4^H (Q3^H W)
  void* ZR = at(c->ZR, y * Nk, c);
  void* ZL = at(c->ZL, y * Nk, c);
  CK(apply_corner(c, Q[1], false, X, Z[0]));
  CK(apply_corner(c, Q[0], false, Z[0], ZR));
  CK(apply_corner(c, Q[2], true, W, Z[0]));
  CK(apply_corner(c, Q[3], true, Z[0], ZL));
  const int k = c->k;
  const int opH = c->cx ? OP_C : OP_T;
  PhaseScope ps(c, PH_SMALL);
  CK(mm_exact(c, opH, OP_N, k, k, c->N, ZL, k, ZR, k, at(c->rho, (size_t)y * k * k, c), k));
  return CTM_OK;
}

// Batched m x m products C[i] = alpha op(A[i]) B[i] in fp64 (A[i] at stride
// sA elements, B and C contiguous).
ctm_status mm_batched(ctm_ctx* c, int m, int opA, int n, const void* A, long sA, const void* B,
                      void* Cm, double alpha) {
  GemmDesc g;
  g.opA = opA;
  g.opB = OP_N;
  g.M = m; g.N = m; g.K = m;
  g.A = A; g.lda = m; g.strideA = sA;
  g.B = B; g.ldb = m; g.strideB = (long)m * m;
  g.C = Cm; g.ldc = m; g.strideC = (long)m * m;
  g.alpha[0] = alpha;
  g.batch = n;
  return gemm(c, g);
}

// fp32 pre-solve of n m x m matrices A (stride sA): the one-sided Jacobi in
// fp32 (jacobi32.cu) gives the right rotations V0, two Newton-Schulz steps
// V <- V (3 I - V^H V) / 2 make them unitary in fp64 (each squares the
// distance from unitarity: ~1e-6 -> ~1e-12 -> rounding), and B = A V0
// (into c->jB) has columns that are already nearly orthogonal. The fp64
// one-sided Jacobi of B from V0 is then the SVD of A.
ctm_status svd_presolve(ctm_ctx* c, int m, int n, const void* A, long sA, const void** V0) {
  CTM_CUDA_OK(jacobi32_presolve(c->cx, m, A, sA, c->jv0, n, 40, nullptr, c->stream,
                                &c->launches));
  void* V = c->jv0;
  void* Vn = c->jv1;
  const int opH = c->cx ? OP_C : OP_T;
  const long mm = (long)m * m;
  for (int it = 0; it < 2; ++it) {
    CK(mm_batched(c, m, opH, n, V, mm, V, c->jT, -0.5));
    CTM_CUDA_OK(add_identity(c->cx, m, c->jT, 1.5, n, c->stream, &c->launches));
    CK(mm_batched(c, m, OP_N, n, V, mm, c->jT, Vn, 1.0));
    std::swap(V, Vn);
  }
  CK(mm_batched(c, m, OP_N, n, A, sA, V, c->jB, 1.0));
  *V0 = V;
  return CTM_OK;
}

bool use_presolve(const ctm_ctx* c, int m) {
  return c->opts.svd_presolve && jacobi32_supported(c->cx, m);
}

// rho = u s v^H for the slots 0 .. n-1 in one cooperative launch (after the
// fp32 pre-solve with opts.svd_presolve).
ctm_status si_small_svd(ctm_ctx* c, int n) {
  PhaseScope ps(c, PH_SMALL);
  const int k = c->k;
  const void* A = c->rho;
  const void* Vinit = nullptr;
  if (use_presolve(c, k)) {
    CK(svd_presolve(c, k, n, c->rho, (long)k * k, &Vinit));
    A = c->jB;
  }
  CTM_CUDA_OK(jacobi_svd_coop(c->cx, k, A, (long)k * k, c->sv, c->u, c->v, true, c->jw, n,
                              c->opts.svd_max_sweeps, c->err, c->num_sms, c->stream, &c->launches,
                              Vinit));
  return CTM_OK;
}

// Second half for slot y: sign fix (step 4), recycling X <- X v, W <- W u
// (Eq. xy_recycle), P_l = Z_R v_chi s^-1/2, P_r^H = Z_L u_chi s^-1/2
// (Eq. projectors_diag).
ctm_status si_finish(ctm_ctx* c, int r, int cut, int y, void* Pl, void* PrH) {
  const size_t Nk = (size_t)c->N * c->k;
  const int k = c->k, chi = c->chi;
  void* X = at(c->X, (size_t)(r * c->S + cut) * Nk, c);
  void* W = at(c->W, (size_t)(r * c->S + cut) * Nk, c);
  void* ZR = at(c->ZR, y * Nk, c);
  void* ZL = at(c->ZL, y * Nk, c);
  void* u = at(c->u, (size_t)y * k * k, c);
  void* v = at(c->v, (size_t)y * k * k, c);
  const double* sv = c->sv + (size_t)y * k;
  PhaseScope ps(c, PH_SMALL);
  if (c->opts.sign_fix) {
    // sign fix of the small SVD (step 4): largest-modulus entry of each
    // column of u real positive, v_i takes the same phase
    CTM_CUDA_OK(column_phase(c->cx, k, k, k, u, c->ph, 1, 0, c->stream, &c->launches));
    CTM_CUDA_OK(scale_columns_conj(c->cx, k, k, k, u, c->ph, c->stream, &c->launches));
    CTM_CUDA_OK(scale_columns_conj(c->cx, k, k, k, v, c->ph, c->stream, &c->launches));
  }
  // recycled bases X v, W u: the next update re-orthonormalises them, so in
  // split contexts they run on the tensor cores
  if (c->split && !c->exact) {
    ctm_status st = split_gemm(c->split, OP_N, X, k, OP_N, v, k, (int)c->N, k, k, c->Xn, k,
                               c->stream, &c->launches);
    if (st == CTM_OK)
      st = split_gemm(c->split, OP_N, W, k, OP_N, u, k, (int)c->N, k, k, c->Wn, k, c->stream,
                      &c->launches);
    if (st != CTM_OK) return fail(c, st, split_last_error(c->split));
  } else {
    CK(mm_small(c, OP_N, OP_N, c->N, k, k, X, k, v, k, c->Xn, k));
    CK(mm_small(c, OP_N, OP_N, c->N, k, k, W, k, u, k, c->Wn, k));
  }
  if (c->opts.recycle_sin2 > 0.0) {
    // mean sin^2 of the principal angles between the leading chi-subspaces
    // of the bases before (X_old) and after (X_upd v) this move:
    // 1 - ||(X_old^H X_upd v)[:chi, :chi]||_F^2 / chi, with X_old = X_upd when
    // the move made no update round
    const int rc = r * c->S + cut;
    const void* Gv = v;
    if (c->si_rounds_used[rc]) {
      CK(mm_small(c, OP_N, OP_N, k, k, k, at(c->sinG, (size_t)y * k * k, c), k, v, k, c->G, k));
      Gv = c->G;
    }
    CTM_CUDA_OK(mean_sin2(c->cx, k, chi, Gv, c->dsin2 + rc, c->stream, &c->launches));
  }
  CTM_CUDA_OK(scale_by_inv_sqrt(c->cx, k, chi, v, sv, c->opts.svd_rel_cutoff, c->Vs,
                                c->stream, &c->launches));
  CTM_CUDA_OK(scale_by_inv_sqrt(c->cx, k, chi, u, sv, c->opts.svd_rel_cutoff, c->Us,
                                c->stream, &c->launches));
  CK(mm_exact(c, OP_N, OP_N, c->N, chi, k, ZR, k, c->Vs, chi, Pl, chi));
  CK(mm_exact(c, OP_N, OP_N, c->N, chi, k, ZL, k, c->Us, chi, PrH, chi));
  CTM_CUDA_OK(cudaMemcpyAsync(X, c->Xn, Nk * c->es, cudaMemcpyDeviceToDevice, c->stream));
  CTM_CUDA_OK(cudaMemcpyAsync(W, c->Wn, Nk * c->es, cudaMemcpyDeviceToDevice, c->stream));
  return CTM_OK;
}

// -------------------------------------------------------------- absorb
// New C1, T4, C4 of column x+1 (End Matter, left move): C1' = P_r (C1 T1)
// with the projector of the cut above, C4' = (T3 C4) P_l with the one below,
// T4' = P_r (T4 A B) P_l with the cut below (P_r) and above (P_l).
ctm_status absorb_site(ctm_ctx* c, int r, int x, int y, int Lyf) {
  const long chi = c->chi, Dk = c->Dk, Db = c->Db, d = c->d;
  const size_t NC = (size_t)c->N * c->chi;
  const int up = (y - 1 + Lyf) % Lyf, dn = y;
  void* PrH_up = at(c->PrH, up * NC, c);
  void* Pl_up = at(c->Pl, up * NC, c);
  void* PrH_dn = at(c->PrH, dn * NC, c);
  void* Pl_dn = at(c->Pl, dn * NC, c);
  const int site = frame_site(c, r, x, y);
  void* C1 = fC(c, r, 0, x, y);
  void* T1 = fT(c, r, 0, x, y);
  void* T3 = fT(c, r, 2, x, y);
  void* C4 = fC(c, r, 3, x, y);
  void* T4 = fT(c, r, 3, x, y);
  void* A = KETp(c, r, site);
  void* B = BRAp(c, r, site);
  void* oC1 = at(c->stC1, (size_t)y * elems_C(c), c);
  void* oC4 = at(c->stC4, (size_t)y * elems_C(c), c);
  void* oT4 = at(c->stT4, (size_t)y * elems_T(c), c);
  // C1'
  Tn E1 = tn(c->pipe[0], {chi, chi, Dk, Db});
  CK(ein(c, "pm,mnuv->pnuv", tn(C1, {chi, chi}), false, tn(T1, {chi, chi, Dk, Db}), false, E1));
  CK(ein(c, "puva,pnuv->an", tn(PrH_up, {chi, Dk, Db, chi}), true, E1, false,
         tn(oC1, {chi, chi})));
  // C4'
  Tn E4 = tn(c->pipe[0], {chi, chi, Dk, Db});
  CK(ein(c, "tmdD,mn->tndD", tn(T3, {chi, chi, Dk, Db}), false, tn(C4, {chi, chi}), false, E4));
  CK(ein(c, "tndD,ndDc->tc", E4, false, tn(Pl_dn, {chi, Dk, Db, chi}), false,
         tn(oC4, {chi, chi})));
  // T4'
  if (!c->exact && use_fused_absorb(c->cx, c->split != nullptr, c->opts, (int)Dk, (int)Db, (int)d)) {
    Tn Y1 = tn(c->pipe[0], {chi, Dk, Db, chi, Dk, Db});
    CK(ein(c, "tqlw,quvc->tlwcuv", tn(T4, {chi, chi, Dk, Db}), false,
           tn(Pl_up, {chi, Dk, Db, chi}), false, Y1));
    Tn R2 = tn(c->pipe[1], {chi, Dk, Db, chi, Dk, Db});
    CTM_CUDA_OK(absorb_ab(c->cx, c->split != nullptr, (int)chi, (int)Dk, (int)Db, (int)d, Y1.p, A,
                          B, R2.p, c->num_sms, c->stream, &c->launches));
    CK(ein(c, "tdDa,tdDceE->aceE", tn(PrH_dn, {chi, Dk, Db, chi}), true, R2, false,
           tn(oT4, {chi, chi, Dk, Db})));
    return CTM_OK;
  }
  Tn Y1 = tn(c->pipe[0], {chi, Dk, Db, Dk, Db, chi});
  CK(ein(c, "tqlw,quvc->tlwuvc", tn(T4, {chi, chi, Dk, Db}), false,
         tn(Pl_up, {chi, Dk, Db, chi}), false, Y1));
  Tn R1 = tn(c->pipe[1], {chi, Db, Db, chi, d, Dk, Dk});
  CK(ein(c, "tlwuvc,sulde->twvcsde", Y1, false, tn(A, {d, Dk, Dk, Dk, Dk}), false, R1));
  Tn R2 = tn(c->pipe[0], {chi, Dk, Db, chi, Dk, Db});
  CK(ein(c, "twvcsde,svwDE->tdDceE", R1, false, tn(B, {d, Db, Db, Db, Db}), false, R2));
  CK(ein(c, "tdDa,tdDceE->aceE", tn(PrH_dn, {chi, Dk, Db, chi}), true, R2, false,
         tn(oT4, {chi, chi, Dk, Db})));
  return CTM_OK;
}

// C = op(A) op(B) for the large products of the standard-SVD path: the
// tensor cores in split contexts (exact digits during the refinement), fp64
// otherwise
ctm_status mm_big(ctm_ctx* c, int opA, int opB, long M, long Nn, long K, const void* A, long lda,
                  const void* B, long ldb, void* Cm, long ldc) {
  if (c->split) {
    const ctm_status st =
        c->exact ? oz_gemm(c->split, opA, A, lda, opB, B, ldb, (int)M, (int)Nn, (int)K, Cm, ldc,
                           c->stream, &c->launches)
                 : split_gemm(c->split, opA, A, lda, opB, B, ldb, (int)M, (int)Nn, (int)K, Cm,
                              ldc, c->stream, &c->launches);
    return st == CTM_OK ? CTM_OK : fail(c, st, split_last_error(c->split));
  }
  return mm_small(c, opA, opB, M, Nn, K, A, lda, B, ldb, Cm, ldc);
}

// Standard CTMRG projectors of one cut (Eq. svd_projectors_diag): H_R = Q1 Q2,
// H_L = Q3 Q4, M = H_L H_R = U S V^H truncated to chi (sign fix on U),
// P_l = H_R V s^-1/2, P_r^H = H_L^H U s^-1/2.
ctm_status svd_projectors(ctm_ctx* c, void* Pl, void* PrH) {
  const long N = c->N, chi = c->chi;
  void* HR = c->pipe[0];
  void* HL = c->pipe[1];
  PhaseScope ps(c, PH_SMALL);
  CK(mm_big(c, OP_N, OP_N, N, N, N, c->Q[0], N, c->Q[1], N, HR, N));
  CK(mm_big(c, OP_N, OP_N, N, N, N, c->Q[2], N, c->Q[3], N, HL, N));
  CK(mm_big(c, OP_N, OP_N, N, N, N, HL, N, HR, N, c->svdM, N));
  const ctm_status st = svd_truncated(c->svd, c->svdM, (int)chi, c->opts.svd_rel_cutoff,
                                      c->opts.sign_fix != 0, c->svdUs, c->svdVs, c->err,
                                      c->stream, &c->launches);
  if (st != CTM_OK) return fail(c, st, svd_last_error(c->svd));
  CK(mm_big(c, OP_N, OP_N, N, chi, N, HR, N, c->svdVs, chi, Pl, chi));
  CK(mm_big(c, c->cx ? OP_C : OP_T, OP_N, N, chi, N, HL, N, c->svdUs, chi, PrH, chi));
  return CTM_OK;
}

ctm_status check_err(ctm_ctx* c) {
  int h = 0;
  CTM_CUDA_OK(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CTM_CUDA_OK(cudaStreamSynchronize(c->stream));
  if (h) {
    CTM_CUDA_OK(cudaMemsetAsync(c->err, 0, sizeof(int), c->stream));
    if (h & DEV_CHOL_PIVOT) return fail(c, CTM_ENUMERIC, "non-positive Cholesky pivot in CholeskyQR");
    if (h & DEV_NONFINITE) return fail(c, CTM_ENUMERIC, "non-finite value in the small SVD");
    if (h & DEV_MBAR_TIMEOUT) return fail(c, CTM_ETIMEOUT, "tensor-core pipeline wait gave up");
    if (h & DEV_JACOBI_NOCONV) return fail(c, CTM_ENOCONV, "Jacobi SVD sweep budget exhausted");
  }
  return CTM_OK;
}

ctm_status move_impl(ctm_ctx* c, int r) {
  CK(grad_checkpoint(c, r));
  c->spectra_fresh = false;
  const int Lxf = (r & 1) ? c->Ly : c->Lx, Lyf = (r & 1) ? c->Lx : c->Ly;
  const size_t NC = (size_t)c->N * c->chi;
  const bool svd = c->opts.method == CTM_PROJ_SVD;
  std::vector<char> prefetched(Lyf, 0);
  for (int x = 0; x < Lxf; ++x) {
    if (svd) {
      for (int y = 0; y < Lyf; ++y) {
        {
          PhaseScope ps(c, PH_CORNER);
          for (int i = 0; i < 4; ++i) CK(enlarged_corner(c, r, i, x, y, c->Q[i]));
        }
        const int cut = y * Lxf + x;
        CK(svd_projectors(c, at(c->Pl, y * NC, c), at(c->PrH, y * NC, c)));
        CTM_CUDA_OK(cudaMemcpyAsync(at(c->lastPl, cut * NC, c), at(c->Pl, y * NC, c),
                                    NC * c->es, cudaMemcpyDeviceToDevice, c->stream));
        CTM_CUDA_OK(cudaMemcpyAsync(at(c->lastPrH, cut * NC, c), at(c->PrH, y * NC, c),
                                    NC * c->es, cudaMemcpyDeviceToDevice, c->stream));
      }
    }
    // the cuts of the column run on lanes 1 .. nw (round robin), after the
    // previous column's absorption on lane 0
    const int nl = svd ? 1 : std::max<int>(1, (int)c->lanes.size());
    const int nw = nl - 1;
    auto lane_of = [&](int y) { return nw > 0 ? 1 + y % nw : 0; };
    LaneReset lane_reset{c};
    if (nw > 0) {
      CTM_CUDA_OK(cudaEventRecord(c->lanes[0].ev, c->lanes[0].stream));
      for (int l = 1; l < nl; ++l)
        CTM_CUDA_OK(cudaStreamWaitEvent(c->lanes[l].stream, c->lanes[0].ev, 0));
    }
    for (int y = 0; y < (svd ? 0 : Lyf); ++y) {
      use_lane(c, lane_of(y));
      const bool pre = prefetched[y] != 0;   // Q2, Q3 already built and sliced
      {
        PhaseScope ps(c, PH_CORNER);
        for (int i = 0; i < 4; ++i)
          if (!(pre && (i == 1 || i == 2))) CK(enlarged_corner(c, r, i, x, y, c->Q[i]));
      }
      if (c->split && !c->exact) {
        PhaseScope ps(c, PH_SLICE);
        const ctm_status st = split_prepare_corners(c->split, c->Q, c->N, pre ? 0x9u : 0xFu,
                                                    c->stream, &c->launches);
        if (st != CTM_OK) return fail(c, st, split_last_error(c->split));
      }
      prefetched[y] = 0;
      CK(si_rho(c, r, y * Lxf + x, y));
    }
    use_lane(c, 0);
    if (nw > 0) {
      for (int l = 1; l < nl; ++l) {
        CTM_CUDA_OK(cudaEventRecord(c->lanes[l].ev, c->lanes[l].stream));
        CTM_CUDA_OK(cudaStreamWaitEvent(c->lanes[0].stream, c->lanes[l].ev, 0));
      }
      // Q2 and Q3 of the next column's cuts sit two columns to the right of
      // this one, which this column's absorption does not touch (Lxf >= 2):
      // the lanes build and slice them while lane 0 finishes this column
      if (!svd && x + 1 < Lxf && Lxf >= 2) {
        for (int y = 0; y < Lyf; ++y) {
          use_lane(c, lane_of(y));
          {
            PhaseScope ps(c, PH_CORNER);
            CK(enlarged_corner(c, r, 1, x + 1, y, c->Q[1]));
            CK(enlarged_corner(c, r, 2, x + 1, y, c->Q[2]));
          }
          if (c->split && !c->exact) {
            PhaseScope ps(c, PH_SLICE);
            const ctm_status st =
                split_prepare_corners(c->split, c->Q, c->N, 0x6u, c->stream, &c->launches);
            if (st != CTM_OK) return fail(c, st, split_last_error(c->split));
          }
          prefetched[y] = 1;
        }
        use_lane(c, 0);
      }
    }
    // the cuts of a column are independent until the absorption: their
    // small SVDs share one launch
    if (!svd) CK(si_small_svd(c, Lyf));
    // the projector step of each cut (recycled bases, P_l, P_r^H) runs on the
    // cut's lane once the batched SVD is done; lane 0 absorbs after all of them
    if (!svd && nw > 0) {
      CTM_CUDA_OK(cudaEventRecord(c->lanes[0].ev, c->lanes[0].stream));
      for (int l = 1; l < nl; ++l)
        CTM_CUDA_OK(cudaStreamWaitEvent(c->lanes[l].stream, c->lanes[0].ev, 0));
    }
    for (int y = 0; y < (svd ? 0 : Lyf); ++y) {
      const int cut = y * Lxf + x;
      use_lane(c, lane_of(y));
      CK(si_finish(c, r, cut, y, at(c->Pl, y * NC, c), at(c->PrH, y * NC, c)));
      CTM_CUDA_OK(cudaMemcpyAsync(at(c->lastPl, cut * NC, c), at(c->Pl, y * NC, c), NC * c->es,
                                  cudaMemcpyDeviceToDevice, c->stream));
      CTM_CUDA_OK(cudaMemcpyAsync(at(c->lastPrH, cut * NC, c), at(c->PrH, y * NC, c),
                                  NC * c->es, cudaMemcpyDeviceToDevice, c->stream));
    }
    // the absorption of site y uses the projectors of cuts y and y - 1: every
    // lane waits for all projector steps, then absorbs its own sites
    if (!svd && nw > 0) {
      for (int l = 1; l < nl; ++l)
        CTM_CUDA_OK(cudaEventRecord(c->lanes[l].ev, c->lanes[l].stream));
      for (int l = 1; l < nl; ++l)
        for (int m = 1; m < nl; ++m)
          if (m != l) CTM_CUDA_OK(cudaStreamWaitEvent(c->lanes[l].stream, c->lanes[m].ev, 0));
    }
    for (int y = 0; y < Lyf; ++y) {
      use_lane(c, svd ? 0 : lane_of(y));
      PhaseScope ps(c, PH_ABSORB);
      CK(absorb_site(c, r, x, y, Lyf));
    }
    use_lane(c, 0);
    if (!svd && nw > 0)
      for (int l = 1; l < nl; ++l) {
        CTM_CUDA_OK(cudaEventRecord(c->lanes[l].ev, c->lanes[l].stream));
        CTM_CUDA_OK(cudaStreamWaitEvent(c->lanes[0].stream, c->lanes[l].ev, 0));
      }
    PhaseScope psn(c, PH_NORM);
    if (c->opts.normalize) {
      const size_t mark = c->scratch_off;
      void* w = scratch_alloc(c, (size_t)3 * 152 * Lyf * sizeof(double));
      if (!w) return fail(c, CTM_ENOMEM, "scratch arena too small for the norms");
      CTM_CUDA_OK(normalize_phase(c->cx, elems_C(c), c->stC1, elems_C(c), Lyf, c->fac, w,
                                  c->stream, &c->launches));
      CTM_CUDA_OK(normalize_phase(c->cx, elems_C(c), c->stC4, elems_C(c), Lyf, c->fac, w,
                                  c->stream, &c->launches));
      CTM_CUDA_OK(normalize_phase(c->cx, elems_T(c), c->stT4, elems_T(c), Lyf, c->fac, w,
                                  c->stream, &c->launches));
      c->scratch_off = mark;
    }
    for (int y = 0; y < Lyf; ++y) {
      CTM_CUDA_OK(cudaMemcpyAsync(fC(c, r, 0, x + 1, y), at(c->stC1, y * elems_C(c), c),
                                  elems_C(c) * c->es, cudaMemcpyDeviceToDevice, c->stream));
      CTM_CUDA_OK(cudaMemcpyAsync(fT(c, r, 3, x + 1, y), at(c->stT4, y * elems_T(c), c),
                                  elems_T(c) * c->es, cudaMemcpyDeviceToDevice, c->stream));
      CTM_CUDA_OK(cudaMemcpyAsync(fC(c, r, 3, x + 1, y), at(c->stC4, y * elems_C(c), c),
                                  elems_C(c) * c->es, cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  c->moves_done[r] += 1;
  c->last_dir = r;
  return CTM_OK;
}

ctm_status corner_spectra(ctm_ctx* c, double* out) {
  PhaseScope ps(c, PH_SPECTRA);
  // unnormalised singular values of all 4 S corners, [label][site][chi]
  const void* A = c->C;
  long sA = (long)elems_C(c);
  if (use_presolve(c, c->chi)) {
    const void* V0 = nullptr;
    CK(svd_presolve(c, c->chi, 4 * (int)c->S, c->C, sA, &V0));
    A = c->jB;
    sA = (long)c->chi * c->chi;
  }
  CTM_CUDA_OK(jacobi_svd_coop(c->cx, c->chi, A, sA, out, nullptr, nullptr,
                              false, c->jw, 4 * c->S, c->opts.svd_max_sweeps, c->err, c->num_sms, c->stream,
                              &c->launches));
  return CTM_OK;
}

void fill_normal(std::vector<double>& v, uint64_t seed, uint64_t stream_id, double scale) {
  // splitmix64 counter stream -> Box-Muller normals (default initial state)
  uint64_t ctr = seed * 0x9E3779B97F4A7C15ull + stream_id * 0xD1B54A32D192ED03ull;
  auto next = [&]() {
    uint64_t z = (ctr += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  for (size_t i = 0; i < v.size(); i += 2) {
    const double u1 = next(), u2 = next();
    const double rr = std::sqrt(-2.0 * std::log(u1));
    v[i] = rr * std::cos(6.283185307179586 * u2) * scale;
    if (i + 1 < v.size()) v[i + 1] = rr * std::sin(6.283185307179586 * u2) * scale;
  }
}

// Forget the recycling history (new rangefinders): every cut updates again.
ctm_status reset_recycling(ctm_ctx* c) {
  std::fill(c->si_updates.begin(), c->si_updates.end(), 0);
  std::fill(c->si_skip.begin(), c->si_skip.end(), 0);
  std::vector<double> one(4 * c->S, 1.0);
  if (c->dsin2)
    CTM_CUDA_OK(cudaMemcpyAsync(c->dsin2, one.data(), one.size() * sizeof(double),
                                cudaMemcpyHostToDevice, c->stream));
  CTM_CUDA_OK(cudaStreamSynchronize(c->stream));
  return CTM_OK;
}

// the initial raw blocks, kept for the randomized-SVD warm-up
ctm_status keep_raw_rangefinders(ctm_ctx* c) {
  if (!c->Xraw) return CTM_OK;
  const size_t n = (size_t)4 * c->S * c->N * c->k * c->es;
  CTM_CUDA_OK(cudaMemcpyAsync(c->Xraw, c->X, n, cudaMemcpyDeviceToDevice, c->stream));
  CTM_CUDA_OK(cudaMemcpyAsync(c->Wraw, c->W, n, cudaMemcpyDeviceToDevice, c->stream));
  return CTM_OK;
}

ctm_status upload_default_state(ctm_ctx* c) {
  const size_t per = c->cx ? 2 : 1;
  const double sc = c->cx ? std::sqrt(0.5) : 1.0;
  std::vector<double> h;
  // corners and edges, each normalised to unit Frobenius norm
  for (int kind = 0; kind < 2; ++kind) {
    const size_t n = kind == 0 ? elems_C(c) : elems_T(c);
    h.assign(n * per * 4 * c->S, 0.0);
    fill_normal(h, c->opts.seed, 1 + kind, sc);
    for (int t = 0; t < 4 * c->S; ++t) {
      double s2 = 0.0;
      for (size_t i = 0; i < n * per; ++i) s2 += h[t * n * per + i] * h[t * n * per + i];
      const double inv = 1.0 / std::sqrt(s2);
      for (size_t i = 0; i < n * per; ++i) h[t * n * per + i] *= inv;
    }
    CTM_CUDA_OK(cudaMemcpyAsync(kind == 0 ? c->C : c->T, h.data(), h.size() * sizeof(double),
                                cudaMemcpyHostToDevice, c->stream));
  }
  const size_t nrf = (size_t)4 * c->S * c->N * c->k * per;
  h.assign(nrf, 0.0);
  fill_normal(h, c->opts.seed, 3, sc);
  CTM_CUDA_OK(cudaMemcpyAsync(c->X, h.data(), nrf * sizeof(double), cudaMemcpyHostToDevice,
                              c->stream));
  fill_normal(h, c->opts.seed, 4, sc);
  CTM_CUDA_OK(cudaMemcpyAsync(c->W, h.data(), nrf * sizeof(double), cudaMemcpyHostToDevice,
                              c->stream));
  CK(keep_raw_rangefinders(c));
  std::fill(c->rf_ready.begin(), c->rf_ready.end(), 0);
  c->spectra_init = false;
  c->spectra_fresh = false;
  for (int r = 0; r < 4; ++r) c->moves_done[r] = 0;
  return reset_recycling(c);
}

// Initial environment from the on-site tensors (init_mode CTM_INIT_FROM_A):
// corner i of a site is the double layer of the site's tensor turned by i
// quarter turns with its up and left bond pairs traced, as a (d d') x (r r')
// matrix; edge i the double layer of the turned tensor with its up pair
// traced, [(l l')][(r r')][d][d']; both embedded in (or cut to) the
// top-left block of the chi bonds, then normalised like a move's output.
ctm_status init_env_from_tensors(ctm_ctx* c) {
  const long chi = c->chi, Dk = c->Dk, Db = c->Db, d = c->d, DD = Dk * Db;
  const long m = std::min<long>(chi, DD);
  if ((size_t)(DD * DD * DD) > c->pipe_elems)
    return fail(c, CTM_EINVAL, "init_mode CTM_INIT_FROM_A needs chi * d >= D (edge buffer)");
  CTM_CUDA_OK(cudaMemsetAsync(c->C, 0, 4 * c->S * elems_C(c) * c->es, c->stream));
  CTM_CUDA_OK(cudaMemsetAsync(c->T, 0, 4 * c->S * elems_T(c) * c->es, c->stream));
  for (int i = 0; i < 4; ++i) {
    for (int site = 0; site < c->S; ++site) {
      void* A = KETp(c, i, site);
      void* B = BRAp(c, i, site);
      Tn cc = tn(c->pipe[0], {Dk, Db, Dk, Db});
      CK(ein(c, "sulde,sulDE->dDeE", tn(A, {d, Dk, Dk, Dk, Dk}), false,
             tn(B, {d, Db, Db, Db, Db}), false, cc));
      CTM_CUDA_OK(cudaMemcpy2DAsync(Cp(c, i, site), chi * c->es, cc.p, DD * c->es, m * c->es, m,
                                    cudaMemcpyDeviceToDevice, c->stream));
      Tn tt = tn(c->pipe[1], {Dk, Db, Dk, Db, Dk, Db});
      CK(ein(c, "sulde,suLDE->lLeEdD", tn(A, {d, Dk, Dk, Dk, Dk}), false,
             tn(B, {d, Db, Db, Db, Db}), false, tt));
      CTM_CUDA_OK(cudaMemcpy2DAsync(Tp(c, i, site), chi * DD * c->es, tt.p, DD * DD * c->es,
                                    m * DD * c->es, m, cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  const size_t mark = c->scratch_off;
  void* w = scratch_alloc(c, (size_t)3 * 152 * 4 * c->S * sizeof(double));
  void* f = scratch_alloc(c, (size_t)4 * c->S * c->es);
  if (!w || !f) return fail(c, CTM_ENOMEM, "scratch arena too small for the norms");
  CTM_CUDA_OK(normalize_phase(c->cx, elems_C(c), c->C, elems_C(c), 4 * c->S, f, w, c->stream,
                              &c->launches));
  CTM_CUDA_OK(normalize_phase(c->cx, elems_T(c), c->T, elems_T(c), 4 * c->S, f, w, c->stream,
                              &c->launches));
  c->scratch_off = mark;
  return CTM_OK;
}

// After a synchronisation: fold the mean sin^2 of the last moves into the
// recycling decisions (a cut recycles without an update round while its
// angle stays below recycle_sin2, once it had min_si_steps updates).
ctm_status update_recycling(ctm_ctx* c) {
  if (!(c->opts.recycle_sin2 > 0.0)) return CTM_OK;
  std::vector<double> h(4 * c->S);
  CTM_CUDA_OK(cudaMemcpyAsync(h.data(), c->dsin2, h.size() * sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
  CTM_CUDA_OK(cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < h.size(); ++i)
    c->si_skip[i] = (h[i] < c->opts.recycle_sin2 && c->si_updates[i] >= c->opts.min_si_steps) ? 1 : 0;
  return CTM_OK;
}

ctm_status create(ctm_ctx** out, int Lx, int Ly, int d, int Dk, int Db, int chi, bool cx,
                  const ctm_opts* opts, const void* const* kets, const void* const* bras,
                  bool classical) {
  if (!out) return fail(nullptr, CTM_EINVAL, "out is NULL");
  *out = nullptr;
  if (Lx < 1 || Ly < 1 || d < 1 || Dk < 1 || Db < 1 || chi < 1)
    return fail(nullptr, CTM_EINVAL, "Lx, Ly, d, D and chi must be >= 1");
  if (!kets) return fail(nullptr, CTM_EINVAL, "tensor pointers are NULL");
  for (int i = 0; i < Lx * Ly; ++i)
    if (!kets[i]) return fail(nullptr, CTM_EINVAL, "a tensor pointer is NULL");
  ctm_ctx* c = new ctm_ctx();
  g_cur = c;
  c->Lx = Lx; c->Ly = Ly; c->S = Lx * Ly;
  c->d = d; c->Dk = Dk; c->Db = Db; c->chi = chi; c->cx = cx;
  c->bra_is_conj = !bras && !classical;
  c->es = cx ? 16 : 8;
  if (opts) c->opts = *opts;
  else ctm_default_opts(&c->opts);
  if (c->opts.p < 0 || c->opts.si_rounds < 0 || c->opts.warmup_iters < 0 ||
      c->opts.warmup_rounds < 0 || c->opts.svd_max_sweeps < 1 || c->opts.min_si_steps < 0 ||
      c->opts.prec < CTM_PREC_FP64 || c->opts.prec > CTM_PREC_SPLIT_TF32 ||
      !(c->opts.recycle_sin2 >= 0.0) ||
      (c->opts.init_mode != CTM_INIT_RANDOM && c->opts.init_mode != CTM_INIT_FROM_A) ||
      (c->opts.svd_presolve != 0 && c->opts.svd_presolve != 1) ||
      (c->opts.fp64_tc != 0 && c->opts.fp64_tc != 1) || !(c->opts.split_refine >= 0.0)) {
    delete c;
    g_cur = nullptr;
    return fail(nullptr, CTM_EINVAL,
                "p, si_rounds, warm-up counts and min_si_steps must be >= 0, svd_max_sweeps >= 1, "
                "recycle_sin2, split_refine >= 0, init_mode, fp64_tc and svd_presolve 0 or 1");
  }
  c->N = chi * Dk * Db;
  c->k = std::min(chi + c->opts.p, c->N);
  if (chi > c->N) {
    delete c;
    g_cur = nullptr;
    return fail(nullptr, CTM_EINVAL, "chi must not exceed chi*Dk*Db");
  }
  auto bail = [&](ctm_status st) {
    std::string m = c->msg;
    ctm_free(c);
    g_cur = nullptr;
    g_create_error = m;
    return st;
  };
  if (c->opts.stream) {
    c->stream = static_cast<cudaStream_t>(c->opts.stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__));
    c->own_stream = true;
  }
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess)
    return bail(fail(c, CTM_ECUDA, "cudaEventCreate failed"));
  {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return bail(fail(c, CTM_ECUDA, "cannot query the SM count"));
  }
  const size_t S = c->S, N = c->N, k = c->k, es = c->es;
  const size_t nk = elems_ket(c), nb = elems_bra(c);
  const size_t NN = N * N;
  const size_t maxT = (size_t)d * d * NN + 64;
  c->pipe_elems = maxT;
  ctm_status st = CTM_OK;
#define AL(ptr, bytes) \
  if ((st = dalloc(c, (void**)&(ptr), (bytes))) != CTM_OK) return bail(st)
  for (int r = 0; r < 4; ++r) {
    AL(c->ket[r], S * nk * es);
    AL(c->bra[r], S * nb * es);
  }
  AL(c->C, 4 * S * elems_C(c) * es);
  AL(c->T, 4 * S * elems_T(c) * es);
  AL(c->X, 4 * S * N * k * es);
  AL(c->W, 4 * S * N * k * es);
  for (int i = 0; i < 4; ++i) AL(c->Q[i], NN * es);
  AL(c->pipe[0], maxT * es);
  AL(c->pipe[1], maxT * es);
  c->scratch_bytes = 3 * maxT * es + ((size_t)64 << 20);
  AL(c->scratch, c->scratch_bytes);
  const int Lmax = std::max(Lx, Ly);
  AL(c->Pl, Lmax * N * chi * es);
  AL(c->PrH, Lmax * N * chi * es);
  AL(c->lastPl, S * N * chi * es);
  AL(c->lastPrH, S * N * chi * es);
  for (int i = 0; i < 4; ++i) AL(c->Z[i], N * k * es);
  AL(c->Xn, N * k * es);
  AL(c->Wn, N * k * es);
  AL(c->G, k * k * es);
  AL(c->Linv, k * k * es);
  AL(c->ZR, Lmax * N * k * es);
  AL(c->ZL, Lmax * N * k * es);
  AL(c->rho, Lmax * k * k * es);
  AL(c->u, Lmax * k * k * es);
  AL(c->v, Lmax * k * k * es);
  {
    const size_t jn = std::max(Lmax * k * k, 4 * S * (size_t)chi * chi) * es;
    AL(c->jv0, jn);
    AL(c->jv1, jn);
    AL(c->jT, jn);
    AL(c->jB, jn);
  }
  AL(c->jw, std::max(jacobi_coop_work_bytes(cx, (int)k, Lmax),
                     jacobi_coop_work_bytes(cx, chi, 4 * (int)S)));
  AL(c->ph, std::max(k, (size_t)chi) * es);
  AL(c->Vs, k * chi * es);
  AL(c->Us, k * chi * es);
  AL(c->sv, std::max(Lmax * k, 4 * S * (size_t)chi) * sizeof(double));
  AL(c->stC1, Lmax * elems_C(c) * es);
  AL(c->stC4, Lmax * elems_C(c) * es);
  AL(c->stT4, Lmax * elems_T(c) * es);
  AL(c->spec_old, 4 * S * chi * sizeof(double));
  AL(c->spec_new, 4 * S * chi * sizeof(double));
  AL(c->dscal, 64 * sizeof(double));
  AL(c->op, (size_t)d * d * d * d * es);
  AL(c->rho2, (size_t)d * d * d * d * es);
  AL(c->imp[0], nk * es);
  AL(c->imp[1], nk * es);
  AL(c->err, sizeof(int));
  AL(c->dead, k * sizeof(int));
  AL(c->chol_work, chol_coop_work_bytes((int)k, 1));
  AL(c->dsc, k * sizeof(double));
  AL(c->fac, Lmax * es);
  AL(c->dsin2, 4 * S * sizeof(double));
  AL(c->sinG, Lmax * k * k * es);
  if (c->opts.warmup_rsvd) {
    AL(c->Xraw, 4 * S * N * k * es);
    AL(c->Wraw, 4 * S * N * k * es);
  }
#undef AL
  c->si_updates.assign(4 * S, 0);
  c->si_skip.assign(4 * S, 0);
  c->si_rounds_used.assign(4 * S, 0);
  // every upload goes through the context's stream: a copy on the legacy
  // default stream is not ordered before kernels on a non-blocking stream
  if (cudaMemsetAsync(c->err, 0, sizeof(int), c->stream) != cudaSuccess)
    return bail(fail(c, CTM_ECUDA, "cudaMemset failed"));
  c->rf_ready.assign(4 * S, 0);
  // tensors: upload rotation 0, derive the other three on the device
  for (int i = 0; i < c->S; ++i) {
    if (cudaMemcpyAsync(at(c->ket[0], i * nk, c), kets[i], nk * es, cudaMemcpyHostToDevice,
                        c->stream) != cudaSuccess)
      return bail(fail(c, CTM_ECUDA, "upload of A failed"));
    if (classical) {
      const double one[2] = {1.0, 0.0};
      if (cudaMemcpyAsync(at(c->bra[0], i * nb, c), one, es, cudaMemcpyHostToDevice,
                          c->stream) != cudaSuccess)
        return bail(fail(c, CTM_ECUDA, "upload of B failed"));
    } else if (bras) {
      if (cudaMemcpyAsync(at(c->bra[0], i * nb, c), bras[i], nb * es, cudaMemcpyHostToDevice,
                          c->stream) != cudaSuccess)
        return bail(fail(c, CTM_ECUDA, "upload of B failed"));
    } else {
      const long dims1[1] = {(long)nk};
      const int perm1[1] = {0};
      cudaError_t e = permute(at(c->ket[0], i * nk, c), at(c->bra[0], i * nb, c), 1, dims1, perm1,
                              cx, true, c->stream, &c->launches);
      if (e != cudaSuccess) return bail(cuda_fail(e, "conj(A)", __FILE__, __LINE__));
    }
  }
  static const int rot[4][5] = {{0, 1, 2, 3, 4}, {0, 4, 1, 2, 3}, {0, 3, 4, 1, 2}, {0, 2, 3, 4, 1}};
  for (int r = 1; r < 4; ++r) {
    for (int i = 0; i < c->S; ++i) {
      const long dk[5] = {d, Dk, Dk, Dk, Dk}, db[5] = {d, Db, Db, Db, Db};
      cudaError_t e = permute(at(c->ket[0], i * nk, c), at(c->ket[r], i * nk, c), 5, dk, rot[r],
                              cx, false, c->stream, &c->launches);
      if (e == cudaSuccess)
        e = permute(at(c->bra[0], i * nb, c), at(c->bra[r], i * nb, c), 5, db, rot[r], cx, false,
                    c->stream, &c->launches);
      if (e != cudaSuccess) return bail(cuda_fail(e, "rotate A", __FILE__, __LINE__));
    }
  }
  if ((st = upload_default_state(c)) != CTM_OK) return bail(st);
  if (c->opts.init_mode == CTM_INIT_FROM_A && (st = init_env_from_tensors(c)) != CTM_OK)
    return bail(st);
  if (c->opts.prec != CTM_PREC_FP64) {
    st = split_create(&c->split, cx, c->opts.prec == CTM_PREC_SPLIT_TF32, (int)N, (int)k, c->err,
                      c->stream);
    if (st != CTM_OK) {
      c->msg = "split-precision setup failed";
      return bail(st);
    }
  }
  {
    // lane 0: the buffers above; lanes 1 .. nl-1 for the other cuts of a
    // column (SI path, cells with more than one cut per column)
    ctm_ctx::Lane L0;
    L0.stream = c->stream;
    for (int q = 0; q < 4; ++q) L0.Q[q] = c->Q[q];
    L0.pipe[0] = c->pipe[0];
    L0.pipe[1] = c->pipe[1];
    L0.scratch = c->scratch;
    L0.scratch_bytes = c->scratch_bytes;
    L0.split = c->split;
    for (int q = 0; q < 4; ++q) L0.Z[q] = c->Z[q];
    L0.G = c->G;
    L0.Linv = c->Linv;
    L0.dsc = c->dsc;
    L0.dead = c->dead;
    L0.chol_work = c->chol_work;
    L0.Xn = c->Xn;
    L0.Wn = c->Wn;
    L0.Vs = c->Vs;
    L0.Us = c->Us;
    L0.ph = c->ph;
    if (cudaEventCreateWithFlags(&L0.ev, cudaEventDisableTiming) != cudaSuccess)
      return bail(fail(c, CTM_ECUDA, "cudaEventCreate failed"));
    c->lanes.push_back(L0);
    const int nl = c->opts.method == CTM_PROJ_SI ? lanes_for(Lx, Ly) : 1;
    for (int l = 1; l < nl; ++l) {
      ctm_ctx::Lane L;
      c->lanes.push_back(L);
      ctm_ctx::Lane& M = c->lanes.back();
      if (cudaStreamCreateWithFlags(&M.stream, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&M.ev, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(c, CTM_ECUDA, "lane stream creation failed"));
      // a lane only builds corners and runs the SI round: its pipelines hold
      // N^2 elements (d N^2 for the unfused absorption, which the refinement
      // uses), not the d^2 N^2 of the two-site observables of lane 0
      const bool fused = !(c->opts.split_refine > 0.0) &&
                         use_fused_absorb(cx, c->opts.prec != CTM_PREC_FP64, c->opts,
                                          (int)Dk, (int)Db, d);
      const size_t laneT = (size_t)(fused ? 1 : d) * NN + 64;
      M.scratch_bytes = 2 * laneT * es + ((size_t)64 << 20);
      for (int q = 0; q < 4; ++q)
        if ((st = dalloc(c, &M.Q[q], NN * es)) != CTM_OK) return bail(st);
      if ((st = dalloc(c, &M.pipe[0], laneT * es)) != CTM_OK ||
          (st = dalloc(c, &M.pipe[1], laneT * es)) != CTM_OK ||
          (st = dalloc(c, (void**)&M.scratch, M.scratch_bytes)) != CTM_OK)
        return bail(st);
      for (int q = 0; q < 4; ++q)
        if ((st = dalloc(c, &M.Z[q], N * k * es)) != CTM_OK) return bail(st);
      if ((st = dalloc(c, &M.G, k * k * es)) != CTM_OK ||
          (st = dalloc(c, &M.Linv, k * k * es)) != CTM_OK ||
          (st = dalloc(c, (void**)&M.dsc, k * sizeof(double))) != CTM_OK ||
          (st = dalloc(c, (void**)&M.dead, k * sizeof(int))) != CTM_OK ||
          (st = dalloc(c, &M.chol_work, chol_coop_work_bytes((int)k, 1))) != CTM_OK ||
          (st = dalloc(c, &M.Xn, N * k * es)) != CTM_OK ||
          (st = dalloc(c, &M.Wn, N * k * es)) != CTM_OK ||
          (st = dalloc(c, &M.Vs, k * chi * es)) != CTM_OK ||
          (st = dalloc(c, &M.Us, k * chi * es)) != CTM_OK ||
          (st = dalloc(c, &M.ph, std::max(k, (size_t)chi) * es)) != CTM_OK)
        return bail(st);
      if (c->opts.prec != CTM_PREC_FP64 &&
          (st = split_create(&M.split, cx, c->opts.prec == CTM_PREC_SPLIT_TF32, (int)N, (int)k,
                             c->err, M.stream)) != CTM_OK) {
        c->msg = "split-precision setup failed";
        return bail(st);
      }
    }
  }
  if (c->opts.method == CTM_PROJ_SVD) {
    st = svd_create(&c->svd, cx, (int)N, chi);
    if (st != CTM_OK) {
      c->msg = std::string("dense SVD setup failed: ") + svd_last_error(c->svd);
      return bail(st);
    }
    if ((st = dalloc(c, &c->svdM, N * N * es)) != CTM_OK) return bail(st);
    if ((st = dalloc(c, &c->svdUs, N * chi * es)) != CTM_OK) return bail(st);
    if ((st = dalloc(c, &c->svdVs, N * chi * es)) != CTM_OK) return bail(st);
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bail(fail(c, CTM_ECUDA, "initialisation failed on the device"));
  *out = c;
  g_cur = nullptr;
  return CTM_OK;
}


// one-site patch with the ket at (x, y) of frame 0 replaced by K (device);
// result: scalar Z at out (open = false) or rho[s][t] (open = true)
ctm_status one_site(ctm_ctx* c, int x, int y, void* K, bool open, void* out) {
  const long chi = c->chi, Dk = c->Dk, Db = c->Db, d = c->d;
  const int r = 0;
  const int site = frame_site(c, r, x, y);
  void* B = BRAp(c, 0, site);
  Tn E1 = tn(c->pipe[0], {chi, chi, Dk, Db});
  CK(ein(c, "ab,bcuU->acuU", tn(fC(c, r, 0, x, y), {chi, chi}), false,
         tn(fT(c, r, 0, x, y), {chi, chi, Dk, Db}), false, E1));
  Tn E2 = tn(c->pipe[1], {chi, Dk, Db, chi, Dk, Db});
  CK(ein(c, "ialL,acuU->ilLcuU", tn(fT(c, r, 3, x, y), {chi, chi, Dk, Db}), false, E1, false, E2));
  Tn E3 = tn(c->pipe[0], {chi, Db, chi, Db, d, Dk, Dk});
  CK(ein(c, "ilLcuU,sulwr->iLcUswr", E2, false, tn(K, {d, Dk, Dk, Dk, Dk}), false, E3));
  Tn Qx;
  if (open) {
    Qx = tn(c->pipe[1], {chi, chi, Dk, Db, Dk, Db, d, d});
    CK(ein(c, "iLcUswr,tULWR->icwWrRst", E3, false, tn(B, {d, Db, Db, Db, Db}), false, Qx));
  } else {
    Qx = tn(c->pipe[1], {chi, chi, Dk, Db, Dk, Db});
    CK(ein(c, "iLcUswr,sULWR->icwWrR", E3, false, tn(B, {d, Db, Db, Db, Db}), false, Qx));
  }
  // rest of the ring: C2 T2 C3 T3 C4 -> F[c, r, R, w, W, i]; keep Qx in pipe[1]
  // and build F in the Q[0]/Q[1] buffers (N^2 elements each)
  Tn F1 = tn(c->Q[0], {chi, chi, Dk, Db});
  CK(ein(c, "ce,efrR->cfrR", tn(fC(c, r, 1, x, y), {chi, chi}), false,
         tn(fT(c, r, 1, x, y), {chi, chi, Dk, Db}), false, F1));
  Tn F2 = tn(c->Q[1], {chi, Dk, Db, chi});
  CK(ein(c, "cfrR,fg->crRg", F1, false, tn(fC(c, r, 2, x, y), {chi, chi}), false, F2));
  Tn F3 = tn(c->Q[0], {chi, Dk, Db, chi, Dk, Db});
  CK(ein(c, "crRg,ghwW->crRhwW", F2, false, tn(fT(c, r, 2, x, y), {chi, chi, Dk, Db}), false, F3));
  Tn F4 = tn(c->Q[1], {chi, Dk, Db, Dk, Db, chi});
  CK(ein(c, "crRhwW,hi->crRwWi", F3, false, tn(fC(c, r, 3, x, y), {chi, chi}), false, F4));
  if (open)
    CK(ein(c, "icwWrRst,crRwWi->st", Qx, false, F4, false, tn(out, {d, d})));
  else
    CK(ein(c, "icwWrR,crRwWi->", Qx, false, F4, false, tn(out, {})));
  return CTM_OK;
}

// two-site patch of frame r at (x, y), (x+1, y); kets K1, K2 are frame
// rotated; result rho[s1][s2][t1][t2] at out (unnormalised)
ctm_status two_site(ctm_ctx* c, int r, int x, int y, void* K1, void* K2, void* out) {
  const long chi = c->chi, Dk = c->Dk, Db = c->Db, d = c->d;
  void* B1 = BRAp(c, r, frame_site(c, r, x, y));
  void* B2 = BRAp(c, r, frame_site(c, r, x + 1, y));
  const Tn tC = tn(nullptr, {chi, chi}), tT = tn(nullptr, {chi, chi, Dk, Db});
  auto C_ = [&](int i, int xx) { Tn t = tC; t.p = fC(c, r, i, xx, y); return t; };
  auto T_ = [&](int i, int xx) { Tn t = tT; t.p = fT(c, r, i, xx, y); return t; };
  // the two halves live in the scratch arena (chi^2 d^2 Dk Db elements each)
  const size_t mark = c->scratch_off;
  const size_t half = (size_t)chi * chi * d * d * Dk * Db * c->es;
  void* Lbuf = scratch_alloc(c, half);
  void* Rbuf = scratch_alloc(c, half);
  if (!Lbuf || !Rbuf) return fail(c, CTM_ENOMEM, "scratch arena too small for the two-site patch");
  // left half L[i, c, s, m, t, M]
  CK(ein(c, "ab,bcuU->acuU", C_(0, x), false, T_(0, x), false, tn(c->pipe[0], {chi, chi, Dk, Db})));
  CK(ein(c, "kalL,acuU->klLcuU", T_(3, x), false, tn(c->pipe[0], {chi, chi, Dk, Db}), false,
         tn(c->pipe[1], {chi, Dk, Db, chi, Dk, Db})));
  CK(ein(c, "klLcuU,sulxm->kLcUsxm", tn(c->pipe[1], {chi, Dk, Db, chi, Dk, Db}), false,
         tn(K1, {d, Dk, Dk, Dk, Dk}), false, tn(c->pipe[0], {chi, Db, chi, Db, d, Dk, Dk})));
  CK(ein(c, "kLcUsxm,tULXM->kcsxmtXM", tn(c->pipe[0], {chi, Db, chi, Db, d, Dk, Dk}), false,
         tn(B1, {d, Db, Db, Db, Db}), false, tn(c->pipe[1], {chi, chi, d, Dk, Dk, d, Db, Db})));
  CK(ein(c, "kcsxmtXM,jk->jcsxmtXM", tn(c->pipe[1], {chi, chi, d, Dk, Dk, d, Db, Db}), false,
         C_(3, x), false, tn(c->pipe[0], {chi, chi, d, Dk, Dk, d, Db, Db})));
  Tn L = tn(Lbuf, {chi, chi, d, Dk, d, Db});
  CK(ein(c, "jcsxmtXM,ijxX->icsmtM", tn(c->pipe[0], {chi, chi, d, Dk, Dk, d, Db, Db}), false,
         T_(2, x), false, L));
  // right half R[c, i, q, m, v, M]
  CK(ein(c, "ceoO,ef->cfoO", T_(0, x + 1), false, C_(1, x + 1), false,
         tn(c->pipe[0], {chi, chi, Dk, Db})));
  CK(ein(c, "cfoO,fgrR->cgoOrR", tn(c->pipe[0], {chi, chi, Dk, Db}), false, T_(1, x + 1), false,
         tn(c->pipe[1], {chi, chi, Dk, Db, Dk, Db})));
  CK(ein(c, "cgoOrR,qomwr->cgORqmw", tn(c->pipe[1], {chi, chi, Dk, Db, Dk, Db}), false,
         tn(K2, {d, Dk, Dk, Dk, Dk}), false, tn(c->pipe[0], {chi, chi, Db, Db, d, Dk, Dk})));
  CK(ein(c, "cgORqmw,vOMWR->cgqmwvMW", tn(c->pipe[0], {chi, chi, Db, Db, d, Dk, Dk}), false,
         tn(B2, {d, Db, Db, Db, Db}), false, tn(c->pipe[1], {chi, chi, d, Dk, Dk, d, Db, Db})));
  CK(ein(c, "cgqmwvMW,gh->chqmwvMW", tn(c->pipe[1], {chi, chi, d, Dk, Dk, d, Db, Db}), false,
         C_(2, x + 1), false, tn(c->pipe[0], {chi, chi, d, Dk, Dk, d, Db, Db})));
  Tn R = tn(Rbuf, {chi, chi, d, Dk, d, Db});
  CK(ein(c, "chqmwvMW,hiwW->ciqmvM", tn(c->pipe[0], {chi, chi, d, Dk, Dk, d, Db, Db}), false,
         T_(2, x + 1), false, R));
  CK(ein(c, "icsmtM,ciqmvM->sqtv", L, false, R, false, tn(out, {d, d, d, d})));
  c->scratch_off = mark;
  return CTM_OK;
}

// frame and frame positions of the bond (x, y) -> right (dir 0) / down (dir 1)
void bond_frame(const ctm_ctx* c, int x, int y, int dir, int* r, int* fx, int* fy) {
  if (dir == 0) { *r = 0; *fx = x; *fy = y; }
  else { *r = 1; *fx = y; *fy = ((-x) % c->Lx + c->Lx) % c->Lx; }
}

ctm_status rho2_device(ctm_ctx* c, int x, int y, int dir, const void* h1, const void* h2,
                       void* out) {
  int r, fx, fy;
  bond_frame(c, x, y, dir, &r, &fx, &fy);
  void* K1 = KETp(c, r, frame_site(c, r, fx, fy));
  void* K2 = KETp(c, r, frame_site(c, r, fx + 1, fy));
  static const int rot[4][5] = {{0, 1, 2, 3, 4}, {0, 4, 1, 2, 3}, {0, 3, 4, 1, 2}, {0, 2, 3, 4, 1}};
  const long dk[5] = {c->d, c->Dk, c->Dk, c->Dk, c->Dk};
  const size_t nk = elems_ket(c);
  if (h1) {
    CTM_CUDA_OK(cudaMemcpyAsync(c->pipe[1], h1, nk * c->es, cudaMemcpyHostToDevice, c->stream));
    CTM_CUDA_OK(permute(c->pipe[1], c->imp[0], 5, dk, rot[r], c->cx, false, c->stream, &c->launches));
    K1 = c->imp[0];
  }
  if (h2) {
    CTM_CUDA_OK(cudaMemcpyAsync(c->pipe[1], h2, nk * c->es, cudaMemcpyHostToDevice, c->stream));
    CTM_CUDA_OK(permute(c->pipe[1], c->imp[1], 5, dk, rot[r], c->cx, false, c->stream, &c->launches));
    K2 = c->imp[1];
  }
  return two_site(c, r, fx, fy, K1, K2, out);
}

bool valid_site(const ctm_ctx* c, int x, int y) {
  return x >= 0 && y >= 0 && x < c->Lx && y < c->Ly;
}

}  // namespace ctmi

// =============================================================== C ABI
extern "C" {

void ctm_default_opts(ctm_opts* o) {
  if (!o) return;
  o->p = 5;
  o->si_rounds = 1;
  o->warmup_iters = 5;
  o->warmup_rounds = 8;
  o->method = CTM_PROJ_SI;
  o->prec = CTM_PREC_FP64;
  o->svd_rel_cutoff = 1e-12;
  o->normalize = 1;
  o->sign_fix = 1;
  o->seed = 0;
  o->svd_max_sweeps = 80;
  o->init_mode = CTM_INIT_RANDOM;
  o->recycle_sin2 = 0.0;
  o->min_si_steps = 3;
  o->absorb_tc = 0;
  o->si_coupled = 0;
  o->warmup_rsvd = 0;
  o->fp64_tc = 1;
  o->svd_presolve = 1;
  o->split_refine = 0.0;
  o->stream = nullptr;
}

ctm_status ctm_init(ctm_ctx** out, int Lx, int Ly, const void* const* A, const void* const* bra,
                    ctm_dtype dtype, int d, int D, int chi, const ctm_opts* opts) {
  if (dtype != CTM_F64 && dtype != CTM_C128) return fail(nullptr, CTM_EINVAL, "bad dtype");
  return create(out, Lx, Ly, d, D, D, chi, dtype == CTM_C128, opts, A, bra, false);
}

ctm_status ctm_init_network(ctm_ctx** out, int Lx, int Ly, const double* const* a, int k, int chi,
                            const ctm_opts* opts) {
  return create(out, Lx, Ly, 1, k, 1, chi, false, opts, reinterpret_cast<const void* const*>(a),
                nullptr, true);
}

ctm_status ctm_set_env(ctm_ctx* c, const void* C, const void* T) {
  if (!c || !C || !T) return fail(c, CTM_EINVAL, "NULL argument");
  Guard gd(c);
  CTM_CUDA_OK(cudaMemcpyAsync(c->C, C, 4 * c->S * elems_C(c) * c->es, cudaMemcpyHostToDevice, c->stream));
  CTM_CUDA_OK(cudaMemcpyAsync(c->T, T, 4 * c->S * elems_T(c) * c->es, cudaMemcpyHostToDevice, c->stream));
  CTM_CUDA_OK(cudaStreamSynchronize(c->stream));
  c->spectra_init = false;
  c->spectra_fresh = false;
  return CTM_OK;
}

ctm_status ctm_get_env(ctm_ctx* c, void* C, void* T) {
  if (!c || !C || !T) return fail(c, CTM_EINVAL, "NULL argument");
  Guard gd(c);
  CTM_CUDA_OK(cudaMemcpyAsync(C, c->C, 4 * c->S * elems_C(c) * c->es, cudaMemcpyDeviceToHost, c->stream));
  CTM_CUDA_OK(cudaMemcpyAsync(T, c->T, 4 * c->S * elems_T(c) * c->es, cudaMemcpyDeviceToHost, c->stream));
  CTM_CUDA_OK(cudaStreamSynchronize(c->stream));
  return CTM_OK;
}

ctm_status ctm_set_rangefinders(ctm_ctx* c, const void* X, const void* W) {
  if (!c || !X || !W) return fail(c, CTM_EINVAL, "NULL argument");
  Guard gd(c);
  const size_t n = (size_t)4 * c->S * c->N * c->k * c->es;
  CTM_CUDA_OK(cudaMemcpyAsync(c->X, X, n, cudaMemcpyHostToDevice, c->stream));
  CTM_CUDA_OK(cudaMemcpyAsync(c->W, W, n, cudaMemcpyHostToDevice, c->stream));
  CK(keep_raw_rangefinders(c));
  CTM_CUDA_OK(cudaStreamSynchronize(c->stream));
  std::fill(c->rf_ready.begin(), c->rf_ready.end(), 0);
  for (int r = 0; r < 4; ++r) c->moves_done[r] = 0;
  return reset_recycling(c);
}

// ------------------------------------------------------------ footprint
// Device bytes a context of these dimensions allocates (the list of create(),
// plus the split-precision slice caches and partial sums and the dense-SVD
// buffers), rounded up by 5 % + 64 MB for allocator granularity.
static size_t footprint_bytes(int Lx, int Ly, int d, int Dk, int Db, int chi, bool cx,
                       const ctm_opts* o) {
  const size_t S = (size_t)Lx * Ly, es = cx ? 16 : 8;
  const size_t N = (size_t)chi * Dk * Db;
  const size_t k = std::min<size_t>((size_t)chi + o->p, N);
  const size_t NN = N * N, maxT = (size_t)d * d * NN + 64;
  const size_t Lmax = std::max(Lx, Ly);
  const size_t eC = (size_t)chi * chi, eT = eC * Dk * Db;
  const size_t nk = (size_t)d * Dk * Dk * Dk * Dk, nb = (size_t)d * Db * Db * Db * Db;
  size_t b = 0;
  b += 4 * S * (nk + nb) * es;                     // kets, bras
  b += 4 * S * (eC + eT) * es;                     // C, T
  b += 2 * 4 * S * N * k * es;                     // X, W
  b += 4 * NN * es + 2 * maxT * es;                // Q, pipes
  b += 3 * maxT * es + ((size_t)64 << 20);         // scratch
  b += 2 * Lmax * N * chi * es + 2 * S * N * chi * es;   // Pl, PrH, last*
  b += 6 * N * k * es + 2 * k * k * es;            // Z, Xn, Wn, G, Linv
  b += 2 * Lmax * N * k * es + 3 * Lmax * k * k * es;    // ZR, ZL, rho, u, v
  b += 4 * std::max(Lmax * k * k, 4 * S * (size_t)chi * chi) * es;   // pre-solve
  b += std::max(jacobi_coop_work_bytes(cx, (int)k, (int)Lmax),
                jacobi_coop_work_bytes(cx, chi, 4 * (int)S));
  b += (std::max(k, (size_t)chi) + 2 * k * chi) * es;
  b += std::max(Lmax * k, 4 * S * (size_t)chi) * sizeof(double);
  b += Lmax * (2 * eC + eT) * es + 8 * S * chi * sizeof(double);
  b += 2 * (size_t)d * d * d * d * es + 2 * nk * es + ((size_t)1 << 20);
  b += Lmax * k * k * es + 4 * S * sizeof(double);   // recycling policy
  if (o->warmup_rsvd) b += 2 * 4 * S * N * k * es;    // raw blocks
  if (o->prec != CTM_PREC_FP64) {
    // slices: 3 bf16 (6 bytes) or 2 tf32 (8 bytes) per element
    const size_t Kp = ((cx ? 2 : 1) * N + 63) / 64 * 64;
    const size_t sb = o->prec == CTM_PREC_SPLIT_TF32 ? 8 : 6;
    b += 8 * N * Kp * sb;                          // corner slices, both orientations
    b += 2 * N * Kp * sb;                          // operand slices of general products
    b += split_partial_splits(N, cx) * N * ((cx ? 2 : 1) * k + 160) * 4;   // split-K partials
  }
  // refinement: eight 2-byte digits per real component of the operands
  // (complex B operands as 2 x 2 real blocks, K padded to at most twice) and
  // fp32-pair partials, for operands of up to d N^2 elements on the lanes and
  // d^2 N^2 for the two-site observables of lane 0
  const bool refine = o->prec != CTM_PREC_FP64 && o->split_refine > 0.0;
  const size_t oz_refine = refine ? 12 * (size_t)d * NN * es : 0;
  b += (size_t)d * oz_refine;
  if (o->method == CTM_PROJ_SVD) b += 3 * NN * es + 2 * N * chi * es + (size_t)64 * N * es;
  if (o->method == CTM_PROJ_SI) {
    // lanes 1 .. nl-1: corners, pipes, scratch, N x k blocks, QR work, split state
    const bool fused =
        !(o->split_refine > 0.0) && use_fused_absorb(cx, o->prec != CTM_PREC_FP64, *o, Dk, Db, d);
    const size_t laneT = (size_t)(fused ? 1 : d) * NN + 64;
    size_t lane = 4 * NN * es + 4 * laneT * es + ((size_t)64 << 20) + 4 * N * k * es +
                  2 * k * k * es + 12 * k + chol_coop_work_bytes((int)k, 1) +
                  (2 * N * k + 2 * k * chi + std::max(k, (size_t)chi)) * es;   // si_finish
    if (o->prec != CTM_PREC_FP64) {
      const size_t Kp = ((cx ? 2 : 1) * N + 63) / 64 * 64;
      const size_t sb = o->prec == CTM_PREC_SPLIT_TF32 ? 8 : 6;
      lane += 10 * N * Kp * sb + split_partial_splits(N, cx) * N * ((cx ? 2 : 1) * k + 160) * 4;
    }
    lane += oz_refine;
    b += (size_t)(lanes_for(Lx, Ly) - 1) * lane;
  }
  return b + b / 20 + ((size_t)64 << 20);
}

// ---------------------------------------------------- checkpoint / resume
namespace {

struct SaveHeader {
  char magic[8];             // "CTMSAVE1"
  int32_t Lx, Ly, d, Dk, Db, chi, N, k, cx, last_dir;
  int32_t moves_done[4];
  int32_t spectra_init;
  uint64_t qr_calls;
};

size_t save_bytes(const ctm_ctx* c) {
  const size_t env = (size_t)4 * c->S * (elems_C(c) + elems_T(c)) * c->es;
  const size_t rf = (size_t)2 * 4 * c->S * c->N * c->k * c->es;
  return sizeof(SaveHeader) + env + rf + (size_t)4 * c->S + (size_t)4 * c->S * c->chi * sizeof(double);
}

}  // namespace

ctm_status ctm_save(const ctm_ctx* cc, void* buf, size_t* nbytes) {
  ctm_ctx* c = const_cast<ctm_ctx*>(cc);
  if (!c || !nbytes) return fail(c, CTM_EINVAL, "NULL argument");
  const size_t need = save_bytes(c);
  if (!buf) {
    *nbytes = need;
    return CTM_OK;
  }
  if (*nbytes < need) return fail(c, CTM_EINVAL, "checkpoint buffer too small");
  Guard gd(c);
  SaveHeader h{};
  memcpy(h.magic, "CTMSAVE1", 8);
  h.Lx = c->Lx; h.Ly = c->Ly; h.d = c->d; h.Dk = c->Dk; h.Db = c->Db; h.chi = c->chi;
  h.N = c->N; h.k = c->k; h.cx = c->cx ? 1 : 0; h.last_dir = c->last_dir;
  for (int r = 0; r < 4; ++r) h.moves_done[r] = c->moves_done[r];
  h.spectra_init = c->spectra_init ? 1 : 0;
  h.qr_calls = c->qr_calls;
  char* p = static_cast<char*>(buf);
  memcpy(p, &h, sizeof h);
  p += sizeof h;
  const size_t nC = (size_t)4 * c->S * elems_C(c) * c->es, nT = (size_t)4 * c->S * elems_T(c) * c->es;
  const size_t nX = (size_t)4 * c->S * c->N * c->k * c->es;
  const size_t nS = (size_t)4 * c->S * c->chi * sizeof(double);
  CTM_CUDA_OK(cudaMemcpyAsync(p, c->C, nC, cudaMemcpyDeviceToHost, c->stream));
  p += nC;
  CTM_CUDA_OK(cudaMemcpyAsync(p, c->T, nT, cudaMemcpyDeviceToHost, c->stream));
  p += nT;
  CTM_CUDA_OK(cudaMemcpyAsync(p, c->X, nX, cudaMemcpyDeviceToHost, c->stream));
  p += nX;
  CTM_CUDA_OK(cudaMemcpyAsync(p, c->W, nX, cudaMemcpyDeviceToHost, c->stream));
  p += nX;
  CTM_CUDA_OK(cudaMemcpyAsync(p, c->spec_old, nS, cudaMemcpyDeviceToHost, c->stream));
  p += nS;
  memcpy(p, c->rf_ready.data(), (size_t)4 * c->S);
  CTM_CUDA_OK(cudaStreamSynchronize(c->stream));
  *nbytes = need;
  return CTM_OK;
}

ctm_status ctm_load(ctm_ctx* c, const void* buf, size_t nbytes) {
  if (!c || !buf) return fail(c, CTM_EINVAL, "NULL argument");
  if (nbytes < sizeof(SaveHeader) || nbytes < save_bytes(c))
    return fail(c, CTM_EINVAL, "checkpoint too short for this context");
  SaveHeader h;
  memcpy(&h, buf, sizeof h);
  if (memcmp(h.magic, "CTMSAVE1", 8) != 0) return fail(c, CTM_EINVAL, "not a checkpoint");
  if (h.Lx != c->Lx || h.Ly != c->Ly || h.d != c->d || h.Dk != c->Dk || h.Db != c->Db ||
      h.chi != c->chi || h.N != c->N || h.k != c->k || h.cx != (c->cx ? 1 : 0))
    return fail(c, CTM_EINVAL, "checkpoint dimensions differ from the context");
  Guard gd(c);
  const char* p = static_cast<const char*>(buf) + sizeof h;
  const size_t nC = (size_t)4 * c->S * elems_C(c) * c->es, nT = (size_t)4 * c->S * elems_T(c) * c->es;
  const size_t nX = (size_t)4 * c->S * c->N * c->k * c->es;
  const size_t nS = (size_t)4 * c->S * c->chi * sizeof(double);
  CTM_CUDA_OK(cudaMemcpyAsync(c->C, p, nC, cudaMemcpyHostToDevice, c->stream));
  p += nC;
  CTM_CUDA_OK(cudaMemcpyAsync(c->T, p, nT, cudaMemcpyHostToDevice, c->stream));
  p += nT;
  CTM_CUDA_OK(cudaMemcpyAsync(c->X, p, nX, cudaMemcpyHostToDevice, c->stream));
  p += nX;
  CTM_CUDA_OK(cudaMemcpyAsync(c->W, p, nX, cudaMemcpyHostToDevice, c->stream));
  p += nX;
  CTM_CUDA_OK(cudaMemcpyAsync(c->spec_old, p, nS, cudaMemcpyHostToDevice, c->stream));
  p += nS;
  memcpy(c->rf_ready.data(), p, (size_t)4 * c->S);
  CTM_CUDA_OK(cudaStreamSynchronize(c->stream));
  for (int r = 0; r < 4; ++r) c->moves_done[r] = h.moves_done[r];
  c->last_dir = h.last_dir;
  c->spectra_init = h.spectra_init != 0;
  c->spectra_fresh = false;
  c->qr_calls = h.qr_calls;
  return CTM_OK;
}

ctm_status ctm_footprint(int Lx, int Ly, int d, int D, int chi, ctm_dtype dtype,
                         const ctm_opts* opts, size_t* bytes) {
  if (!bytes || Lx < 1 || Ly < 1 || d < 1 || D < 1 || chi < 1 ||
      (dtype != CTM_F64 && dtype != CTM_C128))
    return CTM_EINVAL;
  ctm_opts o;
  if (opts) o = *opts;
  else ctm_default_opts(&o);
  *bytes = footprint_bytes(Lx, Ly, d, D, D, chi, dtype == CTM_C128, &o);
  return CTM_OK;
}

ctm_status ctm_dims(const ctm_ctx* c, int* N, int* k) {
  if (!c || !N || !k) return CTM_EINVAL;
  *N = c->N;
  *k = c->k;
  return CTM_OK;
}

// Exact-digit products (c->exact) for the lifetime of the scope. Observables
// of a context with the refinement (split_refine > 0) use them too: the
// environment they contract is fp64-accurate, and split products would add
// their ~1e-7 again. split_refine = +inf makes every move exact from the
// start.
struct ExactScope {
  ctm_ctx* c;
  ExactScope(ctm_ctx* cc, bool on) : c(cc) { c->exact = on; }
  ~ExactScope() { c->exact = false; }
};
bool refine_on(const ctm_ctx* c) { return c->split != nullptr && c->opts.split_refine > 0.0; }
bool exact_always(const ctm_ctx* c) { return refine_on(c) && std::isinf(c->opts.split_refine); }

ctm_status ctm_move(ctm_ctx* c, ctm_dir dir) {
  if (!c) return fail(c, CTM_EINVAL, "ctx is NULL");
  if (dir < 0 || dir > 3) return fail(c, CTM_EINVAL, "direction must be 0..3");
  Guard gd(c);
  ExactScope xs(c, exact_always(c));
  const long l0 = c->launches;
  CTM_CUDA_OK(cudaEventRecord(c->ev0, c->stream));
  CK(move_impl(c, (int)dir));
  CTM_CUDA_OK(cudaEventRecord(c->ev1, c->stream));
  CK(check_err(c));
  CK(update_recycling(c));
  float ms = 0.f;
  CTM_CUDA_OK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  c->last_ms = ms;
  c->last_launches = c->launches - l0;
  return CTM_OK;
}

ctm_status ctm_converge(ctm_ctx* c, double tol, int max_iter, int* iters_out, double* delta_out) {
  if (!c) return fail(c, CTM_EINVAL, "ctx is NULL");
  if (max_iter < 0) return fail(c, CTM_EINVAL, "max_iter must be >= 0");
  Guard gd(c);
  const long l0 = c->launches;
  CTM_CUDA_OK(cudaEventRecord(c->ev0, c->stream));
  const int nspec = 4 * c->S * c->chi;
  if (!c->spectra_init) {
    CK(corner_spectra(c, c->spec_new));
    CTM_CUDA_OK(cudaMemsetAsync(c->spec_old, 0, nspec * sizeof(double), c->stream));
    CTM_CUDA_OK(spectra_delta(c->chi, 4 * c->S, c->spec_new, c->spec_old, c->dscal, c->stream, &c->launches));
    c->spectra_init = true;
    c->spectra_fresh = true;
  }
  // refinement (split_refine): exact-digit products once the spectra have
  // settled to that level, for the rest of this call only
  ExactScope xs(c, exact_always(c));
  double delta = INFINITY;
  int it = 0;
  while (it < max_iter) {
    if (c->split && c->opts.split_refine > 0.0 && delta < c->opts.split_refine) c->exact = true;
    for (int r = 0; r < 4; ++r) CK(move_impl(c, r));
    ++it;
    CK(corner_spectra(c, c->spec_new));
    CTM_CUDA_OK(spectra_delta(c->chi, 4 * c->S, c->spec_new, c->spec_old, c->dscal + 1, c->stream, &c->launches));
    c->spectra_fresh = true;
    CTM_CUDA_OK(cudaMemcpyAsync(&delta, c->dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(check_err(c));
    CK(update_recycling(c));
    if (delta < tol) break;
  }
  CTM_CUDA_OK(cudaEventRecord(c->ev1, c->stream));
  CTM_CUDA_OK(cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  CTM_CUDA_OK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  c->last_ms = ms;
  c->last_launches = c->launches - l0;
  if (iters_out) *iters_out = it;
  if (delta_out) *delta_out = delta;
  if (!(delta < tol)) {
    c->msg = "max_iter reached before the corner spectra converged";
    return CTM_ENOCONV;
  }
  return CTM_OK;
}

ctm_status ctm_spectrum(ctm_ctx* c, int x, int y, int label, double* s_out) {
  if (!c || !s_out) return fail(c, CTM_EINVAL, "NULL argument");
  if (!valid_site(c, x, y) || label < 1 || label > 4) return fail(c, CTM_EINVAL, "bad site or label");
  Guard gd(c);
  const int site = y * c->Lx + x;
  CTM_CUDA_OK(jacobi_svd_coop(c->cx, c->chi, Cp(c, label - 1, site), 0, c->sv, nullptr,
                              nullptr, false, c->jw, 1, c->opts.svd_max_sweeps, c->err, c->num_sms, c->stream,
                              &c->launches));
  CTM_CUDA_OK(normalize(false, c->chi, c->sv, 0, 1, c->dscal, true, c->scratch, c->stream, &c->launches));
  CTM_CUDA_OK(cudaMemcpyAsync(s_out, c->sv, c->chi * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(check_err(c));
  return CTM_OK;
}

ctm_status ctm_spectra(ctm_ctx* c, double* s_out) {
  if (!c || !s_out) return fail(c, CTM_EINVAL, "NULL argument");
  Guard gd(c);
  const int nb = 4 * c->S;
  if (c->spectra_fresh) {
    // the convergence measure of the last iteration already holds them
    CTM_CUDA_OK(cudaMemcpyAsync(s_out, c->spec_old, (size_t)nb * c->chi * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
    CK(check_err(c));
    return CTM_OK;
  }
  CK(corner_spectra(c, c->sv));
  const size_t mark = c->scratch_off;
  double* nrm = static_cast<double*>(scratch_alloc(c, (size_t)nb * sizeof(double)));
  void* w = scratch_alloc(c, (size_t)nb * 152 * sizeof(double));
  if (!nrm || !w) return fail(c, CTM_ENOMEM, "scratch arena too small for the spectra");
  CTM_CUDA_OK(normalize(false, c->chi, c->sv, c->chi, nb, nrm, true, w, c->stream, &c->launches));
  c->scratch_off = mark;
  CTM_CUDA_OK(cudaMemcpyAsync(s_out, c->sv, (size_t)nb * c->chi * sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
  CK(check_err(c));
  return CTM_OK;
}

ctm_status ctm_rdm2(ctm_ctx* c, int x, int y, int dir, double* rho_out) {
  if (!c || !rho_out) return fail(c, CTM_EINVAL, "NULL argument");
  if (!valid_site(c, x, y) || (dir != 0 && dir != 1)) return fail(c, CTM_EINVAL, "bad site or dir");
  Guard gd(c);
  ExactScope xs(c, refine_on(c));
  const int d2 = c->d * c->d;
  CK(rho2_device(c, x, y, dir, nullptr, nullptr, c->rho2));
  std::vector<double> h((size_t)d2 * d2 * (c->cx ? 2 : 1));
  CTM_CUDA_OK(cudaMemcpyAsync(h.data(), c->rho2, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(check_err(c));
  double tr_re = 0.0, tr_im = 0.0;
  for (int i = 0; i < d2; ++i) {
    if (c->cx) { tr_re += h[2 * (i * d2 + i)]; tr_im += h[2 * (i * d2 + i) + 1]; }
    else tr_re += h[i * d2 + i];
  }
  const double den = tr_re * tr_re + tr_im * tr_im;
  for (int i = 0; i < d2 * d2; ++i) {
    double re = c->cx ? h[2 * i] : h[i], im = c->cx ? h[2 * i + 1] : 0.0;
    rho_out[2 * i] = (re * tr_re + im * tr_im) / den;
    rho_out[2 * i + 1] = (im * tr_re - re * tr_im) / den;
  }
  return CTM_OK;
}

ctm_status ctm_expect(ctm_ctx* c, const void* op, int x, int y, int dir, double out[2]) {
  if (!c || !op || !out) return fail(c, CTM_EINVAL, "NULL argument");
  if (!valid_site(c, x, y) || (dir != 0 && dir != 1)) return fail(c, CTM_EINVAL, "bad site or dir");
  Guard gd(c);
  ExactScope xs(c, refine_on(c));
  const int d2 = c->d * c->d;
  CTM_CUDA_OK(cudaMemcpyAsync(c->op, op, (size_t)d2 * d2 * c->es, cudaMemcpyHostToDevice, c->stream));
  CK(rho2_device(c, x, y, dir, nullptr, nullptr, c->rho2));
  CTM_CUDA_OK(trace_products(c->cx, d2, c->op, c->rho2, c->dscal + 8, c->stream, &c->launches));
  double h[4];
  CTM_CUDA_OK(cudaMemcpyAsync(h, c->dscal + 8, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(check_err(c));
  const double den = h[2] * h[2] + h[3] * h[3];
  out[0] = (h[0] * h[2] + h[1] * h[3]) / den;
  out[1] = (h[1] * h[2] - h[0] * h[3]) / den;
  return CTM_OK;
}

ctm_status ctm_expect_bond(ctm_ctx* c, const void* imp1, const void* imp2, int x, int y, int dir,
                           double out[2]) {
  if (!c || !imp1 || !imp2 || !out) return fail(c, CTM_EINVAL, "NULL argument");
  if (!valid_site(c, x, y) || (dir != 0 && dir != 1)) return fail(c, CTM_EINVAL, "bad site or dir");
  Guard gd(c);
  ExactScope xs(c, refine_on(c));
  const int d2 = c->d * c->d;
  // identity operator: the traces of the two density matrices
  std::vector<double> eye((size_t)d2 * d2 * (c->cx ? 2 : 1), 0.0);
  for (int i = 0; i < d2; ++i) eye[(size_t)(i * d2 + i) * (c->cx ? 2 : 1)] = 1.0;
  CTM_CUDA_OK(cudaMemcpyAsync(c->op, eye.data(), eye.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(rho2_device(c, x, y, dir, nullptr, nullptr, c->rho2));
  CTM_CUDA_OK(trace_products(c->cx, d2, c->op, c->rho2, c->dscal + 8, c->stream, &c->launches));
  CK(rho2_device(c, x, y, dir, imp1, imp2, c->rho2));
  CTM_CUDA_OK(trace_products(c->cx, d2, c->op, c->rho2, c->dscal + 12, c->stream, &c->launches));
  double h[8];
  CTM_CUDA_OK(cudaMemcpyAsync(h, c->dscal + 8, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(check_err(c));
  const double den = h[2] * h[2] + h[3] * h[3];
  out[0] = (h[6] * h[2] + h[7] * h[3]) / den;
  out[1] = (h[7] * h[2] - h[6] * h[3]) / den;
  return CTM_OK;
}

ctm_status ctm_expect_site(ctm_ctx* c, const void* imp, int x, int y, double out[2]) {
  if (!c || !imp || !out) return fail(c, CTM_EINVAL, "NULL argument");
  if (!valid_site(c, x, y)) return fail(c, CTM_EINVAL, "bad site");
  Guard gd(c);
  ExactScope xs(c, refine_on(c));
  const size_t nk = elems_ket(c);
  CTM_CUDA_OK(cudaMemcpyAsync(c->imp[0], imp, nk * c->es, cudaMemcpyHostToDevice, c->stream));
  const int site = y * c->Lx + x;
  CK(one_site(c, x, y, KETp(c, 0, site), false, c->dscal + 16));
  CK(one_site(c, x, y, c->imp[0], false, c->dscal + 20));
  double h[8];
  CTM_CUDA_OK(cudaMemcpyAsync(h, c->dscal + 16, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(check_err(c));
  double z0r = h[0], z0i = c->cx ? h[1] : 0.0, z1r = h[4], z1i = c->cx ? h[5] : 0.0;
  const double den = z0r * z0r + z0i * z0i;
  out[0] = (z1r * z0r + z1i * z0i) / den;
  out[1] = (z1i * z0r - z1r * z0i) / den;
  return CTM_OK;
}

ctm_status ctm_free_energy(ctm_ctx* c, double* ln_kappa) {
  if (!c || !ln_kappa) return fail(c, CTM_EINVAL, "NULL argument");
  if (c->S != 1) return fail(c, CTM_EINVAL, "free energy per site needs a 1x1 cell");
  Guard gd(c);
  ExactScope xs(c, refine_on(c));
  const long chi = c->chi, Dk = c->Dk, Db = c->Db;
  CK(one_site(c, 0, 0, KETp(c, 0, 0), false, c->dscal + 24));
  auto Ct = [&](int i) { return tn(Cp(c, i, 0), {chi, chi}); };
  auto Tt = [&](int i) { return tn(Tp(c, i, 0), {chi, chi, Dk, Db}); };
  void* p0 = c->pipe[0];
  void* p1 = c->pipe[1];
  // Z0 = tr(C1 C2 C3 C4)
  CK(ein(c, "ab,bc->ac", Ct(0), false, Ct(1), false, tn(p0, {chi, chi})));
  CK(ein(c, "ac,ce->ae", tn(p0, {chi, chi}), false, Ct(2), false, tn(p1, {chi, chi})));
  CK(ein(c, "ae,ea->", tn(p1, {chi, chi}), false, Ct(3), false, tn(c->dscal + 28, {})));
  // Z13: T1 and T3 joined
  CK(ein(c, "ab,bcuU->acuU", Ct(0), false, Tt(0), false, tn(p0, {chi, chi, Dk, Db})));
  CK(ein(c, "acuU,ce->aeuU", tn(p0, {chi, chi, Dk, Db}), false, Ct(1), false, tn(p1, {chi, chi, Dk, Db})));
  CK(ein(c, "aeuU,ef->afuU", tn(p1, {chi, chi, Dk, Db}), false, Ct(2), false, tn(p0, {chi, chi, Dk, Db})));
  CK(ein(c, "afuU,fguU->ag", tn(p0, {chi, chi, Dk, Db}), false, Tt(2), false, tn(p1, {chi, chi})));
  CK(ein(c, "ag,ga->", tn(p1, {chi, chi}), false, Ct(3), false, tn(c->dscal + 32, {})));
  // Z24: T2 and T4 joined
  CK(ein(c, "ab,bc->ac", Ct(0), false, Ct(1), false, tn(p0, {chi, chi})));
  CK(ein(c, "ac,ceuU->aeuU", tn(p0, {chi, chi}), false, Tt(1), false, tn(p1, {chi, chi, Dk, Db})));
  CK(ein(c, "aeuU,ef->afuU", tn(p1, {chi, chi, Dk, Db}), false, Ct(2), false, tn(p0, {chi, chi, Dk, Db})));
  CK(ein(c, "afuU,fg->aguU", tn(p0, {chi, chi, Dk, Db}), false, Ct(3), false, tn(p1, {chi, chi, Dk, Db})));
  CK(ein(c, "aguU,gauU->", tn(p1, {chi, chi, Dk, Db}), false, Tt(3), false, tn(c->dscal + 36, {})));
  double h[16];
  CTM_CUDA_OK(cudaMemcpyAsync(h, c->dscal + 24, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(check_err(c));
  const double z1 = h[0], z0 = h[4], z13 = h[8], z24 = h[12];
  const double ratio = z1 * z0 / (z13 * z24);
  if (!(ratio > 0.0)) return fail(c, CTM_ENUMERIC, "non-positive kappa");
  *ln_kappa = std::log(ratio);
  return CTM_OK;
}

ctm_status ctm_get_projectors(ctm_ctx* c, ctm_dir dir, int x, int y, void* Pl, void* PrH) {
  if (!c || !Pl || !PrH) return fail(c, CTM_EINVAL, "NULL argument");
  if ((int)dir != c->last_dir) return fail(c, CTM_EINVAL, "projectors are kept for the last move only");
  const int r = (int)dir;
  const int Lxf = (r & 1) ? c->Ly : c->Lx, Lyf = (r & 1) ? c->Lx : c->Ly;
  if (x < 0 || y < 0 || x >= Lxf || y >= Lyf) return fail(c, CTM_EINVAL, "bad cut");
  Guard gd(c);
  const size_t NC = (size_t)c->N * c->chi;
  const int cut = y * Lxf + x;
  CTM_CUDA_OK(cudaMemcpyAsync(Pl, at(c->lastPl, cut * NC, c), NC * c->es, cudaMemcpyDeviceToHost, c->stream));
  CTM_CUDA_OK(cudaMemcpyAsync(PrH, at(c->lastPrH, cut * NC, c), NC * c->es, cudaMemcpyDeviceToHost, c->stream));
  CTM_CUDA_OK(cudaStreamSynchronize(c->stream));
  return CTM_OK;
}

ctm_status ctm_corner(ctm_ctx* c, ctm_dir dir, int x, int y, int i, void* Q_out) {
  if (!c || !Q_out) return fail(c, CTM_EINVAL, "NULL argument");
  const int r = (int)dir;
  if (r < 0 || r > 3 || i < 1 || i > 4) return fail(c, CTM_EINVAL, "bad direction or corner");
  const int Lxf = (r & 1) ? c->Ly : c->Lx, Lyf = (r & 1) ? c->Lx : c->Ly;
  if (x < 0 || y < 0 || x >= Lxf || y >= Lyf) return fail(c, CTM_EINVAL, "bad cut");
  Guard gd(c);
  use_lane(c, 0);
  CK(enlarged_corner(c, r, i - 1, x, y, c->Q[i - 1]));
  CTM_CUDA_OK(cudaMemcpyAsync(Q_out, c->Q[i - 1], (size_t)c->N * c->N * c->es,
                              cudaMemcpyDeviceToHost, c->stream));
  CK(check_err(c));
  return CTM_OK;
}

ctm_status ctm_corner_apply(ctm_ctx* c, ctm_dir dir, int x, int y, int i, int herm,
                            const void* Z_in, void* Z_out) {
  if (!c || !Z_in || !Z_out) return fail(c, CTM_EINVAL, "NULL argument");
  const int r = (int)dir;
  if (r < 0 || r > 3 || i < 1 || i > 4) return fail(c, CTM_EINVAL, "bad direction or corner");
  const int Lxf = (r & 1) ? c->Ly : c->Lx, Lyf = (r & 1) ? c->Lx : c->Ly;
  if (x < 0 || y < 0 || x >= Lxf || y >= Lyf) return fail(c, CTM_EINVAL, "bad cut");
  Guard gd(c);
  use_lane(c, 0);
  const size_t Nk = (size_t)c->N * c->k;
  CK(enlarged_corner(c, r, i - 1, x, y, c->Q[i - 1]));
  if (c->split) {
    const ctm_status st = split_prepare_corners(c->split, c->Q, c->N, 1u << (i - 1), c->stream,
                                                &c->launches);
    if (st != CTM_OK) return fail(c, st, split_last_error(c->split));
  }
  CTM_CUDA_OK(cudaMemcpyAsync(c->Z[0], Z_in, Nk * c->es, cudaMemcpyHostToDevice, c->stream));
  CK(apply_corner(c, c->Q[i - 1], herm != 0, c->Z[0], c->Z[1]));
  CTM_CUDA_OK(cudaMemcpyAsync(Z_out, c->Z[1], Nk * c->es, cudaMemcpyDeviceToHost, c->stream));
  CK(check_err(c));
  return CTM_OK;
}

ctm_status ctm_transfer_spectrum(ctm_ctx* c, int dir, int row, int nvals, double* lam_out,
                                 double* xi_out) {
  if (!c || !lam_out) return fail(c, CTM_EINVAL, "NULL argument");
  if (dir < 0 || dir > 1) return fail(c, CTM_EINVAL, "dir must be 0 (along x) or 1 (along y)");
  const int r = dir;
  const int Lxf = (r & 1) ? c->Ly : c->Lx, Lyf = (r & 1) ? c->Lx : c->Ly;
  if (row < 0 || row >= Lyf) return fail(c, CTM_EINVAL, "bad row");
  const long chi = c->chi, Dk = c->Dk, Db = c->Db, n = chi * chi;
  if (nvals < 2 || nvals > 24 || nvals > n)
    return fail(c, CTM_EINVAL, "nvals must be in 2 .. min(24, chi^2)");
  Guard gd(c);
  ExactScope xs(c, refine_on(c));
  use_lane(c, 0);
  // subspace iteration with m vectors, Rayleigh-Ritz every 5 applications
  const int m = (int)std::min<long>(n, std::max(nvals + 4, 8));
  const size_t es = c->es, mark = c->scratch_off;
  void* V = scratch_alloc(c, (size_t)n * m * es);
  void* V2 = scratch_alloc(c, (size_t)n * m * es);
  void* Ta = scratch_alloc(c, (size_t)n * m * es);
  void* Tb = scratch_alloc(c, (size_t)n * m * es);
  void* G = scratch_alloc(c, (size_t)m * m * es);
  void* Li = scratch_alloc(c, (size_t)m * m * es);
  void* H = scratch_alloc(c, (size_t)m * m * es);
  double* ev = static_cast<double*>(scratch_alloc(c, 2 * 32 * sizeof(double)));
  int* st = static_cast<int*>(scratch_alloc(c, 64 * sizeof(int)));
  int* dead = st + 16;
  void* Wb = scratch_alloc(c, (size_t)n * m * Dk * Db * es);
  if (!V || !V2 || !Ta || !Tb || !G || !Li || !H || !ev || !st || !Wb)
    return fail(c, CTM_ENOMEM, "scratch arena too small for the transfer vectors");
  const int opH = c->cx ? OP_C : OP_T;
  CTM_CUDA_OK(hash_fill((long)(n * m * (c->cx ? 2 : 1)), 7919, static_cast<double*>(V), c->stream,
                        &c->launches));
  // Y = E_{Lxf-1}^T ... E_0^T V, the row's edges T1 above and T3 below
  // (the first contraction of each column reads its input into the
  // pipeline buffer, so the last column may write over the input block)
  auto apply = [&](void* X, void* Y) -> ctm_status {
    void* in = X;
    for (int x = 0; x < Lxf; ++x) {
      void* out = (x == Lxf - 1) ? Y : (in == Ta ? Tb : Ta);
      Tn W = tn(Wb, {chi, m, chi, Dk, Db});
      CK(ein(c, "adm,abuv->dmbuv", tn(in, {chi, chi, m}), false,
             tn(fT(c, r, 0, x, row), {chi, chi, Dk, Db}), false, W));
      CK(ein(c, "dmbuv,cduv->bcm", W, false, tn(fT(c, r, 2, x, row), {chi, chi, Dk, Db}), false,
             tn(out, {chi, chi, m})));
      in = out;
    }
    return CTM_OK;
  };
  // orthonormal columns of X (n x m), twice: Gram, Cholesky, X L^-H
  auto orth = [&](void* X) -> ctm_status {
    for (int pass = 0; pass < 2; ++pass) {
      CK(mm_small(c, opH, OP_N, m, m, n, X, m, X, m, G, m));
      CTM_CUDA_OK(chol_inv(c->cx, m, n, false, G, Li, 1, dead, c->err, c->stream, &c->launches));
      CK(mm_small(c, OP_N, opH, n, m, m, X, m, Li, m, V2, m));
      CTM_CUDA_OK(repair_dead_columns(c->cx, n, m, V2, dead, 104729ull + pass, c->stream,
                                      &c->launches));
      CTM_CUDA_OK(cudaMemcpyAsync(X, V2, (size_t)n * m * es, cudaMemcpyDeviceToDevice, c->stream));
    }
    return CTM_OK;
  };
  CTM_CUDA_OK(cudaMemsetAsync(dead, 0, 16 * sizeof(int), c->stream));
  CK(orth(V));
  std::vector<double> h(2 * m), prev(2 * nvals, 0.0);
  double ratio = 0.0;
  bool conv = false;
  const int max_apply = 2000;
  for (int it = 1; it <= max_apply; ++it) {
    CK(apply(V, V));
    CK(orth(V));
    if (it % 5) continue;
    // Ritz values of the projected transfer matrix H = V^H E V
    CK(apply(V, V2));
    CK(mm_small(c, opH, OP_N, m, m, n, V, m, V2, m, H, m));
    CTM_CUDA_OK(small_eig(c->cx, m, H, ev, st, c->stream, &c->launches));
    int hst = 0;
    CTM_CUDA_OK(cudaMemcpyAsync(h.data(), ev, 2 * m * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CTM_CUDA_OK(cudaMemcpyAsync(&hst, st, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(check_err(c));
    if (hst < 0) return fail(c, CTM_ENOCONV, "small eigenproblem did not converge");
    const double a0 = std::hypot(h[0], h[1]);
    if (!(a0 > 0.0)) return fail(c, CTM_ENUMERIC, "zero transfer matrix");
    double change = 0.0;
    for (int i = 0; i < nvals; ++i) {
      const double ai = std::hypot(h[2 * i], h[2 * i + 1]) / a0;
      change = std::max(change, std::fabs(ai - prev[i]));
      prev[i] = ai;
    }
    ratio = prev[1];
    if (change < 1e-13) {
      conv = true;
      break;
    }
  }
  const double a0 = std::hypot(h[0], h[1]);
  for (int i = 0; i < nvals; ++i) {
    lam_out[2 * i] = h[2 * i] / a0;
    lam_out[2 * i + 1] = h[2 * i + 1] / a0;
  }
  if (xi_out) *xi_out = ratio > 0.0 ? -(double)Lxf / std::log(ratio) : 0.0;
  c->scratch_off = mark;
  if (!conv) return fail(c, CTM_ENOCONV, "transfer-matrix eigenvalues did not converge");
  return CTM_OK;
}

ctm_status ctm_si_stats(const ctm_ctx* c, long* updates, long* skipped) {
  if (!c) return CTM_EINVAL;
  if (updates) *updates = c->n_updates;
  if (skipped) *skipped = c->n_skipped;
  return CTM_OK;
}

ctm_status ctm_gemm_fp64tc(ctm_dtype dtype, int opA, const void* A, long lda, const void* B,
                           long ldb, int M, int N, int K, void* C, long ldc) {
  if ((dtype != CTM_F64 && dtype != CTM_C128) || opA < OP_N || opA > OP_C || !A || !B || !C ||
      M < 1 || N < 1 || K < 1 || ldb < N || ldc < N || lda < (opA == OP_N ? K : M))
    return fail(nullptr, CTM_EINVAL, "bad arguments of ctm_gemm_fp64tc");
  const bool cx = dtype == CTM_C128;
  const size_t es = cx ? 16 : 8;
  const size_t na = (size_t)(opA == OP_N ? M : K) * lda, nb = (size_t)K * ldb, nc = (size_t)M * ldc;
  void *dA = nullptr, *dB = nullptr, *dC = nullptr;
  int* err = nullptr;
  SplitCtx* sc = nullptr;
  cudaStream_t s = nullptr;
  ctm_status st = CTM_OK;
  auto done = [&](ctm_status r, const char* m) {
    if (sc) split_destroy(sc);
    if (dA) cudaFree(dA);
    if (dB) cudaFree(dB);
    if (dC) cudaFree(dC);
    if (err) cudaFree(err);
    if (s) cudaStreamDestroy(s);
    return r == CTM_OK ? CTM_OK : fail(nullptr, r, m);
  };
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&dA, na * es) != cudaSuccess || cudaMalloc(&dB, nb * es) != cudaSuccess ||
      cudaMalloc(&dC, nc * es) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return done(CTM_ENOMEM, "device allocation failed");
  }
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess ||
      cudaMemcpyAsync(dA, A, na * es, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dB, B, nb * es, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return done(CTM_ECUDA, "host to device copy failed");
  st = split_create(&sc, cx, false, 1, 1, err, s);
  if (st != CTM_OK) return done(st, "tensor-core product unavailable");
  st = oz_gemm(sc, opA, dA, lda, OP_N, dB, ldb, M, N, K, dC, ldc, s, nullptr);
  if (st != CTM_OK) return done(st, split_last_error(sc));
  int herr = 0;
  if (cudaMemcpyAsync(C, dC, nc * es, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return done(CTM_ECUDA, "device to host copy failed");
  if (herr) return done(CTM_ECUDA, "a bounded wait of the tensor-core product gave up");
  return done(CTM_OK, "");
}

void ctm_debug_fail_alloc(int after) { g_fail_alloc_after.store(after < 0 ? -1 : after); }

ctm_status ctm_last_timing(const ctm_ctx* c, double* ms, long* launches) {
  if (!c) return CTM_EINVAL;
  if (ms) *ms = c->last_ms;
  if (launches) *launches = c->last_launches;
  return CTM_OK;
}

ctm_status ctm_profile_enable(ctm_ctx* c, int on) {
  if (!c) return CTM_EINVAL;
  Guard gd(c);
  if (on && c->pev.empty()) {
    c->pev.resize(32768);
    c->pph.resize(c->pev.size() / 2);
    for (auto& e : c->pev)
      if (cudaEventCreate(&e) != cudaSuccess) return fail(c, CTM_ECUDA, "event creation failed");
  }
  c->prof = on != 0;
  c->pev_used = 0;
  for (double& v : c->phase_ms) v = 0.0;
  if (!c->split) return CTM_OK;
  for (size_t l = 0; l < std::max<size_t>(1, c->lanes.size()); ++l) {
    SplitCtx* sp = c->lanes.empty() ? c->split : c->lanes[l].split;
    const ctm_status st = split_profile(sp, on ? 1 : 0, nullptr, nullptr, nullptr, nullptr);
    if (st != CTM_OK) return fail(c, st, split_last_error(sp));
  }
  return CTM_OK;
}

ctm_status ctm_profile_read(ctm_ctx* c, double* ms, long* launches, double* flops,
                            double* bytes) {
  if (!c) return CTM_EINVAL;
  if (!c->split) return fail(c, CTM_EUNSUPPORTED, "profiling covers the split-precision kernel");
  Guard gd(c);
  double tms = 0, tfl = 0, tby = 0;
  long tl = 0;
  for (size_t l = 0; l < std::max<size_t>(1, c->lanes.size()); ++l) {
    SplitCtx* sp = c->lanes.empty() ? c->split : c->lanes[l].split;
    double m = 0, f = 0, b = 0;
    long n = 0;
    const ctm_status st = split_profile(sp, -1, &m, &n, &f, &b);
    if (st != CTM_OK) return fail(c, st, split_last_error(sp));
    tms += m; tl += n; tfl += f; tby += b;
  }
  if (ms) *ms = tms;
  if (launches) *launches = tl;
  if (flops) *flops = tfl;
  if (bytes) *bytes = tby;
  return CTM_OK;
}

ctm_status ctm_profile_phases(ctm_ctx* c, double ms[CTM_NPHASES]) {
  if (!c || !ms) return CTM_EINVAL;
  Guard gd(c);
  phases_fold(c);
  for (int i = 0; i < CTM_NPHASES; ++i) ms[i] = c->phase_ms[i];
  return CTM_OK;
}

void ctm_free(ctm_ctx* c) {
  if (!c) return;
  use_lane(c, 0);
  grad_destroy(c);
  for (auto& L : c->lanes)
    if (L.stream) cudaStreamSynchronize(L.stream);
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& e : c->pev) cudaEventDestroy(e);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->split) split_destroy(c->split);
  for (size_t l = 1; l < c->lanes.size(); ++l) {
    if (c->lanes[l].split) split_destroy(c->lanes[l].split);
    if (c->lanes[l].stream) cudaStreamDestroy(c->lanes[l].stream);
  }
  for (auto& L : c->lanes)
    if (L.ev) cudaEventDestroy(L.ev);
  if (c->svd) svd_destroy(c->svd);
  for (void* p : c->allocs) cudaFree(p);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* ctm_last_error(const ctm_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->msg.c_str();
}

}  // extern "C"
