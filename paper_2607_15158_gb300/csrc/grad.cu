// Reverse-mode differentiation of SI-CTMRG (hand-written adjoints).
//
// Paper, section "Variational optimization": the energy gradient with
// respect to the on-site tensors is obtained by recording the forward CTMRG
// and applying the chain rule in reverse ("unrolled" differentiation, the
// form the paper times); section "Differentiable fixed point", Eq. implicit:
// at the fixed point x = F(x, A) the gradient is
// dg/dA + dg/dx [I - dF/dx]^-1 dF/dA, solved by iterating vector-Jacobian
// products of one CTMRG step.
//
// Design. While recording, every move saves a checkpoint of its input state
// (C, T and the rangefinders of its direction, on the device). The backward
// pass recomputes each move from its checkpoint on a tape (the enlarged
// corners and half-system products included: recomputation instead of
// storage), in fp64 through the same einsum-to-GEMM contractions as the
// forward, then sweeps the tape in reverse with these adjoints:
//   contraction O = A.B       dA += O'.B, dB += A.O' (einsum specs swapped)
//   QR Z = Q R (R_ii > 0)     dZ += [dQ - Q sym(triu(Q^T dQ))] R^-T
//   SVD rho = u s v^T         drho += u [diag(ds) + (F o (J - J^T)) s
//     (full, sign fixed)             + s (F o (K - K^T))] v^T,
//                             J = u^T du, K = v^T dv, F_ij = 1/(s_j^2 - s_i^2)
//                             with its factor 1/(s_j - s_i) Lorentzian-
//                             broadened, (s_j - s_i) / ((s_j - s_i)^2 + eps),
//                             eps = (1e-12 s_1)^2
//   V s^-1/2                  dV += dVs s^-1/2, ds_j -= 1/2 s_j^-3/2 <dVs_j, V_j>
//   t' = sign t / ||t||       dt += (sign / ||t||) (dt' - t' <t', dt'>)
//   permutes                  inverse permutes
//   e = Tr(op rho) / Tr rho   drho += de (op^T - e I) / Tr rho
// Sign fixes, pivots and the cutoff mask are piecewise constant and carry no
// derivative. Real (CTM_F64) iPEPS contexts in fp64 with SI projectors.
#include <cmath>
#include <cstring>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "ctx.h"

using namespace ctm;

namespace ctmi {

struct Checkpoint {
  int r = 0;
  void* C = nullptr;           // all corners before the move
  void* T = nullptr;           // all edges
  void* X = nullptr;           // [S][N k] rangefinders of direction r
  void* W = nullptr;
  std::vector<char> ready;     // rf_ready of direction r, per cut
  int moves_done = 0;          // moves made in direction r before this one
};

struct GradState {
  bool recording = false;
  std::vector<Checkpoint> cps;
  void release() {
    for (auto& cp : cps) {
      cudaFree(cp.C);
      cudaFree(cp.T);
      cudaFree(cp.X);
      cudaFree(cp.W);
    }
    cps.clear();
  }
};

namespace {

// ---------------------------------------------------------------- kernels
unsigned blocks_for(long n) {
  long b = (n + 255) / 256;
  if (b > 152L * 16) b = 152L * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

__global__ void axpy_kernel(long n, double a, const double* x, double* y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

// S = triu(P) + triu(P, 1)^T (k x k)
__global__ void sym_upper_kernel(int k, const double* P, double* S) {
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)k * k;
       idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / k), j = (int)(idx % k);
    S[idx] = i <= j ? P[(long)i * k + j] : P[(long)j * k + i];
  }
}

// y = x - y
__global__ void rsub_kernel(long n, const double* x, double* y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = x[i] - y[i];
}

// X = R^-1 for the upper triangle of R (k x k): thread c solves R x = e_c by
// back substitution (x_j = 0 for j > c)
__global__ void inv_upper_kernel(int k, const double* R, double* X) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  for (int j = k - 1; j > c; --j) X[(long)j * k + c] = 0.0;
  for (int j = c; j >= 0; --j) {
    double acc = j == c ? 1.0 : 0.0;
    for (int i = j + 1; i <= c; ++i) acc -= R[(long)j * k + i] * X[(long)i * k + c];
    X[(long)j * k + c] = acc / R[(long)j * k + j];
  }
}

// inner = diag(ds) + (F o (J - J^T)) s + s (F o (K - K^T)) (k x k) with
// F_ij = 1 / (s_j^2 - s_i^2), written as
//   inner_ij = 1/2 (a + b)_ij L(s_j - s_i) + 1/2 (a - b)_ij / (s_i + s_j),
// a = J - J^T, b = K - K^T, and the Lorentzian L(x) = x / (x^2 + eps)
// broadening only the factor 1 / (s_j - s_i): its numerator a + b (a joint
// rotation of u_i, u_j and v_i, v_j) vanishes for losses that do not depend
// on the basis inside a degenerate pair, while the second term stays finite
// and must be kept (broadening the whole F drops it when the tail of rho's
// spectrum is nearly degenerate, as the recycled bases make it)
__global__ void svd_inner_kernel(int k, const double* J, const double* K, const double* s,
                                 const double* ds, double* inner) {
  const double w = 1e-12 * s[0];
  const double eps = w * w;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < (long)k * k;
       idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / k), j = (int)(idx % k);
    double v = 0.0;
    if (i == j) {
      v = ds ? ds[i] : 0.0;
    } else {
      const double aij = J ? (J[(long)i * k + j] - J[(long)j * k + i]) : 0.0;
      const double bij = K ? (K[(long)i * k + j] - K[(long)j * k + i]) : 0.0;
      const double dm = s[j] - s[i], sp = s[j] + s[i];
      v = 0.5 * (aij + bij) * dm / (dm * dm + eps);
      if (sp > 0.0) v += 0.5 * (aij - bij) / sp;
    }
    inner[idx] = v;
  }
}

// dV[:, :c] += dVs s^-1/2 and ds_j -= 1/2 s_j^-3/2 sum_i dVs_ij V_ij for the
// kept columns (s_j > cutoff s_0); one block, thread per column
__global__ void scale_bwd_kernel(int k, int c, const double* V, const double* s, double cutoff,
                                 const double* dVs, double* dV, double* ds) {
  for (int j = threadIdx.x; j < c; j += blockDim.x) {
    if (!(s[j] > cutoff * s[0])) continue;
    const double is = 1.0 / sqrt(s[j]);
    double acc = 0.0;
    for (int i = 0; i < k; ++i) {
      const double g = dVs[(long)i * c + j];
      if (dV) dV[(long)i * k + j] += g * is;
      acc += g * V[(long)i * k + j];
    }
    if (ds) ds[j] += -0.5 * is * is * is * acc;
  }
}

// deterministic dot product: partial sums per block, then one block
__global__ void dot_partial_kernel(long n, const double* x, const double* y, double* part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    acc = fma(x[i], y[i], acc);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
__global__ void sum_kernel(int n, const double* part, double* out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// dt += f (dt' - t' <t', dt'>), f = the factor the forward applied
__global__ void norm_bwd_kernel(long n, const double* tp, const double* dtp, const double* fac,
                                const double* dot, double* dt) {
  const double f = fac[0], d = dot[0];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    dt[i] += f * (dtp[i] - tp[i] * d);
}

// e = sum_ij op_ij rho_ji / sum_i rho_ii; aux = (e, Tr rho)
__global__ void energy_fwd_kernel(int d2, const double* op, const double* rho, double* aux) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double num = 0.0, tr = 0.0;
  for (int i = 0; i < d2; ++i) {
    tr += rho[(long)i * d2 + i];
    for (int j = 0; j < d2; ++j) num += op[(long)i * d2 + j] * rho[(long)j * d2 + i];
  }
  aux[0] = num / tr;
  aux[1] = tr;
}
// drho_ji += de (op_ij - e delta_ij) / Tr rho
__global__ void energy_bwd_kernel(int d2, const double* op, const double* aux, const double* de,
                                  double* drho) {
  const double e = aux[0], tr = aux[1], g = de[0];
  for (int idx = threadIdx.x; idx < d2 * d2; idx += blockDim.x) {
    const int j = idx / d2, i = idx % d2;
    drho[idx] += g * (op[(long)i * d2 + j] - (i == j ? e : 0.0)) / tr;
  }
}

// sum of (a - b)^2 and of a^2 into out[0], out[1] (atomic, per launch)
__global__ void diff_norm_kernel(long n, const double* a, const double* b, double* out) {
  __shared__ double s1[256], s2[256];
  double x = 0.0, y = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double d = a[i] - b[i];
    x = fma(d, d, x);
    y = fma(a[i], a[i], y);
  }
  s1[threadIdx.x] = x;
  s2[threadIdx.x] = y;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(out, s1[0]);
    atomicAdd(out + 1, s2[0]);
  }
}

// ------------------------------------------------------------------ arena
// Device bump allocator in large chunks; released as a whole.
class Arena {
 public:
  ~Arena() { release(); }
  void* get(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    if (chunks_.empty() || off_ + bytes > caps_.back()) {
      const size_t cap = std::max(bytes, (size_t)256 << 20);
      void* p = nullptr;
      if (cudaMalloc(&p, cap) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      chunks_.push_back(p);
      caps_.push_back(cap);
      off_ = 0;
    }
    void* p = static_cast<char*>(chunks_.back()) + off_;
    off_ += bytes;
    return p;
  }
  void release() {
    for (void* p : chunks_) cudaFree(p);
    chunks_.clear();
    caps_.clear();
    off_ = 0;
  }

 private:
  std::vector<void*> chunks_;
  std::vector<size_t> caps_;
  size_t off_ = 0;
};

// ------------------------------------------------------------------- tape
enum Kind { K_EIN, K_PERM, K_QR, K_SVD, K_SCALE, K_NORM, K_ENERGY };

struct Node {
  Kind kind;
  std::string spec;     // K_EIN
  Tn a, b, o;           // K_EIN operands; K_PERM: a -> o
  int perm[8] = {0};    // K_PERM
  void* p[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  long n = 0;           // K_NORM: elements; K_SCALE: chi; K_ENERGY: d^2
};

struct Tape {
  ctm_ctx* c;
  Arena vals, adjs, tmp;
  std::vector<Node> nodes;
  std::unordered_map<void*, void*> adj;
  std::unordered_map<void*, long> len;      // elements of each recorded value
  std::unordered_set<void*> constant;       // values with no adjoint
  double* dwork = nullptr;                  // reduction scratch (>= 2 + 2432)
  explicit Tape(ctm_ctx* cc) : c(cc) {}

  cudaStream_t st() const { return c->stream; }

  void* val(long n) {
    void* p = vals.get((size_t)n * 8);
    if (p) len[p] = n;
    return p;
  }
  void* tmpbuf(long n) { return tmp.get((size_t)n * 8); }
  // the adjoint of value v (n elements), created zero on first use
  void* adj_of(void* v, long n) {
    auto it = adj.find(v);
    if (it != adj.end()) return it->second;
    void* a = adjs.get((size_t)n * 8);
    if (!a) return nullptr;
    if (cudaMemsetAsync(a, 0, (size_t)n * 8, st()) != cudaSuccess) return nullptr;
    adj[v] = a;
    return a;
  }
  void* adj_if(void* v) const {
    auto it = adj.find(v);
    return it == adj.end() ? nullptr : it->second;
  }
  void reset_adjoints() {
    adj.clear();
    adjs.release();
  }
};

ctm_status nomem(ctm_ctx* c) { return fail(c, CTM_ENOMEM, "device memory for the gradient tape"); }

ctm_status axpy(Tape& T, long n, double a, const void* x, void* y) {
  axpy_kernel<<<blocks_for(n), 256, 0, T.st()>>>(n, a, (const double*)x, (double*)y);
  ++T.c->launches;
  CTM_CUDA_OK(cudaGetLastError());
  return CTM_OK;
}

// ---------------------------------------------------------- forward ops
ctm_status ein_t(Tape& T, const char* spec, const Tn& A, const Tn& B,
                 std::initializer_list<long> dims, Tn* out) {
  Tn o = tn(nullptr, dims);
  o.p = T.val(o.size());
  if (!o.p) return nomem(T.c);
  CK(ein(T.c, spec, A, false, B, false, o));
  Node nd;
  nd.kind = K_EIN;
  nd.spec = spec;
  nd.a = A;
  nd.b = B;
  nd.o = o;
  T.nodes.push_back(nd);
  *out = o;
  return CTM_OK;
}

ctm_status perm_t(Tape& T, const Tn& A, const int* perm, Tn* out) {
  Tn o;
  o.r = A.r;
  for (int j = 0; j < A.r; ++j) o.d[j] = A.d[perm[j]];
  o.p = T.val(o.size());
  if (!o.p) return nomem(T.c);
  CTM_CUDA_OK(permute(A.p, o.p, A.r, A.d, perm, false, false, T.st(), &T.c->launches));
  Node nd;
  nd.kind = K_PERM;
  nd.a = A;
  nd.o = o;
  for (int j = 0; j < A.r; ++j) nd.perm[j] = perm[j];
  T.nodes.push_back(nd);
  *out = o;
  return CTM_OK;
}

// Q of Z (N x k) by the library's CholeskyQR: R has a positive diagonal, so
// Q is the unique factor whose derivative the adjoint below is
ctm_status qr_t(Tape& T, void* Z, void** Q) {
  ctm_ctx* c = T.c;
  const long nk = (long)c->N * c->k;
  void* q = T.val(nk);
  void* w = T.tmpbuf(nk);
  if (!q || !w) return nomem(c);
  CTM_CUDA_OK(cudaMemcpyAsync(q, Z, nk * 8, cudaMemcpyDeviceToDevice, T.st()));
  CK(qr_inplace(c, q, w, false));
  Node nd;
  nd.kind = K_QR;
  nd.p[0] = Z;
  nd.p[1] = q;
  T.nodes.push_back(nd);
  *Q = q;
  return CTM_OK;
}

// rho = u s v^T (k x k, descending s) with the sign fix of step 4
ctm_status svd_t(Tape& T, void* rho, void** u, void** s, void** v) {
  ctm_ctx* c = T.c;
  const int k = c->k;
  void* U = T.val((long)k * k);
  void* V = T.val((long)k * k);
  void* S = T.val(k);
  if (!U || !V || !S) return nomem(c);
  CTM_CUDA_OK(jacobi_svd_coop(false, k, rho, (long)k * k, (double*)S, U, V, true, c->jw, 1,
                              c->opts.svd_max_sweeps, c->err, c->num_sms, T.st(), &c->launches));
  if (c->opts.sign_fix) {
    CTM_CUDA_OK(column_phase(false, k, k, k, U, c->ph, 1, 0, T.st(), &c->launches));
    CTM_CUDA_OK(scale_columns_conj(false, k, k, k, U, c->ph, T.st(), &c->launches));
    CTM_CUDA_OK(scale_columns_conj(false, k, k, k, V, c->ph, T.st(), &c->launches));
  }
  Node nd;
  nd.kind = K_SVD;
  nd.p[0] = rho;
  nd.p[1] = U;
  nd.p[2] = S;
  nd.p[3] = V;
  T.nodes.push_back(nd);
  *u = U;
  *s = S;
  *v = V;
  return CTM_OK;
}

// Vs = V[:, :chi] s^-1/2 (cutoff)
ctm_status scale_t(Tape& T, void* V, void* s, void** Vs) {
  ctm_ctx* c = T.c;
  void* o = T.val((long)c->k * c->chi);
  if (!o) return nomem(c);
  CTM_CUDA_OK(scale_by_inv_sqrt(false, c->k, c->chi, V, (const double*)s, c->opts.svd_rel_cutoff,
                                o, T.st(), &c->launches));
  Node nd;
  nd.kind = K_SCALE;
  nd.p[0] = V;
  nd.p[1] = s;
  nd.p[2] = o;
  nd.n = c->chi;
  T.nodes.push_back(nd);
  *Vs = o;
  return CTM_OK;
}

// t' = t sign(pivot) / ||t|| (the normalisation of a move's outputs)
ctm_status norm_t(Tape& T, void* t, long n, void** out) {
  ctm_ctx* c = T.c;
  void* o = T.val(n);
  double* fac = static_cast<double*>(T.val(1));
  double* w = static_cast<double*>(T.tmpbuf(3 * 152));
  if (!o || !fac || !w) return nomem(c);
  CTM_CUDA_OK(cudaMemcpyAsync(o, t, n * 8, cudaMemcpyDeviceToDevice, T.st()));
  CTM_CUDA_OK(normalize_phase(false, n, o, n, 1, fac, w, T.st(), &c->launches));
  Node nd;
  nd.kind = K_NORM;
  nd.p[0] = t;
  nd.p[1] = o;
  nd.p[2] = fac;
  nd.n = n;
  T.nodes.push_back(nd);
  *out = o;
  return CTM_OK;
}

// e = Tr(op rho) / Tr rho for a d^2 x d^2 rho (value: aux[0])
ctm_status energy_t(Tape& T, void* rho, void* op, int d2, void** e) {
  double* aux = static_cast<double*>(T.val(2));
  if (!aux) return nomem(T.c);
  energy_fwd_kernel<<<1, 32, 0, T.st()>>>(d2, (const double*)op, (const double*)rho, aux);
  ++T.c->launches;
  CTM_CUDA_OK(cudaGetLastError());
  Node nd;
  nd.kind = K_ENERGY;
  nd.p[0] = rho;
  nd.p[1] = aux;
  nd.p[2] = op;
  nd.n = d2;
  T.nodes.push_back(nd);
  *e = aux;
  return CTM_OK;
}

// ---------------------------------------------------------- reverse sweep
void labels(const std::string& spec, std::string* la, std::string* lb, std::string* lo) {
  const size_t comma = spec.find(','), arrow = spec.find("->");
  *la = spec.substr(0, comma);
  *lb = spec.substr(comma + 1, arrow - comma - 1);
  *lo = spec.substr(arrow + 2);
}

ctm_status backward(Tape& T) {
  ctm_ctx* c = T.c;
  const int k = c->k;
  const long N = c->N;
  const long nk = N * k;
  for (size_t ii = T.nodes.size(); ii-- > 0;) {
    Node& nd = T.nodes[ii];
    switch (nd.kind) {
      case K_EIN: {
        void* go = T.adj_if(nd.o.p);
        if (!go) break;
        std::string la, lb, lo;
        labels(nd.spec, &la, &lb, &lo);
        Tn g = nd.o;
        g.p = go;
        if (!T.constant.count(nd.a.p)) {
          Tn t = nd.a;
          t.p = T.tmpbuf(nd.a.size());
          void* ga = T.adj_of(nd.a.p, nd.a.size());
          if (!t.p || !ga) return nomem(c);
          CK(ein(c, (lo + "," + lb + "->" + la).c_str(), g, false, nd.b, false, t));
          CK(axpy(T, nd.a.size(), 1.0, t.p, ga));
        }
        if (!T.constant.count(nd.b.p)) {
          Tn t = nd.b;
          t.p = T.tmpbuf(nd.b.size());
          void* gb = T.adj_of(nd.b.p, nd.b.size());
          if (!t.p || !gb) return nomem(c);
          CK(ein(c, (la + "," + lo + "->" + lb).c_str(), nd.a, false, g, false, t));
          CK(axpy(T, nd.b.size(), 1.0, t.p, gb));
        }
        break;
      }
      case K_PERM: {
        void* go = T.adj_if(nd.o.p);
        if (!go || T.constant.count(nd.a.p)) break;
        int inv[8];
        for (int j = 0; j < nd.a.r; ++j) inv[nd.perm[j]] = j;
        void* t = T.tmpbuf(nd.a.size());
        void* ga = T.adj_of(nd.a.p, nd.a.size());
        if (!t || !ga) return nomem(c);
        CTM_CUDA_OK(permute(go, t, nd.o.r, nd.o.d, inv, false, false, T.st(), &c->launches));
        CK(axpy(T, nd.a.size(), 1.0, t, ga));
        break;
      }
      case K_QR: {
        void* gq = T.adj_if(nd.p[1]);
        if (!gq || T.constant.count(nd.p[0])) break;
        void* Z = nd.p[0];
        void* Q = nd.p[1];
        void* P = T.tmpbuf((long)k * k);
        void* S = T.tmpbuf((long)k * k);
        void* R = T.tmpbuf((long)k * k);
        void* Ri = T.tmpbuf((long)k * k);
        void* G = T.tmpbuf(nk);
        void* t = T.tmpbuf(nk);
        void* gz = T.adj_of(Z, nk);
        if (!P || !S || !R || !Ri || !G || !t || !gz) return nomem(c);
        // P = Q^T dQ, S = sym(triu P), G = dQ - Q S
        CK(mm_small(c, OP_T, OP_N, k, k, N, Q, k, gq, k, P, k));
        sym_upper_kernel<<<blocks_for((long)k * k), 256, 0, T.st()>>>(k, (const double*)P, (double*)S);
        CK(mm_small(c, OP_N, OP_N, N, k, k, Q, k, S, k, G, k));
        rsub_kernel<<<blocks_for(nk), 256, 0, T.st()>>>(nk, (const double*)gq, (double*)G);
        // R = Q^T Z (upper triangular), dZ += G R^-T
        CK(mm_small(c, OP_T, OP_N, k, k, N, Q, k, Z, k, R, k));
        inv_upper_kernel<<<(k + 127) / 128, 128, 0, T.st()>>>(k, (const double*)R, (double*)Ri);
        c->launches += 3;
        CK(mm_small(c, OP_N, OP_T, N, k, k, G, k, Ri, k, t, k));
        CK(axpy(T, nk, 1.0, t, gz));
        break;
      }
      case K_SVD: {
        void* gu = T.adj_if(nd.p[1]);
        void* gs = T.adj_if(nd.p[2]);
        void* gv = T.adj_if(nd.p[3]);
        if ((!gu && !gs && !gv) || T.constant.count(nd.p[0])) break;
        void* U = nd.p[1];
        void* V = nd.p[3];
        void* J = gu ? T.tmpbuf((long)k * k) : nullptr;
        void* K = gv ? T.tmpbuf((long)k * k) : nullptr;
        void* inner = T.tmpbuf((long)k * k);
        void* t1 = T.tmpbuf((long)k * k);
        void* t2 = T.tmpbuf((long)k * k);
        void* grho = T.adj_of(nd.p[0], (long)k * k);
        if (!inner || !t1 || !t2 || !grho || (gu && !J) || (gv && !K)) return nomem(c);
        if (gu) CK(mm_small(c, OP_T, OP_N, k, k, k, U, k, gu, k, J, k));
        if (gv) CK(mm_small(c, OP_T, OP_N, k, k, k, V, k, gv, k, K, k));
        svd_inner_kernel<<<blocks_for((long)k * k), 256, 0, T.st()>>>(
            k, (const double*)J, (const double*)K, (const double*)nd.p[2], (const double*)gs,
            (double*)inner);
        ++c->launches;
        CK(mm_small(c, OP_N, OP_N, k, k, k, U, k, inner, k, t1, k));
        CK(mm_small(c, OP_N, OP_T, k, k, k, t1, k, V, k, t2, k));
        CK(axpy(T, (long)k * k, 1.0, t2, grho));
        break;
      }
      case K_SCALE: {
        void* go = T.adj_if(nd.p[2]);
        if (!go) break;
        void* gV = T.constant.count(nd.p[0]) ? nullptr : T.adj_of(nd.p[0], (long)k * k);
        void* gs = T.constant.count(nd.p[1]) ? nullptr : T.adj_of(nd.p[1], k);
        scale_bwd_kernel<<<1, 256, 0, T.st()>>>(k, (int)nd.n, (const double*)nd.p[0],
                                                (const double*)nd.p[1], c->opts.svd_rel_cutoff,
                                                (const double*)go, (double*)gV, (double*)gs);
        ++c->launches;
        break;
      }
      case K_NORM: {
        void* go = T.adj_if(nd.p[1]);
        if (!go || T.constant.count(nd.p[0])) break;
        void* gt = T.adj_of(nd.p[0], nd.n);
        if (!gt) return nomem(c);
        const unsigned nb = std::min(blocks_for(nd.n), 2048u);
        dot_partial_kernel<<<nb, 256, 0, T.st()>>>(nd.n, (const double*)nd.p[1], (const double*)go,
                                                   T.dwork + 2);
        sum_kernel<<<1, 256, 0, T.st()>>>((int)nb, T.dwork + 2, T.dwork);
        norm_bwd_kernel<<<blocks_for(nd.n), 256, 0, T.st()>>>(
            nd.n, (const double*)nd.p[1], (const double*)go, (const double*)nd.p[2], T.dwork,
            (double*)gt);
        c->launches += 3;
        break;
      }
      case K_ENERGY: {
        void* ge = T.adj_if(nd.p[1]);
        if (!ge) break;
        const int d2 = (int)nd.n;
        void* gr = T.adj_of(nd.p[0], (long)d2 * d2);
        if (!gr) return nomem(c);
        energy_bwd_kernel<<<1, 256, 0, T.st()>>>(d2, (const double*)nd.p[2], (const double*)nd.p[1],
                                                 (const double*)ge, (double*)gr);
        ++c->launches;
        break;
      }
    }
    CTM_CUDA_OK(cudaGetLastError());
  }
  return CTM_OK;
}

// ------------------------------------------------------- move and energy
// Values of one state: corners and edges [label * S + site], the base tensor
// A of each site and its four rotations (ket = bra for a real iPEPS).
struct StateVals {
  std::vector<void*> C, T;      // 4 S each
  std::vector<void*> A;         // S base tensors
  std::vector<void*> rot[4];    // S rotated tensors each
  std::vector<void*> X[4], W[4];  // S rangefinders per direction
};

ctm_status make_rotations(Tape& T, StateVals& s) {
  ctm_ctx* c = T.c;
  static const int rot[4][5] = {{0, 1, 2, 3, 4}, {0, 4, 1, 2, 3}, {0, 3, 4, 1, 2}, {0, 2, 3, 4, 1}};
  const long d = c->d, D = c->Dk;
  for (int r = 0; r < 4; ++r) s.rot[r].assign(c->S, nullptr);
  for (int i = 0; i < c->S; ++i) {
    s.rot[0][i] = s.A[i];
    for (int r = 1; r < 4; ++r) {
      Tn out;
      CK(perm_t(T, tn(s.A[i], {d, D, D, D, D}), rot[r], &out));
      s.rot[r][i] = out.p;
    }
  }
  return CTM_OK;
}

// One left move of the frame turned by r, recorded on T: the same steps as
// the library's fp64 move (enlarged corners as pairwise contractions, a QR
// after each application of M or M^T, small SVD, projectors, recycling,
// absorption with the A, B absorption as two contractions, normalisation).
ctm_status tape_move(Tape& T, StateVals& s, int r, const std::vector<char>& ready,
                     int moves_done) {
  ctm_ctx* c = T.c;
  const long chi = c->chi, Dk = c->Dk, Db = c->Db, d = c->d, N = c->N, k = c->k;
  const int S = c->S;
  const int Lxf = (r & 1) ? c->Ly : c->Lx, Lyf = (r & 1) ? c->Lx : c->Ly;
  auto Cv = [&](int i, int x, int y) { return s.C[frame_label(r, i) * S + frame_site(c, r, x, y)]; };
  auto Tv = [&](int i, int x, int y) { return s.T[frame_label(r, i) * S + frame_site(c, r, x, y)]; };
  const bool warm = moves_done < c->opts.warmup_iters;
  const int rounds = warm ? c->opts.warmup_rounds : c->opts.si_rounds;
  static const int dx[4] = {0, 1, 1, 0}, dy[4] = {0, 0, 1, 1};
  auto apply = [&](void* Q, bool herm, void* Z, void** out) -> ctm_status {
    Tn o;
    CK(ein_t(T, herm ? "ba,bc->ac" : "ab,bc->ac", tn(Q, {N, N}), tn(Z, {N, k}), {N, k}, &o));
    *out = o.p;
    return CTM_OK;
  };
  for (int x = 0; x < Lxf; ++x) {
    std::vector<void*> Pl(Lyf), PrH(Lyf);
    for (int y = 0; y < Lyf; ++y) {
      void* Q[4];
      for (int i = 0; i < 4; ++i) {
        const int sx = x + dx[i], sy = y + dy[i];
        const int site = frame_site(c, r, sx, sy);
        void* A = s.rot[(r + i) & 3][site];
        Tn CT, CTT, R1, Qt;
        CK(ein_t(T, "pm,mnuv->pnuv", tn(Cv(i, sx, sy), {chi, chi}),
                 tn(Tv(i, sx, sy), {chi, chi, Dk, Db}), {chi, chi, Dk, Db}, &CT));
        CK(ein_t(T, "tplw,pnuv->tlwnuv", tn(Tv((i + 3) & 3, sx, sy), {chi, chi, Dk, Db}), CT,
                 {chi, Dk, Db, chi, Dk, Db}, &CTT));
        CK(ein_t(T, "tlwnuv,sulde->twnvsde", CTT, tn(A, {d, Dk, Dk, Dk, Dk}),
                 {chi, Db, chi, Db, d, Dk, Dk}, &R1));
        CK(ein_t(T, "twnvsde,svwDE->tdDneE", R1, tn(A, {d, Db, Db, Db, Db}),
                 {chi, Dk, Db, chi, Dk, Db}, &Qt));
        Q[i] = Qt.p;
      }
      const int cut = y * Lxf + x;
      void* X = s.X[r][cut];
      void* W = s.W[r][cut];
      if (!ready[cut]) {
        CK(qr_t(T, X, &X));
        CK(qr_t(T, W, &W));
      }
      for (int round = 0; round < rounds; ++round) {
        void *a, *b;
        // X <- qr(M^T qr(M X)), M = Q3 Q4 Q1 Q2
        CK(apply(Q[1], false, X, &a));
        CK(apply(Q[0], false, a, &b));
        CK(apply(Q[3], false, b, &a));
        CK(apply(Q[2], false, a, &b));
        CK(qr_t(T, b, &b));
        CK(apply(Q[2], true, b, &a));
        CK(apply(Q[3], true, a, &b));
        CK(apply(Q[0], true, b, &a));
        CK(apply(Q[1], true, a, &b));
        CK(qr_t(T, b, &X));
        // W <- qr(M qr(M^T W))
        CK(apply(Q[2], true, W, &a));
        CK(apply(Q[3], true, a, &b));
        CK(apply(Q[0], true, b, &a));
        CK(apply(Q[1], true, a, &b));
        CK(qr_t(T, b, &b));
        CK(apply(Q[1], false, b, &a));
        CK(apply(Q[0], false, a, &b));
        CK(apply(Q[3], false, b, &a));
        CK(apply(Q[2], false, a, &b));
        CK(qr_t(T, b, &W));
      }
      void *a, *ZR, *ZL;
      CK(apply(Q[1], false, X, &a));
      CK(apply(Q[0], false, a, &ZR));
      CK(apply(Q[2], true, W, &a));
      CK(apply(Q[3], true, a, &ZL));
      Tn rho, Xn, Wn, tPl, tPr;
      CK(ein_t(T, "ba,bc->ac", tn(ZL, {N, k}), tn(ZR, {N, k}), {k, k}, &rho));
      void *u, *sv, *v, *Vs, *Us;
      CK(svd_t(T, rho.p, &u, &sv, &v));
      CK(ein_t(T, "ab,bc->ac", tn(X, {N, k}), tn(v, {k, k}), {N, k}, &Xn));
      CK(ein_t(T, "ab,bc->ac", tn(W, {N, k}), tn(u, {k, k}), {N, k}, &Wn));
      CK(scale_t(T, v, sv, &Vs));
      CK(scale_t(T, u, sv, &Us));
      CK(ein_t(T, "ab,bc->ac", tn(ZR, {N, k}), tn(Vs, {k, chi}), {N, chi}, &tPl));
      CK(ein_t(T, "ab,bc->ac", tn(ZL, {N, k}), tn(Us, {k, chi}), {N, chi}, &tPr));
      Pl[y] = tPl.p;
      PrH[y] = tPr.p;
      s.X[r][cut] = Xn.p;
      s.W[r][cut] = Wn.p;
    }
    std::vector<void*> nC1(Lyf), nT4(Lyf), nC4(Lyf);
    for (int y = 0; y < Lyf; ++y) {
      const int up = (y - 1 + Lyf) % Lyf, dn = y;
      const int site = frame_site(c, r, x, y);
      void* A = s.rot[r & 3][site];
      Tn E1, C1n, E4, C4n, Y1, R1, R2, T4n;
      CK(ein_t(T, "pm,mnuv->pnuv", tn(Cv(0, x, y), {chi, chi}), tn(Tv(0, x, y), {chi, chi, Dk, Db}),
               {chi, chi, Dk, Db}, &E1));
      CK(ein_t(T, "puva,pnuv->an", tn(PrH[up], {chi, Dk, Db, chi}), E1, {chi, chi}, &C1n));
      CK(ein_t(T, "tmdD,mn->tndD", tn(Tv(2, x, y), {chi, chi, Dk, Db}), tn(Cv(3, x, y), {chi, chi}),
               {chi, chi, Dk, Db}, &E4));
      CK(ein_t(T, "tndD,ndDc->tc", E4, tn(Pl[dn], {chi, Dk, Db, chi}), {chi, chi}, &C4n));
      CK(ein_t(T, "tqlw,quvc->tlwuvc", tn(Tv(3, x, y), {chi, chi, Dk, Db}),
               tn(Pl[up], {chi, Dk, Db, chi}), {chi, Dk, Db, Dk, Db, chi}, &Y1));
      CK(ein_t(T, "tlwuvc,sulde->twvcsde", Y1, tn(A, {d, Dk, Dk, Dk, Dk}),
               {chi, Db, Db, chi, d, Dk, Dk}, &R1));
      CK(ein_t(T, "twvcsde,svwDE->tdDceE", R1, tn(A, {d, Db, Db, Db, Db}),
               {chi, Dk, Db, chi, Dk, Db}, &R2));
      CK(ein_t(T, "tdDa,tdDceE->aceE", tn(PrH[dn], {chi, Dk, Db, chi}), R2, {chi, chi, Dk, Db},
               &T4n));
      nC1[y] = C1n.p;
      nT4[y] = T4n.p;
      nC4[y] = C4n.p;
      if (c->opts.normalize) {
        CK(norm_t(T, nC1[y], chi * chi, &nC1[y]));
        CK(norm_t(T, nT4[y], chi * chi * Dk * Db, &nT4[y]));
        CK(norm_t(T, nC4[y], chi * chi, &nC4[y]));
      }
    }
    for (int y = 0; y < Lyf; ++y) {
      s.C[frame_label(r, 0) * S + frame_site(c, r, x + 1, y)] = nC1[y];
      s.T[frame_label(r, 3) * S + frame_site(c, r, x + 1, y)] = nT4[y];
      s.C[frame_label(r, 3) * S + frame_site(c, r, x + 1, y)] = nC4[y];
    }
  }
  return CTM_OK;
}

// Two-site density matrix of the bond (x, y) -> right (dir 0) / down (dir 1)
// as the library's observable path computes it, then e = Tr(op rho) / Tr rho.
ctm_status tape_bond_energy(Tape& T, StateVals& s, int x, int y, int dir, void* op, void** e) {
  ctm_ctx* c = T.c;
  const long chi = c->chi, Dk = c->Dk, Db = c->Db, d = c->d;
  const int S = c->S;
  int r, fx, fy;
  if (dir == 0) { r = 0; fx = x; fy = y; }
  else { r = 1; fx = y; fy = ((-x) % c->Lx + c->Lx) % c->Lx; }
  auto Cv = [&](int i, int xx) { return tn(s.C[frame_label(r, i) * S + frame_site(c, r, xx, fy)], {chi, chi}); };
  auto Tv = [&](int i, int xx) {
    return tn(s.T[frame_label(r, i) * S + frame_site(c, r, xx, fy)], {chi, chi, Dk, Db});
  };
  void* K1 = s.rot[r][frame_site(c, r, fx, fy)];
  void* K2 = s.rot[r][frame_site(c, r, fx + 1, fy)];
  Tn a, b, L, R, rho;
  CK(ein_t(T, "ab,bcuU->acuU", Cv(0, fx), Tv(0, fx), {chi, chi, Dk, Db}, &a));
  CK(ein_t(T, "kalL,acuU->klLcuU", Tv(3, fx), a, {chi, Dk, Db, chi, Dk, Db}, &b));
  CK(ein_t(T, "klLcuU,sulxm->kLcUsxm", b, tn(K1, {d, Dk, Dk, Dk, Dk}), {chi, Db, chi, Db, d, Dk, Dk}, &a));
  CK(ein_t(T, "kLcUsxm,tULXM->kcsxmtXM", a, tn(K1, {d, Db, Db, Db, Db}),
           {chi, chi, d, Dk, Dk, d, Db, Db}, &b));
  CK(ein_t(T, "kcsxmtXM,jk->jcsxmtXM", b, Cv(3, fx), {chi, chi, d, Dk, Dk, d, Db, Db}, &a));
  CK(ein_t(T, "jcsxmtXM,ijxX->icsmtM", a, Tv(2, fx), {chi, chi, d, Dk, d, Db}, &L));
  CK(ein_t(T, "ceoO,ef->cfoO", Tv(0, fx + 1), Cv(1, fx + 1), {chi, chi, Dk, Db}, &a));
  CK(ein_t(T, "cfoO,fgrR->cgoOrR", a, Tv(1, fx + 1), {chi, chi, Dk, Db, Dk, Db}, &b));
  CK(ein_t(T, "cgoOrR,qomwr->cgORqmw", b, tn(K2, {d, Dk, Dk, Dk, Dk}), {chi, chi, Db, Db, d, Dk, Dk}, &a));
  CK(ein_t(T, "cgORqmw,vOMWR->cgqmwvMW", a, tn(K2, {d, Db, Db, Db, Db}),
           {chi, chi, d, Dk, Dk, d, Db, Db}, &b));
  CK(ein_t(T, "cgqmwvMW,gh->chqmwvMW", b, Cv(2, fx + 1), {chi, chi, d, Dk, Dk, d, Db, Db}, &a));
  CK(ein_t(T, "chqmwvMW,hiwW->ciqmvM", a, Tv(2, fx + 1), {chi, chi, d, Dk, d, Db}, &R));
  CK(ein_t(T, "icsmtM,ciqmvM->sqtv", L, R, {d, d, d, d}, &rho));
  return energy_t(T, rho.p, op, (int)(d * d), e);
}

// ---------------------------------------------------------------- driver
ctm_status check_supported(ctm_ctx* c) {
  if (c->cx) return fail(c, CTM_EUNSUPPORTED, "gradients are implemented for real (CTM_F64) tensors");
  if (c->split) return fail(c, CTM_EUNSUPPORTED, "gradients run in fp64 (CTM_PREC_FP64 contexts)");
  if (c->opts.method != CTM_PROJ_SI) return fail(c, CTM_EUNSUPPORTED, "gradients need SI projectors");
  if (c->opts.recycle_sin2 > 0.0)
    return fail(c, CTM_EUNSUPPORTED, "gradients need recycle_sin2 = 0 (an update every move)");
  if (!c->bra_is_conj || c->Db != c->Dk)
    return fail(c, CTM_EUNSUPPORTED, "gradients need an iPEPS context with bra = conj(A)");
  return CTM_OK;
}

// base tensors: the context's rotation-0 kets
void base_tensors(ctm_ctx* c, StateVals& s) {
  s.A.resize(c->S);
  for (int i = 0; i < c->S; ++i) s.A[i] = KETp(c, 0, i);
}

// The observable E = sum over sites and both bonds of <op>, recorded on T
// from the state values s; returns the E value pointers.
ctm_status tape_energy(Tape& T, StateVals& s, void* op, std::vector<void*>* es) {
  ctm_ctx* c = T.c;
  for (int y = 0; y < c->Ly; ++y)
    for (int x = 0; x < c->Lx; ++x)
      for (int dir = 0; dir < 2; ++dir) {
        void* e = nullptr;
        CK(tape_bond_energy(T, s, x, y, dir, op, &e));
        es->push_back(e);
      }
  return CTM_OK;
}

ctm_status seed_ones(Tape& T, const std::vector<void*>& es) {
  const double one[2] = {1.0, 0.0};
  for (void* e : es) {
    void* g = T.adj_of(e, 2);
    if (!g) return nomem(T.c);
    CTM_CUDA_OK(cudaMemcpyAsync(g, one, 8, cudaMemcpyHostToDevice, T.st()));
  }
  // the copies above read host memory that goes out of scope
  CTM_CUDA_OK(cudaStreamSynchronize(T.st()));
  return CTM_OK;
}

// Adjoint state: corners, edges, rangefinders of all directions, A.
struct AdjState {
  void* C = nullptr;   // [4 S][chi^2]
  void* T = nullptr;   // [4 S][chi^2 Dk Db]
  void* X = nullptr;   // [4][S][N k]
  void* W = nullptr;
  void* A = nullptr;   // [S][d D^4]
  size_t nC = 0, nT = 0, nX = 0, nA = 0;   // elements of one tensor
};

ctm_status alloc_adj(ctm_ctx* c, Arena& ar, AdjState* g) {
  const size_t S = c->S;
  g->nC = (size_t)c->chi * c->chi;
  g->nT = g->nC * c->Dk * c->Db;
  g->nX = (size_t)c->N * c->k;
  g->nA = elems_ket(c);
  g->C = ar.get(4 * S * g->nC * 8);
  g->T = ar.get(4 * S * g->nT * 8);
  g->X = ar.get(4 * S * g->nX * 8);
  g->W = ar.get(4 * S * g->nX * 8);
  g->A = ar.get(S * g->nA * 8);
  if (!g->C || !g->T || !g->X || !g->W || !g->A) return nomem(c);
  CTM_CUDA_OK(cudaMemsetAsync(g->C, 0, 4 * S * g->nC * 8, c->stream));
  CTM_CUDA_OK(cudaMemsetAsync(g->T, 0, 4 * S * g->nT * 8, c->stream));
  CTM_CUDA_OK(cudaMemsetAsync(g->X, 0, 4 * S * g->nX * 8, c->stream));
  CTM_CUDA_OK(cudaMemsetAsync(g->W, 0, 4 * S * g->nX * 8, c->stream));
  CTM_CUDA_OK(cudaMemsetAsync(g->A, 0, S * g->nA * 8, c->stream));
  return CTM_OK;
}

double* slot(void* base, size_t n, size_t i) { return static_cast<double*>(base) + n * i; }

// dst <- adjoint of value v (zero when v has none); add: dst += instead
ctm_status take_adj(Tape& T, void* v, size_t n, double* dst, bool add) {
  void* a = T.adj_if(v);
  if (add) {
    if (a) CK(axpy(T, (long)n, 1.0, a, dst));
    return CTM_OK;
  }
  if (a) CTM_CUDA_OK(cudaMemcpyAsync(dst, a, n * 8, cudaMemcpyDeviceToDevice, T.st()));
  else CTM_CUDA_OK(cudaMemsetAsync(dst, 0, n * 8, T.st()));
  return CTM_OK;
}

// seed the adjoint of value v with src (added)
ctm_status seed(Tape& T, void* v, size_t n, const double* src) {
  if (!v) return CTM_OK;
  void* a = T.adj_of(v, (long)n);
  if (!a) return nomem(T.c);
  return axpy(T, (long)n, 1.0, src, a);
}

}  // namespace

ctm_status grad_checkpoint(ctm_ctx* c, int r) {
  if (!c->grad || !c->grad->recording) return CTM_OK;
  Checkpoint cp;
  cp.r = r;
  const size_t nC = 4 * (size_t)c->S * elems_C(c) * 8, nT = 4 * (size_t)c->S * elems_T(c) * 8;
  const size_t nX = (size_t)c->S * c->N * c->k * 8;
  if (cudaMalloc(&cp.C, nC) != cudaSuccess || cudaMalloc(&cp.T, nT) != cudaSuccess ||
      cudaMalloc(&cp.X, nX) != cudaSuccess || cudaMalloc(&cp.W, nX) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(cp.C);
    cudaFree(cp.T);
    cudaFree(cp.X);
    cudaFree(cp.W);
    return fail(c, CTM_ENOMEM, "device memory for a recorded move");
  }
  CTM_CUDA_OK(cudaMemcpyAsync(cp.C, c->C, nC, cudaMemcpyDeviceToDevice, c->stream));
  CTM_CUDA_OK(cudaMemcpyAsync(cp.T, c->T, nT, cudaMemcpyDeviceToDevice, c->stream));
  CTM_CUDA_OK(cudaMemcpyAsync(cp.X, at(c->X, (size_t)r * c->S * c->N * c->k, c), nX,
                              cudaMemcpyDeviceToDevice, c->stream));
  CTM_CUDA_OK(cudaMemcpyAsync(cp.W, at(c->W, (size_t)r * c->S * c->N * c->k, c), nX,
                              cudaMemcpyDeviceToDevice, c->stream));
  cp.ready.assign(c->rf_ready.begin() + r * c->S, c->rf_ready.begin() + (r + 1) * c->S);
  cp.moves_done = c->moves_done[r];
  c->grad->cps.push_back(cp);
  return CTM_OK;
}

void grad_destroy(ctm_ctx* c) {
  if (!c->grad) return;
  c->grad->release();
  delete c->grad;
  c->grad = nullptr;
}

}  // namespace ctmi

using namespace ctmi;

extern "C" {

ctm_status ctm_record(ctm_ctx* c, int on) {
  if (!c) return CTM_EINVAL;
  Guard gd(c);
  if (on) CK(check_supported(c));
  if (!c->grad) c->grad = new GradState();
  CTM_CUDA_OK(cudaStreamSynchronize(c->stream));
  if (on) c->grad->release();
  c->grad->recording = on != 0;
  return CTM_OK;
}

ctm_status ctm_grad(ctm_ctx* c, const void* op, double* E_out, void* dA_out) {
  if (!c || !op || !dA_out) return fail(c, CTM_EINVAL, "NULL argument");
  Guard gd(c);
  CK(check_supported(c));
  if (!c->grad) return fail(c, CTM_EINVAL, "no recorded moves: call ctm_record(ctx, 1) first");
  use_lane(c, 0);
  const int S = c->S, d2 = c->d * c->d;
  Arena keep;
  void* dop = keep.get((size_t)d2 * d2 * 8);
  double* dw = static_cast<double*>(keep.get((2 + 2432) * 8));
  AdjState g;
  if (!dop || !dw) return nomem(c);
  CK(alloc_adj(c, keep, &g));
  CTM_CUDA_OK(cudaMemcpyAsync(dop, op, (size_t)d2 * d2 * 8, cudaMemcpyHostToDevice, c->stream));
  double E = 0.0;
  {
    // the observable at the current environment
    Tape T(c);
    T.dwork = dw;
    StateVals s;
    base_tensors(c, s);
    CK(make_rotations(T, s));
    s.C.resize(4 * S);
    s.T.resize(4 * S);
    for (int i = 0; i < 4 * S; ++i) {
      s.C[i] = at(c->C, (size_t)i * elems_C(c), c);
      s.T[i] = at(c->T, (size_t)i * elems_T(c), c);
    }
    T.constant.insert(dop);
    std::vector<void*> es;
    CK(tape_energy(T, s, dop, &es));
    std::vector<double> h(2 * es.size());
    for (size_t i = 0; i < es.size(); ++i)
      CTM_CUDA_OK(cudaMemcpyAsync(&h[2 * i], es[i], 8, cudaMemcpyDeviceToHost, c->stream));
    CK(seed_ones(T, es));
    for (size_t i = 0; i < es.size(); ++i) E += h[2 * i];
    CK(backward(T));
    for (int i = 0; i < 4 * S; ++i) {
      CK(take_adj(T, s.C[i], g.nC, slot(g.C, g.nC, i), false));
      CK(take_adj(T, s.T[i], g.nT, slot(g.T, g.nT, i), false));
    }
    for (int i = 0; i < S; ++i) CK(take_adj(T, s.A[i], g.nA, slot(g.A, g.nA, i), true));
    CK(check_err(c));
  }
  // the recorded moves, last first: recompute each from its checkpoint on a
  // tape, seed its outputs with the adjoint state, sweep back
  auto& cps = c->grad->cps;
  for (size_t m = cps.size(); m-- > 0;) {
    const Checkpoint& cp = cps[m];
    const int r = cp.r;
    Tape T(c);
    T.dwork = dw;
    StateVals s;
    base_tensors(c, s);
    CK(make_rotations(T, s));
    s.C.resize(4 * S);
    s.T.resize(4 * S);
    for (int i = 0; i < 4 * S; ++i) {
      s.C[i] = static_cast<char*>(cp.C) + (size_t)i * elems_C(c) * 8;
      s.T[i] = static_cast<char*>(cp.T) + (size_t)i * elems_T(c) * 8;
    }
    s.X[r].resize(S);
    s.W[r].resize(S);
    for (int i = 0; i < S; ++i) {
      s.X[r][i] = static_cast<char*>(cp.X) + (size_t)i * g.nX * 8;
      s.W[r][i] = static_cast<char*>(cp.W) + (size_t)i * g.nX * 8;
      // a raw initial block enters through its first QR as a constant
      if (!cp.ready[i]) {
        T.constant.insert(s.X[r][i]);
        T.constant.insert(s.W[r][i]);
      }
    }
    const std::vector<void*> inC = s.C, inT = s.T, inX = s.X[r], inW = s.W[r];
    CK(tape_move(T, s, r, cp.ready, cp.moves_done));
    for (int i = 0; i < 4 * S; ++i) {
      CK(seed(T, s.C[i], g.nC, slot(g.C, g.nC, i)));
      CK(seed(T, s.T[i], g.nT, slot(g.T, g.nT, i)));
    }
    for (int i = 0; i < S; ++i) {
      CK(seed(T, s.X[r][i], g.nX, slot(g.X, g.nX, (size_t)r * S + i)));
      CK(seed(T, s.W[r][i], g.nX, slot(g.W, g.nX, (size_t)r * S + i)));
    }
    CK(backward(T));
    for (int i = 0; i < 4 * S; ++i) {
      CK(take_adj(T, inC[i], g.nC, slot(g.C, g.nC, i), false));
      CK(take_adj(T, inT[i], g.nT, slot(g.T, g.nT, i), false));
    }
    for (int i = 0; i < S; ++i) {
      CK(take_adj(T, inX[i], g.nX, slot(g.X, g.nX, (size_t)r * S + i), false));
      CK(take_adj(T, inW[i], g.nX, slot(g.W, g.nX, (size_t)r * S + i), false));
      CK(take_adj(T, s.A[i], g.nA, slot(g.A, g.nA, i), true));
    }
    CK(check_err(c));
  }
  CTM_CUDA_OK(cudaMemcpyAsync(dA_out, g.A, (size_t)S * g.nA * 8, cudaMemcpyDeviceToHost, c->stream));
  CTM_CUDA_OK(cudaStreamSynchronize(c->stream));
  if (E_out) *E_out = E;
  return CTM_OK;
}

ctm_status ctm_grad_fixed_point(ctm_ctx* c, const void* op, double tol, int max_iter,
                                double* E_out, void* dA_out, int* iters_out, double* res_out) {
  if (!c || !op || !dA_out || max_iter < 1) return fail(c, CTM_EINVAL, "bad argument");
  Guard gd(c);
  CK(check_supported(c));
  for (int r = 0; r < 4; ++r)
    if (c->moves_done[r] < c->opts.warmup_iters)
      return fail(c, CTM_EINVAL, "converge the environment (past the warm-up moves) first");
  for (char rd : c->rf_ready)
    if (!rd) return fail(c, CTM_EINVAL, "converge the environment first");
  use_lane(c, 0);
  const int S = c->S, d2 = c->d * c->d;
  Arena keep;
  void* dop = keep.get((size_t)d2 * d2 * 8);
  double* dw = static_cast<double*>(keep.get((2 + 2432) * 8));
  double* nrm = static_cast<double*>(keep.get(16));
  AdjState g, lam, nxt;   // dg/dx, current lambda, next lambda
  if (!dop || !dw || !nrm) return nomem(c);
  CK(alloc_adj(c, keep, &g));
  CK(alloc_adj(c, keep, &lam));
  CK(alloc_adj(c, keep, &nxt));
  CTM_CUDA_OK(cudaMemcpyAsync(dop, op, (size_t)d2 * d2 * 8, cudaMemcpyHostToDevice, c->stream));
  const size_t nX = (size_t)c->N * c->k;
  double E = 0.0;
  {
    Tape T(c);
    T.dwork = dw;
    StateVals s;
    base_tensors(c, s);
    CK(make_rotations(T, s));
    s.C.resize(4 * S);
    s.T.resize(4 * S);
    for (int i = 0; i < 4 * S; ++i) {
      s.C[i] = at(c->C, (size_t)i * elems_C(c), c);
      s.T[i] = at(c->T, (size_t)i * elems_T(c), c);
    }
    T.constant.insert(dop);
    std::vector<void*> es;
    CK(tape_energy(T, s, dop, &es));
    std::vector<double> h(2 * es.size());
    for (size_t i = 0; i < es.size(); ++i)
      CTM_CUDA_OK(cudaMemcpyAsync(&h[2 * i], es[i], 8, cudaMemcpyDeviceToHost, c->stream));
    CK(seed_ones(T, es));
    for (size_t i = 0; i < es.size(); ++i) E += h[2 * i];
    CK(backward(T));
    for (int i = 0; i < 4 * S; ++i) {
      CK(take_adj(T, s.C[i], g.nC, slot(g.C, g.nC, i), false));
      CK(take_adj(T, s.T[i], g.nT, slot(g.T, g.nT, i), false));
    }
    for (int i = 0; i < S; ++i) CK(take_adj(T, s.A[i], g.nA, slot(g.A, g.nA, i), true));
  }
  // one CTMRG iteration (four moves) at the fixed point, recorded once
  Tape T(c);
  T.dwork = dw;
  StateVals s;
  base_tensors(c, s);
  CK(make_rotations(T, s));
  s.C.resize(4 * S);
  s.T.resize(4 * S);
  for (int i = 0; i < 4 * S; ++i) {
    s.C[i] = at(c->C, (size_t)i * elems_C(c), c);
    s.T[i] = at(c->T, (size_t)i * elems_T(c), c);
  }
  for (int r = 0; r < 4; ++r) {
    s.X[r].resize(S);
    s.W[r].resize(S);
    for (int i = 0; i < S; ++i) {
      s.X[r][i] = at(c->X, ((size_t)r * S + i) * nX, c);
      s.W[r][i] = at(c->W, ((size_t)r * S + i) * nX, c);
    }
  }
  const StateVals in = s;
  std::vector<char> ready(S, 1);
  for (int r = 0; r < 4; ++r) CK(tape_move(T, s, r, ready, c->moves_done[r]));
  const size_t totC = 4 * (size_t)S * g.nC, totT = 4 * (size_t)S * g.nT, totX = 4 * (size_t)S * nX;
  // lambda_0 = dg/dx
  CTM_CUDA_OK(cudaMemcpyAsync(lam.C, g.C, totC * 8, cudaMemcpyDeviceToDevice, c->stream));
  CTM_CUDA_OK(cudaMemcpyAsync(lam.T, g.T, totT * 8, cudaMemcpyDeviceToDevice, c->stream));
  // vector-Jacobian product of one iteration: out = (dF/dx)^T lam, A part
  // added to out.A (which starts at zero)
  auto vjp = [&](AdjState& l, AdjState& out) -> ctm_status {
    T.reset_adjoints();
    for (int i = 0; i < 4 * S; ++i) {
      CK(seed(T, s.C[i], g.nC, slot(l.C, g.nC, i)));
      CK(seed(T, s.T[i], g.nT, slot(l.T, g.nT, i)));
    }
    for (int r = 0; r < 4; ++r)
      for (int i = 0; i < S; ++i) {
        CK(seed(T, s.X[r][i], nX, slot(l.X, nX, (size_t)r * S + i)));
        CK(seed(T, s.W[r][i], nX, slot(l.W, nX, (size_t)r * S + i)));
      }
    CK(backward(T));
    for (int i = 0; i < 4 * S; ++i) {
      CK(take_adj(T, in.C[i], g.nC, slot(out.C, g.nC, i), false));
      CK(take_adj(T, in.T[i], g.nT, slot(out.T, g.nT, i), false));
    }
    for (int r = 0; r < 4; ++r)
      for (int i = 0; i < S; ++i) {
        CK(take_adj(T, in.X[r][i], nX, slot(out.X, nX, (size_t)r * S + i), false));
        CK(take_adj(T, in.W[r][i], nX, slot(out.W, nX, (size_t)r * S + i), false));
      }
    CTM_CUDA_OK(cudaMemsetAsync(out.A, 0, (size_t)S * g.nA * 8, c->stream));
    for (int i = 0; i < S; ++i) CK(take_adj(T, s.A[i], g.nA, slot(out.A, g.nA, i), true));
    return CTM_OK;
  };
  int it = 0;
  double res = INFINITY;
  while (it < max_iter) {
    // lambda <- dg/dx + (dF/dx)^T lambda
    CK(vjp(lam, nxt));
    CK(axpy(T, (long)totC, 1.0, g.C, nxt.C));
    CK(axpy(T, (long)totT, 1.0, g.T, nxt.T));
    ++it;
    CTM_CUDA_OK(cudaMemsetAsync(nrm, 0, 16, c->stream));
    diff_norm_kernel<<<blocks_for(totC), 256, 0, c->stream>>>(totC, (const double*)nxt.C, (const double*)lam.C, nrm);
    diff_norm_kernel<<<blocks_for(totT), 256, 0, c->stream>>>(totT, (const double*)nxt.T, (const double*)lam.T, nrm);
    diff_norm_kernel<<<blocks_for(totX), 256, 0, c->stream>>>(totX, (const double*)nxt.X, (const double*)lam.X, nrm);
    diff_norm_kernel<<<blocks_for(totX), 256, 0, c->stream>>>(totX, (const double*)nxt.W, (const double*)lam.W, nrm);
    c->launches += 4;
    CTM_CUDA_OK(cudaGetLastError());
    double h[2] = {0, 0};
    CTM_CUDA_OK(cudaMemcpyAsync(h, nrm, 16, cudaMemcpyDeviceToHost, c->stream));
    CK(check_err(c));
    res = std::sqrt(h[0] / std::max(h[1], 1e-300));
    std::swap(lam, nxt);
    if (res < tol) break;
  }
  // dA = dg/dA + (dF/dA)^T lambda
  CK(vjp(lam, nxt));
  CK(axpy(T, (long)S * g.nA, 1.0, g.A, nxt.A));
  CTM_CUDA_OK(cudaMemcpyAsync(dA_out, nxt.A, (size_t)S * g.nA * 8, cudaMemcpyDeviceToHost, c->stream));
  CTM_CUDA_OK(cudaStreamSynchronize(c->stream));
  CK(check_err(c));
  if (E_out) *E_out = E;
  if (iters_out) *iters_out = it;
  if (res_out) *res_out = res;
  if (!(res < tol)) {
    c->msg = "max_iter reached before the fixed-point adjoint converged";
    return CTM_ENOCONV;
  }
  return CTM_OK;
}

}  // extern "C"
