/*
 * ctm.h -- C ABI of the GB300 (sm_103a) SI-CTMRG library (libctm.so).
 *
 * Contracts an infinite square-lattice tensor network (the norm of an iPEPS,
 * or a classical network such as the 2D Ising model) with the corner transfer
 * matrix renormalisation group, building the truncation projectors either by
 * subspace iteration (SI-CTMRG: "QR-based projector", steps 1-4 of Zhang &
 * Corboz, arXiv 2607.15158) or, for comparison, by the standard truncated SVD
 * of the effective environment M (paper section "Standard CTMRG").
 *
 * Conventions
 *   - Unit cell of Lx x Ly sites; site index i = y * Lx + x.
 *   - On-site ket tensor A[s][u][l][d][r] (physical, up, left, down, right),
 *     row-major; bra tensor B of the same shape with bond Db. For an iPEPS
 *     B = conj(A) (pass bra = NULL); for a classical network a[u][l][d][r]
 *     use ctm_init_network (d = 1, Db = 1, B = 1).
 *   - Corners C_i[prev][next] (chi x chi) and edges T_i[prev][next][ket][bra]
 *     (chi x chi x Dk x Db), legs ordered along the clockwise ring
 *     C1 T1 C2 T2 C3 T3 C4 T4 (C1 upper-left, T1 up, C2 upper-right, T2 right,
 *     C3 lower-right, T3 down, C4 lower-left, T4 left). Host arrays of all
 *     corners are laid out [label 0..3][site][chi][chi], edges
 *     [label][site][chi][chi][Dk][Db].
 *   - Rangefinders X (columns in M's column space) and W = Y^dagger (M's row
 *     space), N x k each with N = chi*Dk*Db, k = min(chi + p, N), laid out
 *     [direction 0..3][cut][N][k]; cut = upper-left site of the 2x2 block in
 *     the frame of that direction.
 *   - Real data is double; complex data is interleaved (re, im) double pairs.
 *
 * Ownership and errors
 *   - Every input is copied; the caller keeps its buffers. Outputs are written
 *     to caller buffers (host memory unless stated).
 *   - Calls are synchronous on the context's stream and never abort. Argument
 *     errors are reported before any device work. A failed call returns a
 *     status and leaves a message readable with ctm_last_error().
 *   - Device-side iterations (Jacobi sweeps, Cholesky) are bounded; running
 *     out of sweeps returns CTM_ENOCONV, a non-positive pivot CTM_ENUMERIC.
 */
#ifndef CTM_H
#define CTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ctm_ctx ctm_ctx;

typedef enum {
  CTM_OK = 0,
  CTM_EINVAL = 1,       /* bad argument or call order */
  CTM_ENOMEM = 2,       /* device allocation failed */
  CTM_ECUDA = 3,        /* CUDA runtime or launch error */
  CTM_ENOCONV = 4,      /* iteration budget exhausted (not fatal) */
  CTM_ETIMEOUT = 5,     /* device wait budget exhausted */
  CTM_ENUMERIC = 6,     /* breakdown: non-positive Cholesky pivot, NaN */
  CTM_EUNSUPPORTED = 7  /* configuration not supported by this build */
} ctm_status;

typedef enum { CTM_F64 = 0, CTM_C128 = 1 } ctm_dtype;

/* Arithmetic of the large contractions. FP64: every product in double.
 * SPLIT_BF16: corner x block products and the large GEMMs of the enlarged
 * corners and the absorption as sums of bf16 slice products on the tensor
 * cores (three bf16 slices of each operand's fp32 rounding, six products)
 * with fp32 accumulation and fp64 reduction, the fused A / conj(A)
 * absorption in fp32. SPLIT_TF32: the same with 3xTF32 (two tf32 slices,
 * three products, the tensor cores' tf32 kind at half the bf16 rate). QR,
 * small SVD, rho, the projectors and s^-1/2 stay fp64-accurate in both (their
 * products as exact fixed-point digit products on the tensor cores with
 * opts.fp64_tc, see ctm_gemm_fp64tc). */
typedef enum { CTM_PREC_FP64 = 0, CTM_PREC_SPLIT_BF16 = 1, CTM_PREC_SPLIT_TF32 = 2 } ctm_prec;

typedef enum { CTM_LEFT = 0, CTM_UP = 1, CTM_RIGHT = 2, CTM_DOWN = 3 } ctm_dir;

/* Projector construction: subspace iteration (QR-based projector, paper
 * Eqs. xy_iter to xy_recycle) or the standard truncated SVD of the explicit
 * M = H_L H_R (Eq. svd_projectors_diag; comparison baseline). The standard
 * method's dense N x N SVD is cuSOLVER's gesvd, opened on first use:
 * ctm_init returns CTM_EUNSUPPORTED when libcusolver cannot be loaded. */
typedef enum { CTM_PROJ_SI = 0, CTM_PROJ_SVD = 1 } ctm_method;

typedef struct {
  int p;                  /* oversampling, k = chi + p (paper: p = 5) */
  int si_rounds;          /* subspace-iteration rounds per projector */
  int warmup_iters;       /* first moves per direction that use ... */
  int warmup_rounds;      /* ... this many rounds (warm-up, paper step 4) */
  ctm_method method;      /* CTM_PROJ_SI or CTM_PROJ_SVD */
  ctm_prec prec;          /* arithmetic of the large contractions */
  double svd_rel_cutoff;  /* s^-1/2 := 0 for s_i <= cutoff * s_1 */
  int normalize;          /* new C, T: unit Frobenius norm, largest entry
                             real positive */
  int sign_fix;           /* phase fix of the small SVD of rho */
  uint64_t seed;          /* seed of the default random C, T, X, W */
  int svd_max_sweeps;     /* sweep budget of the Jacobi SVDs (small problem,
                             corner spectra); running out is CTM_ENOCONV */
  int init_mode;          /* initial C, T: 0 = seeded random normal,
                             1 = from the on-site tensors (CTM_INIT_FROM_A) */
  double recycle_sin2;    /* recycling policy of paper step 4: once the mean
                             sin^2 of the principal angles between successive
                             leading chi-subspaces of a cut falls below this
                             value (paper: 1e-3) after at least min_si_steps
                             updates, the cut's rangefinders are only
                             recycled, with no subspace-iteration round, until
                             the angle grows above it again; 0 = always update */
  int min_si_steps;       /* see recycle_sin2 (paper: at least 3) */
  int absorb_tc;          /* split contexts: 1 = the A / conj(A) absorption as
                             split bf16 tensor-core GEMMs with permutes (the
                             accuracy of the other products), 0 = one fused
                             kernel in fp32 arithmetic */
  int si_coupled;         /* 1 = coupled (Halko) rangefinder update: each round
                             W <- qr(M X), X <- qr(M^H W) (half the corner
                             products of the paper's independent updates of
                             Eq. xy_iter); 0 = the paper's form */
  int warmup_rsvd;        /* 1 = every warm-up move restarts its rounds from
                             the initial random blocks (a randomized SVD per
                             move, End Matter: RSVD before SI on larger unit
                             cells) instead of the recycled bases */
  int fp64_tc;           /* split contexts: 1 = the products that stay fp64
                             (CholeskyQR Grams, rho, the projectors
                             Z v s^-1/2) run as exact fixed-point digit
                             products on the tensor cores (ctm_gemm_fp64tc),
                             0 = fp64 GEMMs on the CUDA cores */
  int svd_presolve;       /* 1 = the small SVDs of rho (k <= 169 complex, 238
                             real) first run the one-sided Jacobi in fp32,
                             then the fp64 sweeps on rho V0 from V0 made
                             unitary in fp64 (same result to fp64 rounding,
                             fewer fp64 sweeps); 0 = fp64 sweeps only */
  double split_refine;    /* split contexts: once the corner-spectrum change of
                             ctm_converge falls below this value, the rest of
                             that call runs every large product (corners,
                             subspace products, QR, absorption) as an
                             exact-digit fp64-accurate tensor-core product and
                             the absorption without the fp32 fused kernel:
                             mixed-precision refinement of the fixed point to
                             fp64 accuracy. The observables of such a context
                             (ctm_expect*, ctm_rdm2, ctm_free_energy,
                             ctm_transfer_spectrum) use the same products.
                             +inf: every move (ctm_move, ctm_converge) runs
                             them from the start, an fp64-accurate mode on
                             the tensor cores. 0 = off */
  void* stream;           /* cudaStream_t to run on, NULL = a private stream */
} ctm_opts;

/* init_mode values. CTM_INIT_FROM_A: every corner is the double-layer tensor
 * of its site with the two outer bond pairs traced (C1 = sum over s, u, l of
 * A[s,u,l,d,r] conj(A)[s,u,l,d',r'] as a (d d') x (r r') matrix, the other
 * corners the same form of the turned tensor), every edge the double layer
 * with its outer pair traced, and both are embedded in the top-left block of
 * the chi x chi bonds (zero elsewhere) or cut to it when D^2 > chi; then
 * normalised. */
enum { CTM_INIT_RANDOM = 0, CTM_INIT_FROM_A = 1 };

/* Defaults: p = 5, si_rounds = 1, warmup_iters = 5, warmup_rounds = 8, SI,
 * FP64, cutoff 1e-12, normalize = 1, sign_fix = 1, seed = 0,
 * svd_max_sweeps = 80, init_mode = CTM_INIT_RANDOM, recycle_sin2 = 0 (always
 * update), min_si_steps = 3, absorb_tc = 0, si_coupled = 0, warmup_rsvd = 0,
 * fp64_tc = 1, svd_presolve = 1, split_refine = 0, stream = NULL. */
void ctm_default_opts(ctm_opts* opts);

/* Create a context for an iPEPS unit cell (paper: "iPEPS", Eq. ipeps_ansatz
 * and the double layer of Eq. double_layer; End Matter for Lx x Ly cells).
 * A: Lx*Ly host pointers to A[d][D][D][D][D] (dtype elements). bra: NULL for
 * conj(A), else Lx*Ly host pointers to B of the same shape. The environment
 * and rangefinders start from seeded random normal draws (replace them with
 * ctm_set_env / ctm_set_rangefinders). Returns CTM_EINVAL for Lx, Ly, d, D,
 * chi < 1, CTM_ENOMEM when the state does not fit on the device. */
ctm_status ctm_init(ctm_ctx** out, int Lx, int Ly, const void* const* A,
                    const void* const* bra, ctm_dtype dtype, int d, int D,
                    int chi, const ctm_opts* opts);

/* Create a context for a classical network: a[u][l][d][r] real, bond k, one
 * tensor per site (Lx*Ly host pointers). Edges have shape chi x chi x k x 1. */
ctm_status ctm_init_network(ctm_ctx** out, int Lx, int Ly,
                            const double* const* a, int k, int chi,
                            const ctm_opts* opts);

/* Replace the environment: C [4][Lx*Ly][chi][chi], T [4][Lx*Ly][chi][chi][Dk][Db]
 * (host, dtype of the context). */
ctm_status ctm_set_env(ctm_ctx* ctx, const void* C, const void* T);

/* Copy the environment out (same layouts as ctm_set_env). */
ctm_status ctm_get_env(ctm_ctx* ctx, void* C, void* T);

/* Replace the raw rangefinder blocks X, W ([4][Lx*Ly][N][k], host); they are
 * orthonormalised on their first use (QR of a Gaussian block, step 1). */
ctm_status ctm_set_rangefinders(ctm_ctx* ctx, const void* X, const void* W);

/* Query N = chi*Dk*Db and k = min(chi + p, N). */
ctm_status ctm_dims(const ctm_ctx* ctx, int* N, int* k);

/* One directional move over the whole cell (End Matter, left move; up /
 * right / down are the left move of the cell turned by 1 / 2 / 3
 * counter-clockwise quarter turns): column by column, the projectors of all
 * cuts of a column are built, then C1, T4, C4 of the next column are
 * absorbed, truncated and normalised. */
ctm_status ctm_move(ctm_ctx* ctx, ctm_dir dir);

/* Iterations of the four moves (left, up, right, down) until the
 * corner-spectrum change Delta < tol or max_iter; Delta = max over corners
 * and sites of ||s_new - s_old||_2 of unit-normalised spectra. The paper
 * iterates CTMRG steps until the environment converges (section "CTMRG" and
 * step 4 of the QR-based projector: with the sign fix, C and T converge
 * element-wise); the corner-spectrum change is the gauge-invariant form of
 * that criterion. Returns CTM_ENOCONV (not fatal) when max_iter is reached.
 * iters_out, delta_out may be NULL. */
ctm_status ctm_converge(ctm_ctx* ctx, double tol, int max_iter,
                        int* iters_out, double* delta_out);

/* Normalised singular values (descending, unit 2-norm) of corner C_label
 * (label 1..4) at site (x, y); s_out has chi entries (host). The corner
 * spectrum is the quantity whose change measures convergence (see
 * ctm_converge); the paper's corners are the C_i of Fig. ctmrg-step. */
ctm_status ctm_spectrum(ctm_ctx* ctx, int x, int y, int label, double* s_out);

/* The same for all corners in one batched call: s_out has 4*Lx*Ly*chi
 * entries, laid out [label 0..3][site][chi] (the convergence measure of
 * ctm_converge compares these). Right after ctm_converge, with no move,
 * ctm_set_env or ctm_load in between, it returns the spectra that the last
 * convergence measure computed instead of computing them again. */
ctm_status ctm_spectra(ctm_ctx* ctx, double* s_out);

/* Two-site expectation <O> = Tr(O rho) / Tr(rho) on the bond from (x, y) to
 * its right (dir = 0) or lower (dir = 1) neighbour; op is d^2 x d^2,
 * row-major O[(s1', s2')][(s1, s2)] (row = bra), dtype of the context; site 1
 * is (x, y). out = (re, im). This is the observable g(A, C*, T*) of the
 * paper's optimisation section, evaluated on the converged environment
 * (for the Heisenberg model, the bond energy <S.S>). */
ctm_status ctm_expect(ctm_ctx* ctx, const void* op, int x, int y, int dir,
                      double out[2]);

/* Two-site reduced density matrix rho[(s1 s2)][(t1 t2)] (ket, bra), trace 1,
 * complex (re, im) pairs, d^4 entries. */
ctm_status ctm_rdm2(ctm_ctx* ctx, int x, int y, int dir, double* rho_out);

/* Ratio Z(ket at (x,y) replaced by imp) / Z on the one-site patch; imp has the
 * ket's shape and dtype. For a classical network with an impurity tensor this
 * is the local observable (e.g. the Ising magnetisation). */
ctm_status ctm_expect_site(ctm_ctx* ctx, const void* imp, int x, int y,
                           double out[2]);

/* Ratio Z(kets at both ends of the bond replaced) / Z on the two-site patch
 * (e.g. a nearest-neighbour spin correlation of a classical network). */
ctm_status ctm_expect_bond(ctm_ctx* ctx, const void* imp1, const void* imp2,
                           int x, int y, int dir, double out[2]);

/* ln kappa per site of a 1x1 cell, kappa = Z1 Z0 / (Z13 Z24): one-site patch,
 * four corners, corners with T1-T3 joined, corners with T2-T4 joined
 * (-beta f for a classical partition function). CTM_EINVAL for larger cells. */
ctm_status ctm_free_energy(ctm_ctx* ctx, double* ln_kappa);

/* The projectors of the last move in direction dir for cut (x, y) of that
 * direction's frame: P_l (N x chi) and P_r^dagger (N x chi), host, dtype of
 * the context. */
ctm_status ctm_get_projectors(ctm_ctx* ctx, ctm_dir dir, int x, int y,
                              void* Pl, void* PrH);

/* The enlarged corner Q_i (i = 1..4: upper-left, upper-right, lower-right,
 * lower-left) of the 2x2 block whose upper-left position is (x, y) in the
 * frame of direction dir, as an N x N matrix (row-major, N = chi*Dk*Db,
 * rows: the corner's incoming ring bond and the ket/bra legs, columns: its
 * outgoing ones), built by the context's own path and precision from the
 * current environment (Eq. rho_M_diag, Fig. ctmrg-step). Q_out: host, N*N
 * elements of the context's dtype. */
ctm_status ctm_corner(ctm_ctx* ctx, ctm_dir dir, int x, int y, int i, void* Q_out);

/* Z_out = op(Q_i) Z_in for that corner and a host block Z_in of N x k
 * (row-major, k = ctm_dims' k), op = identity (herm = 0) or the conjugate
 * transpose (herm = 1): the corner x block product of the rangefinder
 * update (Eq. xy_iter), run by the context's own kernels and precision. */
ctm_status ctm_corner_apply(ctm_ctx* ctx, ctm_dir dir, int x, int y, int i, int herm,
                            const void* Z_in, void* Z_out);

/* Correlation length from the converged environment (the paper reports xi
 * with its states and extrapolates in it; here without the extrapolation):
 * the leading eigenvalues of the transfer matrix of the boundary formed by
 * the edges above and below one row, E[(a,d),(b,c)] = sum over u, u' of
 * T1[a][b][u][u'] T3[c][d][u][u'], multiplied over the Lx sites of the row
 * period (dir = 0, row = y) or, for dir = 1, over the Ly sites of column
 * x = row (the edges T2, T4 beside it). nvals (2 .. 24) eigenvalues of
 * largest modulus, sorted by descending modulus and divided by the modulus
 * of the first, into lam_out (host, nvals (re, im) pairs); xi_out = -L /
 * ln|lam_2 / lam_1| in lattice spacings (0 for a rank-one transfer
 * matrix). Subspace iteration on the device with Rayleigh-Ritz; CTM_ENOCONV
 * when the leading moduli do not settle (to 1e-13) within 2000
 * applications. At finite chi this boundary estimate lies below the exact
 * correlation length (the paper extrapolates it in chi). */
ctm_status ctm_transfer_spectrum(ctm_ctx* ctx, int dir, int row, int nvals, double* lam_out,
                                 double* xi_out);

/* Subspace-iteration updates made and skipped (recycling policy of
 * opts.recycle_sin2) over all cuts since the context was created. */
ctm_status ctm_si_stats(const ctm_ctx* ctx, long* updates, long* skipped);

/* C = op(A) B (M x N, inner K) to fp64 accuracy on the bf16 tensor cores,
 * as split contexts run their fp64 products (opts.fp64_tc): every row of
 * op(A) and column of B is written as a 56-bit fixed-point number against
 * the exponent of its largest entry and cut into eight 7-bit digits (an
 * error-free splitting after Ozaki et al.); the digit products of weight
 * <= 7 are exact in the fp32 tensor-memory accumulators and are combined as
 * unevaluated fp32 pairs. The error is about 2^-48 of |op(A)| |B|
 * (elementwise products of the row and column maxima), the order of an fp64
 * product. Host buffers, row-major: A is M x K (opA = 0) or K x M (opA = 1
 * transpose, 2 conjugate transpose), B is K x N, C is M x N; leading
 * dimensions lda, ldb, ldc; dtype CTM_F64 or CTM_C128. Verification entry
 * point of the library's product (allocates, synchronises). */
ctm_status ctm_gemm_fp64tc(ctm_dtype dtype, int opA, const void* A, long lda, const void* B,
                           long ldb, int M, int N, int K, void* C, long ldc);

/* ------------------------------------------------------- differentiation
 * Gradient of the energy E = sum over all sites and both bond directions of
 * Re <op> (op as in ctm_expect) with respect to the on-site tensors A,
 * following the paper's section "Variational optimization" (reverse-mode
 * differentiation of the recorded forward CTMRG, "unrolled") and section
 * "Differentiable fixed point" (Eq. implicit). The adjoints are hand-written
 * (contractions, CholeskyQR as the QR with positive diagonal, the small SVD
 * with Lorentzian-broadened 1/(s_j^2 - s_i^2) = 1/((s_j - s_i)(s_j + s_i)),
 * the factor 1/(s_j - s_i) replaced by (s_j - s_i) / ((s_j - s_i)^2 + eps),
 * eps = (1e-12 s_1)^2, the
 * s^-1/2 scaling, the normalisation) and run on the device in fp64; each
 * move is recomputed from a checkpoint (its enlarged corners and
 * half-system products are not stored). Supported for real (CTM_F64)
 * iPEPS contexts (bra = conj(A)) with CTM_PREC_FP64, SI projectors and
 * recycle_sin2 = 0; other contexts return CTM_EUNSUPPORTED. dA_out is host
 * memory of Lx*Ly*d*D^4 doubles laid out like ctm_init's A. */

/* on = 1: forget earlier records and start recording: every following move
 * (ctm_move, ctm_converge) first saves its input state (C, T and the
 * rangefinders of its direction, device memory of about
 * 4 S chi^2 (1 + D^2) + 2 S N k doubles per move). on = 0 stops recording
 * and keeps the records. */
ctm_status ctm_record(ctm_ctx* ctx, int on);

/* Unrolled gradient: E of the current environment and dE/dA through every
 * move recorded since ctm_record(ctx, 1); the environment and rangefinders
 * at the start of the recording are held constant (the initial raw
 * rangefinder blocks enter only through their first QR). The records are
 * kept, so the call can be repeated. E_out may be NULL. */
ctm_status ctm_grad(ctm_ctx* ctx, const void* op, double* E_out, void* dA_out);

/* Fixed-point gradient (Eq. implicit) at the current, converged
 * environment: x = (C, T and the recycled rangefinders X, Y of every
 * direction and cut) is taken as the fixed point of one CTMRG iteration F
 * (four moves); lambda = dE/dx + (dF/dx)^T lambda is iterated from
 * lambda = dE/dx until ||lambda_new - lambda|| < tol ||lambda_new|| or
 * max_iter vector-Jacobian products, then dA = dE/dA + (dF/dA)^T lambda.
 * Memory: one iteration's tape, independent of the number of forward
 * iterations. Returns CTM_ENOCONV (dA_out still written) when max_iter is
 * reached; iters_out, res_out (last relative change) and E_out may be NULL.
 * Needs the warm-up moves of every direction done. */
ctm_status ctm_grad_fixed_point(ctm_ctx* ctx, const void* op, double tol, int max_iter,
                                double* E_out, void* dA_out, int* iters_out, double* res_out);

/* Device milliseconds of the last ctm_move / ctm_converge call and the
 * number of kernels it launched. */
ctm_status ctm_last_timing(const ctm_ctx* ctx, double* ms, long* launches);

/* Per-launch timing of the split-precision tensor-core GEMM kernel (the
 * dominant kernel of CTM_PREC_SPLIT_BF16): ctm_profile_enable(ctx, 1) starts
 * recording CUDA events around each launch on the context's stream and clears
 * the totals; ctm_profile_read returns the summed device time, the launch
 * count, the tensor-pipe flops (six bf16 slice products of the real-embedded,
 * unpadded problem) and the bf16 operand bytes the launches consumed.
 * Kernel statistics are CTM_EUNSUPPORTED for an FP64 context; phase timing
 * (ctm_profile_phases) works for both. */
ctm_status ctm_profile_enable(ctm_ctx* ctx, int on);
ctm_status ctm_profile_read(ctm_ctx* ctx, double* ms, long* launches, double* flops,
                            double* bytes);

/* Device milliseconds spent since ctm_profile_enable in each phase of the
 * move, in this order: enlarged corners, bf16 slicing of the corners,
 * corner x block products, QR, small problem (rho, small SVD, recycling,
 * projectors), absorption, normalisation, corner spectra. */
#define CTM_NPHASES 8
ctm_status ctm_profile_phases(ctm_ctx* ctx, double ms[CTM_NPHASES]);

/* Device bytes a context of these dimensions and options allocates (an
 * upper estimate: the context's arrays, split-precision slice caches and
 * partial sums, dense-SVD buffers, plus 5 % and 64 MB). */
ctm_status ctm_footprint(int Lx, int Ly, int d, int D, int chi, ctm_dtype dtype,
                         const ctm_opts* opts, size_t* bytes);

/* ---------------------------------------------------------------- serving
 * Environment solves of mixed (cell, D, chi) as they arrive (continuous
 * batching). A scheduler admits pending solves first-fit in arrival order
 * while the summed ctm_footprint of the running solves stays within the HBM
 * budget and fewer than max_concurrent run; each admitted solve runs
 * ctm_init + ctm_converge on its own host thread and CUDA stream, with its
 * C, T, X, W resident until it finishes, so concurrent solves overlap on the
 * device. The paper has no serving layer: this serves many independent
 * contractions (for instance the candidate tensors of an optimisation). */
typedef struct ctm_server ctm_server;

typedef struct {
  int Lx, Ly, d, D, chi;
  ctm_dtype dtype;
  const void* const* A;   /* Lx*Ly host pointers to A[d][D][D][D][D], copied */
  const void* op;         /* d^2 x d^2 two-site operator (copied), or NULL */
  double tol;             /* ctm_converge tolerance */
  int max_iter;
  ctm_opts opts;          /* stream is ignored: every solve has its own */
} ctm_solve_spec;

typedef struct {
  ctm_status status;      /* of the solve (CTM_OK also when max_iter ran out) */
  int iters;
  double delta;           /* last convergence measure */
  double queue_ms;        /* submit -> admission */
  double run_ms;          /* admission -> done */
  size_t footprint;       /* device bytes reserved for the solve */
} ctm_solve_result;

/* hbm_budget = 0: 90 % of the free device memory at creation. */
ctm_status ctm_server_create(ctm_server** out, size_t hbm_budget, int max_concurrent);
/* Queues a solve; CTM_ENOMEM when it can never fit the budget. */
ctm_status ctm_server_submit(ctm_server* srv, const ctm_solve_spec* spec, uint64_t* ticket);
/* Blocks until the solve is done, fills res and, when not NULL, spectra
 * ([4][Lx*Ly][chi] unit-normalised corner spectra) and energies
 * ([Lx*Ly][2 directions][re, im] of op); releases the ticket. Returns the
 * solve's status. */
ctm_status ctm_server_result(ctm_server* srv, uint64_t ticket, ctm_solve_result* res,
                             double* spectra, double* energies);
/* Latency percentiles (submit -> done, nearest rank) and throughput of the
 * solves finished so far. */
ctm_status ctm_server_stats(ctm_server* srv, double* p50_ms, double* p99_ms,
                            double* solves_per_s, int* completed);
const char* ctm_server_last_error(const ctm_server* srv);
/* Waits for the running solves, drops the pending ones, frees the server. */
void ctm_server_free(ctm_server* srv);

/* Checkpoint and resume (host buffers). ctm_save with buf = NULL stores the
 * needed size in *nbytes; otherwise it writes the iteration state (C, T, the
 * rangefinders X, W of every direction and cut, the last corner spectra and
 * the move counters) into buf, *nbytes being its capacity on entry and the
 * bytes written on return (CTM_EINVAL if too small). ctm_load restores such a
 * state into a context of the same dimensions (CTM_EINVAL otherwise); the
 * iteration then continues exactly as in the saved context. */
ctm_status ctm_save(const ctm_ctx* ctx, void* buf, size_t* nbytes);
ctm_status ctm_load(ctm_ctx* ctx, const void* buf, size_t nbytes);

void ctm_free(ctm_ctx* ctx);

/* Message of the last failed call on ctx (or of the last failed creation when
 * ctx is NULL); owned by the library, valid until the next call. */
const char* ctm_last_error(const ctm_ctx* ctx);

/* Fault injection for tests of the error paths (the paper has no
 * counterpart): after this call the library's device allocations succeed
 * `after` more times, then the next one fails on the host, before
 * cudaMalloc is called, as if the device were out of memory (CTM_ENOMEM);
 * the hook then disarms itself. after < 0 disarms it. Process-wide. */
void ctm_debug_fail_alloc(int after);

/* Singular values of one k x k matrix, with no device allocation.
 *
 * The paper has no counterpart to this call: it is a library service for
 * callers that cannot let a library allocate device memory (an application
 * that owns all device memory through its own allocator, or a loop in which a
 * cudaMalloc / cudaFree would stall on a device-wide synchronisation). It runs
 * the same one-sided Jacobi kernel as ctm_spectrum, but keeps all of its
 * scratch in one fixed array of 2 MiB + 8 KiB reserved in device memory for
 * every GPU that loads the library, for the life of the process.
 *
 *   A       device pointer, the matrix in column-major order, k*k elements of
 *           double (CTM_F64) or interleaved (re, im) double pairs (CTM_C128);
 *           read only, owned by the caller.
 *   k       1 <= k <= 256 for CTM_C128, k <= 362 for CTM_F64; larger k is
 *           rejected with CTM_EINVAL before any device work.
 *   s       device pointer to k doubles, owned by the caller: the singular
 *           values, not normalised, in descending order.
 *   stream  the cudaStream_t to run on (NULL: the legacy default stream).
 *
 * The first call on a device looks up the device address of the scratch array
 * with that device current; make it before any stream capture. The address is
 * kept for the life of the process: after cudaDeviceReset (or any teardown of
 * the device's primary context) the array lives at a new address, so do not
 * call this entry point again in that process. The call
 * clears the words that must start at zero (error word, grid-barrier
 * counters) on the stream itself, then waits for the stream to read the error
 * word back, so it returns only once s is written. Calls that overlap on one
 * device (from several threads or streams) share the scratch and race:
 * serialise them. Returns CTM_OK, CTM_EINVAL, CTM_ECUDA, CTM_ENUMERIC,
 * CTM_ENOCONV or CTM_ETIMEOUT; the message is read with
 * ctm_noalloc_last_error() (per host thread). */
ctm_status ctm_svdvals_noalloc(const void* A, int k, ctm_dtype dtype, double* s, void* stream);
const char* ctm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CTM_H */
