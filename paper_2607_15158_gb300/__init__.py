"""Python binding of libctm, the GB300 SI-CTMRG library (C ABI in include/ctm.h).

Argument marshalling only: every function forwards to the C entry point of the
same name; all contraction work runs in the library's CUDA kernels. Inputs are
numpy arrays (or anything ``np.ascontiguousarray`` accepts) in host memory; the
library copies them. Loading fails loudly when the library has not been built
(``python -m paper_2607_15158_gb300.build``): there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libctm.so")

CTM_OK, CTM_EINVAL, CTM_ENOMEM, CTM_ECUDA, CTM_ENOCONV, CTM_ETIMEOUT, \
    CTM_ENUMERIC, CTM_EUNSUPPORTED = range(8)
STATUS_NAMES = ["CTM_OK", "CTM_EINVAL", "CTM_ENOMEM", "CTM_ECUDA", "CTM_ENOCONV",
                "CTM_ETIMEOUT", "CTM_ENUMERIC", "CTM_EUNSUPPORTED"]
CTM_F64, CTM_C128 = 0, 1
CTM_PREC_FP64, CTM_PREC_SPLIT_BF16, CTM_PREC_SPLIT_TF32 = 0, 1, 2
CTM_LEFT, CTM_UP, CTM_RIGHT, CTM_DOWN = 0, 1, 2, 3
CTM_PROJ_SI, CTM_PROJ_SVD = 0, 1
CTM_INIT_RANDOM, CTM_INIT_FROM_A = 0, 1


class ctm_opts(C.Structure):
    _fields_ = [("p", C.c_int), ("si_rounds", C.c_int), ("warmup_iters", C.c_int),
                ("warmup_rounds", C.c_int), ("method", C.c_int),
                ("prec", C.c_int), ("svd_rel_cutoff", C.c_double),
                ("normalize", C.c_int), ("sign_fix", C.c_int),
                ("seed", C.c_uint64), ("svd_max_sweeps", C.c_int), ("init_mode", C.c_int),
                ("recycle_sin2", C.c_double), ("min_si_steps", C.c_int),
                ("absorb_tc", C.c_int), ("si_coupled", C.c_int), ("warmup_rsvd", C.c_int),
                ("fp64_tc", C.c_int), ("svd_presolve", C.c_int), ("split_refine", C.c_double),
                ("stream", C.c_void_p)]


class ctm_solve_spec(C.Structure):
    _fields_ = [("Lx", C.c_int), ("Ly", C.c_int), ("d", C.c_int), ("D", C.c_int),
                ("chi", C.c_int), ("dtype", C.c_int), ("A", C.c_void_p), ("op", C.c_void_p),
                ("tol", C.c_double), ("max_iter", C.c_int), ("opts", ctm_opts)]


class ctm_solve_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("delta", C.c_double),
                ("queue_ms", C.c_double), ("run_ms", C.c_double), ("footprint", C.c_size_t)]


class CTMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


_lib = None


def load():
    """Load libctm.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libctm.so not built ({LIB_PATH}); run "
                          "`python -m paper_2607_15158_gb300.build` on a machine with nvcc")
    lib = C.CDLL(LIB_PATH)
    P, I, D, VP = C.POINTER, C.c_int, C.c_double, C.c_void_p
    ctx_p = VP
    sig = {
        "ctm_default_opts": (None, [P(ctm_opts)]),
        "ctm_init": (I, [P(ctx_p), I, I, P(VP), P(VP), I, I, I, I, P(ctm_opts)]),
        "ctm_init_network": (I, [P(ctx_p), I, I, P(VP), I, I, P(ctm_opts)]),
        "ctm_set_env": (I, [ctx_p, VP, VP]),
        "ctm_get_env": (I, [ctx_p, VP, VP]),
        "ctm_set_rangefinders": (I, [ctx_p, VP, VP]),
        "ctm_dims": (I, [ctx_p, P(I), P(I)]),
        "ctm_move": (I, [ctx_p, I]),
        "ctm_converge": (I, [ctx_p, D, I, P(I), P(D)]),
        "ctm_spectrum": (I, [ctx_p, I, I, I, P(D)]),
        "ctm_spectra": (I, [ctx_p, P(D)]),
        "ctm_expect": (I, [ctx_p, VP, I, I, I, P(D)]),
        "ctm_rdm2": (I, [ctx_p, I, I, I, P(D)]),
        "ctm_expect_site": (I, [ctx_p, VP, I, I, P(D)]),
        "ctm_expect_bond": (I, [ctx_p, VP, VP, I, I, I, P(D)]),
        "ctm_free_energy": (I, [ctx_p, P(D)]),
        "ctm_get_projectors": (I, [ctx_p, I, I, I, VP, VP]),
        "ctm_corner": (I, [ctx_p, I, I, I, I, VP]),
        "ctm_corner_apply": (I, [ctx_p, I, I, I, I, I, VP, VP]),
        "ctm_si_stats": (I, [ctx_p, P(C.c_long), P(C.c_long)]),
        "ctm_transfer_spectrum": (I, [ctx_p, I, I, I, P(D), P(D)]),
        "ctm_debug_fail_alloc": (None, [I]),
        "ctm_record": (I, [ctx_p, I]),
        "ctm_grad": (I, [ctx_p, VP, P(D), VP]),
        "ctm_grad_fixed_point": (I, [ctx_p, VP, D, I, P(D), VP, P(I), P(D)]),
        "ctm_last_timing": (I, [ctx_p, P(D), P(C.c_long)]),
        "ctm_profile_enable": (I, [ctx_p, I]),
        "ctm_profile_read": (I, [ctx_p, P(D), P(C.c_long), P(D), P(D)]),
        "ctm_profile_phases": (I, [ctx_p, P(D)]),
        "ctm_footprint": (I, [I, I, I, I, I, I, P(ctm_opts), P(C.c_size_t)]),
        "ctm_server_create": (I, [P(VP), C.c_size_t, I]),
        "ctm_server_submit": (I, [VP, P(ctm_solve_spec), P(C.c_uint64)]),
        "ctm_server_result": (I, [VP, C.c_uint64, P(ctm_solve_result), P(D), P(D)]),
        "ctm_server_stats": (I, [VP, P(D), P(D), P(D), P(I)]),
        "ctm_server_last_error": (C.c_char_p, [VP]),
        "ctm_server_free": (None, [VP]),
        "ctm_save": (I, [ctx_p, VP, P(C.c_size_t)]),
        "ctm_load": (I, [ctx_p, VP, C.c_size_t]),
        "ctm_free": (None, [ctx_p]),
        "ctm_last_error": (C.c_char_p, [ctx_p]),
        "ctm_svdvals_noalloc": (I, [VP, I, I, VP, VP]),
        "ctm_noalloc_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(lib, ctx, st, allow=()):
    if st != CTM_OK and st not in allow:
        raise CTMError(st, (lib.ctm_last_error(ctx) or b"").decode())
    return st


def _host(a, cplx):
    return np.ascontiguousarray(a, dtype=np.complex128 if cplx else np.float64)


def ctm_default_opts(**kw):
    lib = load()
    o = ctm_opts()
    lib.ctm_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Context:
    """Owns one ctm_ctx; methods are the C entry points of the same names."""

    def __init__(self, ptr, Lx, Ly, d, Dk, Db, chi, cplx):
        self.ptr = ptr
        self.Lx, self.Ly, self.d, self.Dk, self.Db, self.chi = Lx, Ly, d, Dk, Db, chi
        self.cplx = cplx
        self.lib = load()
        Nv, kv = C.c_int(), C.c_int()
        _check(self.lib, self.ptr, self.lib.ctm_dims(self.ptr, C.byref(Nv), C.byref(kv)))
        self.N, self.k = Nv.value, kv.value

    # -- lifetime
    def ctm_free(self):
        if self.ptr:
            self.lib.ctm_free(self.ptr)
            self.ptr = None

    close = ctm_free

    def __del__(self):
        try:
            self.ctm_free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.ctm_free()

    @property
    def dtype(self):
        return np.complex128 if self.cplx else np.float64

    # -- state
    def ctm_set_env(self, Cs, Ts):
        """Cs: [4][S][chi][chi], Ts: [4][S][chi][chi][Dk][Db] (nested lists or arrays)."""
        c = _host(np.asarray(Cs), self.cplx)
        t = _host(np.asarray(Ts), self.cplx)
        _check(self.lib, self.ptr, self.lib.ctm_set_env(self.ptr, c.ctypes.data, t.ctypes.data))

    def ctm_get_env(self):
        S = self.Lx * self.Ly
        c = np.empty((4, S, self.chi, self.chi), self.dtype)
        t = np.empty((4, S, self.chi, self.chi, self.Dk, self.Db), self.dtype)
        _check(self.lib, self.ptr, self.lib.ctm_get_env(self.ptr, c.ctypes.data, t.ctypes.data))
        return c, t

    def ctm_set_rangefinders(self, X, W):
        x = _host(np.asarray(X), self.cplx)
        w = _host(np.asarray(W), self.cplx)
        _check(self.lib, self.ptr,
               self.lib.ctm_set_rangefinders(self.ptr, x.ctypes.data, w.ctypes.data))

    # -- iteration
    def ctm_move(self, direction):
        _check(self.lib, self.ptr, self.lib.ctm_move(self.ptr, int(direction)))

    def ctm_converge(self, tol, max_iter):
        it, delta = C.c_int(), C.c_double()
        st = self.lib.ctm_converge(self.ptr, float(tol), int(max_iter), C.byref(it),
                                   C.byref(delta))
        _check(self.lib, self.ptr, st, allow=(CTM_ENOCONV,))
        return it.value, delta.value, st == CTM_OK

    # -- observables
    def ctm_spectrum(self, x, y, label):
        s = np.empty(self.chi)
        _check(self.lib, self.ptr, self.lib.ctm_spectrum(
            self.ptr, x, y, label, s.ctypes.data_as(C.POINTER(C.c_double))))
        return s

    def ctm_spectra(self):
        """All corner spectra, [4][Lx*Ly][chi] (unit-normalised)."""
        s = np.empty((4, self.Lx * self.Ly, self.chi))
        _check(self.lib, self.ptr, self.lib.ctm_spectra(
            self.ptr, s.ctypes.data_as(C.POINTER(C.c_double))))
        return s

    def ctm_expect(self, op, x, y, direction):
        o = _host(op, self.cplx)
        out = np.empty(2)
        _check(self.lib, self.ptr, self.lib.ctm_expect(
            self.ptr, o.ctypes.data, x, y, direction, out.ctypes.data_as(C.POINTER(C.c_double))))
        return complex(out[0], out[1])

    def ctm_rdm2(self, x, y, direction):
        d2 = self.d * self.d
        out = np.empty((d2, d2, 2))
        _check(self.lib, self.ptr, self.lib.ctm_rdm2(
            self.ptr, x, y, direction, out.ctypes.data_as(C.POINTER(C.c_double))))
        return out[..., 0] + 1j * out[..., 1]

    def ctm_expect_site(self, imp, x, y):
        o = _host(imp, self.cplx)
        out = np.empty(2)
        _check(self.lib, self.ptr, self.lib.ctm_expect_site(
            self.ptr, o.ctypes.data, x, y, out.ctypes.data_as(C.POINTER(C.c_double))))
        return complex(out[0], out[1])

    def ctm_expect_bond(self, imp1, imp2, x, y, direction):
        o1, o2 = _host(imp1, self.cplx), _host(imp2, self.cplx)
        out = np.empty(2)
        _check(self.lib, self.ptr, self.lib.ctm_expect_bond(
            self.ptr, o1.ctypes.data, o2.ctypes.data, x, y, direction,
            out.ctypes.data_as(C.POINTER(C.c_double))))
        return complex(out[0], out[1])

    def ctm_free_energy(self):
        v = C.c_double()
        _check(self.lib, self.ptr, self.lib.ctm_free_energy(self.ptr, C.byref(v)))
        return v.value

    def ctm_get_projectors(self, direction, x, y):
        Pl = np.empty((self.N, self.chi), self.dtype)
        PrH = np.empty((self.N, self.chi), self.dtype)
        _check(self.lib, self.ptr, self.lib.ctm_get_projectors(
            self.ptr, int(direction), x, y, Pl.ctypes.data, PrH.ctypes.data))
        return Pl, PrH

    def ctm_corner(self, direction, x, y, i):
        """Enlarged corner Q_i (1..4) of cut (x, y) in the frame of direction,
        N x N, built by the context's own path and precision."""
        Q = np.empty((self.N, self.N), self.dtype)
        _check(self.lib, self.ptr, self.lib.ctm_corner(self.ptr, int(direction), x, y, i,
                                                       Q.ctypes.data))
        return Q

    def ctm_corner_apply(self, direction, x, y, i, Z, herm=False):
        """op(Q_i) Z for a host N x k block (op = conjugate transpose when herm)."""
        z = _host(Z, self.cplx)
        out = np.empty((self.N, self.k), self.dtype)
        _check(self.lib, self.ptr, self.lib.ctm_corner_apply(
            self.ptr, int(direction), x, y, i, 1 if herm else 0, z.ctypes.data, out.ctypes.data))
        return out

    def ctm_record(self, on=True):
        """Start (on) or stop recording moves for ctm_grad."""
        _check(self.lib, self.ptr, self.lib.ctm_record(self.ptr, 1 if on else 0))

    def ctm_grad(self, op):
        """(E, dE/dA) through the recorded moves; dE/dA as [Lx*Ly][d,D,D,D,D]."""
        o = _host(op, False)
        dA = np.empty((self.Lx * self.Ly, self.d, self.Dk, self.Dk, self.Dk, self.Dk))
        E = C.c_double()
        _check(self.lib, self.ptr, self.lib.ctm_grad(self.ptr, o.ctypes.data, C.byref(E),
                                                     dA.ctypes.data))
        return E.value, dA

    def ctm_grad_fixed_point(self, op, tol=1e-10, max_iter=200):
        """(E, dE/dA, iterations, residual) by fixed-point differentiation."""
        o = _host(op, False)
        dA = np.empty((self.Lx * self.Ly, self.d, self.Dk, self.Dk, self.Dk, self.Dk))
        E, it, res = C.c_double(), C.c_int(), C.c_double()
        st = self.lib.ctm_grad_fixed_point(self.ptr, o.ctypes.data, float(tol), int(max_iter),
                                           C.byref(E), dA.ctypes.data, C.byref(it), C.byref(res))
        _check(self.lib, self.ptr, st, allow=(CTM_ENOCONV,))
        return E.value, dA, it.value, res.value

    def ctm_transfer_spectrum(self, direction=0, row=0, nvals=4):
        """(eigenvalues of largest modulus / |lambda_1|, correlation length) of
        the edge transfer matrix of one row (direction 0) or column (1)."""
        lam = np.empty(2 * nvals)
        xi = C.c_double()
        _check(self.lib, self.ptr, self.lib.ctm_transfer_spectrum(
            self.ptr, int(direction), int(row), int(nvals),
            lam.ctypes.data_as(C.POINTER(C.c_double)), C.byref(xi)))
        return lam[0::2] + 1j * lam[1::2], xi.value

    def ctm_si_stats(self):
        u, sk = C.c_long(), C.c_long()
        _check(self.lib, self.ptr, self.lib.ctm_si_stats(self.ptr, C.byref(u), C.byref(sk)))
        return u.value, sk.value

    def ctm_profile_enable(self, on=True):
        _check(self.lib, self.ptr, self.lib.ctm_profile_enable(self.ptr, 1 if on else 0))

    def ctm_profile_read(self):
        ms, n, fl, by = C.c_double(), C.c_long(), C.c_double(), C.c_double()
        _check(self.lib, self.ptr, self.lib.ctm_profile_read(
            self.ptr, C.byref(ms), C.byref(n), C.byref(fl), C.byref(by)))
        return ms.value, n.value, fl.value, by.value

    PHASES = ("corners", "slicing", "products", "qr", "small_problem", "absorption",
              "normalisation", "spectra")

    def ctm_profile_phases(self):
        ms = (C.c_double * len(self.PHASES))()
        _check(self.lib, self.ptr, self.lib.ctm_profile_phases(self.ptr, ms))
        return dict(zip(self.PHASES, list(ms)))

    def ctm_save(self):
        """Checkpoint of the iteration state as a bytes object."""
        n = C.c_size_t(0)
        _check(self.lib, self.ptr, self.lib.ctm_save(self.ptr, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(self.lib, self.ptr, self.lib.ctm_save(self.ptr, buf, C.byref(n)))
        return buf.raw[:n.value]

    def ctm_load(self, state):
        buf = C.create_string_buffer(bytes(state), len(state))
        _check(self.lib, self.ptr, self.lib.ctm_load(self.ptr, buf, len(state)))

    def ctm_last_timing(self):
        ms, n = C.c_double(), C.c_long()
        _check(self.lib, self.ptr, self.lib.ctm_last_timing(self.ptr, C.byref(ms), C.byref(n)))
        return ms.value, n.value


def ctm_footprint(Lx, Ly, d, D, chi, cplx, opts=None):
    """Device bytes a context of these dimensions allocates (upper estimate)."""
    lib = load()
    o = opts if opts is not None else ctm_default_opts()
    n = C.c_size_t(0)
    _check(lib, None, lib.ctm_footprint(Lx, Ly, d, D, chi, CTM_C128 if cplx else CTM_F64,
                                        C.byref(o), C.byref(n)))
    return n.value


class Server:
    """Serving runtime (ctm_server_*): solves of mixed cells admitted by
    device footprint, each on its own stream; methods are the C entry points
    of the same names."""

    def __init__(self, hbm_budget=0, max_concurrent=4):
        self.lib = load()
        self.ptr = C.c_void_p()
        st = self.lib.ctm_server_create(C.byref(self.ptr), hbm_budget, max_concurrent)
        if st != CTM_OK:
            raise CTMError(st, "ctm_server_create failed")
        self._keep = {}

    def ctm_server_submit(self, A, d, D, chi, tol, max_iter, op=None, cplx=None, opts=None,
                          Lx=1, Ly=1):
        if cplx is None:
            cplx = any(np.iscomplexobj(a) for a in A)
        arrs = [_host(a, cplx) for a in A]
        ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
        o = opts if opts is not None else ctm_default_opts()
        opa = _host(op, cplx) if op is not None else None
        spec = ctm_solve_spec(Lx, Ly, d, D, chi, CTM_C128 if cplx else CTM_F64,
                              C.cast(ptrs, C.c_void_p),
                              opa.ctypes.data if opa is not None else None, tol, max_iter, o)
        t = C.c_uint64(0)
        st = self.lib.ctm_server_submit(self.ptr, C.byref(spec), C.byref(t))
        if st != CTM_OK:
            raise CTMError(st, (self.lib.ctm_server_last_error(self.ptr) or b"").decode())
        self._keep[t.value] = (Lx * Ly, chi, opa is not None)
        return t.value

    def ctm_server_result(self, ticket):
        S, chi, has_op = self._keep.pop(ticket)
        res = ctm_solve_result()
        spec = np.empty((4, S, chi))
        en = np.empty((S, 2, 2)) if has_op else None
        st = self.lib.ctm_server_result(
            self.ptr, ticket, C.byref(res), spec.ctypes.data_as(C.POINTER(C.c_double)),
            en.ctypes.data_as(C.POINTER(C.c_double)) if en is not None else None)
        if st != CTM_OK:
            raise CTMError(st, (self.lib.ctm_server_last_error(self.ptr) or b"").decode())
        out = dict(iters=res.iters, delta=res.delta, queue_ms=res.queue_ms, run_ms=res.run_ms,
                   footprint=res.footprint, spectra=spec)
        if en is not None:
            out["energies"] = en[..., 0] + 1j * en[..., 1]
        return out

    def ctm_server_stats(self):
        p50, p99, sps, n = C.c_double(), C.c_double(), C.c_double(), C.c_int()
        self.lib.ctm_server_stats(self.ptr, C.byref(p50), C.byref(p99), C.byref(sps),
                                  C.byref(n))
        return dict(p50_ms=p50.value, p99_ms=p99.value, solves_per_s=sps.value,
                    completed=n.value)

    def ctm_server_free(self):
        if self.ptr:
            self.lib.ctm_server_free(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.ctm_server_free()
        except Exception:  # pragma: no cover
            pass


def ctm_svdvals_noalloc(A_dev, k, dtype, s_dev, stream=0):
    """Singular values of the k x k column-major matrix at device address
    A_dev into k doubles at device address s_dev, with no device allocation
    (scratch is the library's fixed device array); returns the status."""
    lib = load()
    st = lib.ctm_svdvals_noalloc(A_dev, k, dtype, s_dev, stream or None)
    if st != CTM_OK:
        raise CTMError(st, (lib.ctm_noalloc_last_error() or b"").decode())
    return st


def ctm_gemm_fp64tc(A, B, opA=0):
    """op(A) @ B through the library's fp64-accurate tensor-core product
    (host arrays; opA 0 = A, 1 = A^T, 2 = A^H)."""
    lib = load()
    cx = np.iscomplexobj(A) or np.iscomplexobj(B)
    a = _host(A, cx)
    b = _host(B, cx)
    M = a.shape[1] if opA else a.shape[0]
    K = a.shape[0] if opA else a.shape[1]
    if b.shape[0] != K:
        raise ValueError("inner dimensions differ")
    N = b.shape[1]
    c = np.empty((M, N), np.complex128 if cx else np.float64)
    _check(lib, None, lib.ctm_gemm_fp64tc(CTM_C128 if cx else CTM_F64, int(opA), a.ctypes.data,
                                          a.shape[1], b.ctypes.data, N, M, N, K, c.ctypes.data, N))
    return c


def ctm_debug_fail_alloc(after):
    """Make the device allocation after `after` successful ones fail (test
    hook of the error paths); after < 0 disarms it."""
    load().ctm_debug_fail_alloc(int(after))


def ctm_init(Lx, Ly, A, d, D, chi, cplx=None, bra=None, opts=None):
    """Create a context for an iPEPS cell: A is a list of Lx*Ly arrays
    [d, D, D, D, D]; bra=None means conj(A)."""
    lib = load()
    if cplx is None:
        cplx = any(np.iscomplexobj(a) for a in A)
    arrs = [_host(a, cplx) for a in A]
    ptrs = (C.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    bptrs = None
    if bra is not None:
        barrs = [_host(b, cplx) for b in bra]
        bptrs = (C.c_void_p * len(barrs))(*[b.ctypes.data for b in barrs])
    o = opts if opts is not None else ctm_default_opts()
    ptr = C.c_void_p()
    st = lib.ctm_init(C.byref(ptr), Lx, Ly, ptrs, bptrs, CTM_C128 if cplx else CTM_F64, d, D,
                      chi, C.byref(o))
    _check(lib, None, st)
    ctx = Context(ptr, Lx, Ly, d, D, D, chi, cplx)
    ctx._keep = (arrs, o)
    return ctx


def ctm_init_network(Lx, Ly, a, chi, opts=None):
    """Create a context for a classical network: a is a list of Lx*Ly real
    arrays [k, k, k, k] (u, l, d, r)."""
    lib = load()
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in a]
    k = arrs[0].shape[0]
    ptrs = (C.c_void_p * len(arrs))(*[x.ctypes.data for x in arrs])
    o = opts if opts is not None else ctm_default_opts()
    ptr = C.c_void_p()
    st = lib.ctm_init_network(C.byref(ptr), Lx, Ly, ptrs, k, chi, C.byref(o))
    _check(lib, None, st)
    ctx = Context(ptr, Lx, Ly, 1, k, 1, chi, False)
    ctx._keep = (arrs, o)
    return ctx
