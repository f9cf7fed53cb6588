"""ctm_svdvals_noalloc (fixed device scratch, no allocation) against the
existing entry point ctm_spectrum on the same corner matrices.

Both run the one-sided Jacobi SVD; the no-alloc call returns unnormalised
singular values, ctm_spectrum the unit-normalised spectrum, so the test
normalises before comparing. Two calls in a row on the same scratch must both
agree (the error word and barrier counters are cleared by each call).
Tolerance: 1e-10 relative to the largest singular value, the FP64 bar of the
parity tests. Device buffers for the inputs and outputs come from torch; the
call under test allocates nothing.
"""
import numpy as np
import pytest

import ctm_synth as S
import paper_2607_15158_gb300 as pkg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = 1e-10


def _ctx(cplx):
    Lx, Ly, d, D, chi = (2, 1, 2, 2, 20) if cplx else (1, 1, 2, 3, 27)
    A = S.ipeps_tensors(Lx, Ly, d, D, complex_=cplx, seed=0)
    Cs, Ts = S.initial_env(Lx, Ly, chi, D, D, complex_=cplx, seed=1)
    ctx = pkg.ctm_init(Lx, Ly, A, d, D, chi, cplx=cplx,
                       opts=pkg.ctm_default_opts(p=4, si_rounds=2))
    ctx.ctm_set_env(Cs, Ts)
    for direction in range(4):
        ctx.ctm_move(direction)
    return ctx


def _noalloc(mat, cplx):
    """Run the no-alloc call on a device copy of mat; returns host values."""
    k = mat.shape[0]
    a = torch.from_numpy(np.asfortranarray(mat).ravel(order="F").copy()).cuda()
    s = torch.empty(k, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    pkg.ctm_svdvals_noalloc(a.data_ptr(), k, pkg.CTM_C128 if cplx else pkg.CTM_F64,
                            s.data_ptr(), stream)
    return s.cpu().numpy()


def test_noalloc_calls_leave_free_device_memory_unchanged():
    """After a first call on the device (which looks up the scratch address),
    further calls change the device's free memory by nothing: the call itself
    allocates no device memory."""
    rng = np.random.default_rng(7)
    k = 64
    m = rng.standard_normal((k, k))
    a = torch.from_numpy(np.asfortranarray(m).ravel(order="F").copy()).cuda()
    s = torch.empty(k, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    pkg.ctm_svdvals_noalloc(a.data_ptr(), k, pkg.CTM_F64, s.data_ptr(), stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        pkg.ctm_svdvals_noalloc(a.data_ptr(), k, pkg.CTM_F64, s.data_ptr(), stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


@pytest.mark.parametrize("cplx", [False, True])
def test_noalloc_matches_ctm_spectrum_twice(cplx):
    ctx = _ctx(cplx)
    c, _ = ctx.ctm_get_env()
    for label in (1, 3):
        mat = c[label - 1][0]
        ref = ctx.ctm_spectrum(0, 0, label)
        ref = ref / np.linalg.norm(ref)
        for _ in range(2):                   # two calls in a row on one scratch
            s = _noalloc(mat, cplx)
            assert np.all(np.diff(s) <= 0)
            assert np.max(np.abs(s / np.linalg.norm(s) - ref)) <= TOL * ref[0]
            # unnormalised values are the matrix's own singular values
            sv = np.linalg.svd(mat, compute_uv=False)
            assert np.max(np.abs(s - sv)) <= TOL * sv[0]
    ctx.ctm_free()


def test_noalloc_largest_size_and_rejection():
    rng = np.random.default_rng(5)
    k = 256
    m = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
    sv = np.linalg.svd(m, compute_uv=False)
    for _ in range(2):
        s = _noalloc(m, True)
        assert np.max(np.abs(s - sv)) <= TOL * sv[0]
    a = torch.zeros(2 * 257 * 257, dtype=torch.float64, device="cuda")
    out = torch.empty(257, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.CTMError) as e:
        pkg.ctm_svdvals_noalloc(a.data_ptr(), 257, pkg.CTM_C128, out.data_ptr(), 0)
    assert e.value.status == pkg.CTM_EINVAL
