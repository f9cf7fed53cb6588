"""Checkpoint / resume through the C ABI (ctm_save, ctm_load): a context
loaded from a checkpoint continues the iteration exactly (bit for bit) as the
context that wrote it; a checkpoint of other dimensions is refused."""
import numpy as np
import pytest

import ctm_synth as S
import paper_2607_15158_gb300 as pkg

pytestmark = pytest.mark.gpu


def _ctx(prec, chi=8, D=2):
    A = S.ipeps_tensors(2, 1, 2, D, complex_=True, seed=0)
    Cs, Ts = S.initial_env(2, 1, chi, D, D, complex_=True, seed=1)
    ctx = pkg.ctm_init(2, 1, A, 2, D, chi, cplx=True,
                       opts=pkg.ctm_default_opts(prec=prec, warmup_iters=2))
    ctx.ctm_set_env(Cs, Ts)
    return ctx


@pytest.mark.parametrize("prec", [pkg.CTM_PREC_FP64, pkg.CTM_PREC_SPLIT_BF16])
def test_resume_is_bit_exact(prec):
    a = _ctx(prec)
    a.ctm_converge(0.0, 3)
    state = a.ctm_save()
    a.ctm_converge(0.0, 2)
    ca, ta = a.ctm_get_env()
    b = _ctx(prec)
    b.ctm_load(state)
    b.ctm_converge(0.0, 2)
    cb, tb = b.ctm_get_env()
    assert np.array_equal(ca, cb) and np.array_equal(ta, tb)
    a.ctm_free()
    b.ctm_free()


def test_load_refuses_other_dimensions():
    a = _ctx(pkg.CTM_PREC_FP64, chi=8)
    b = _ctx(pkg.CTM_PREC_FP64, chi=9)
    state = a.ctm_save()
    with pytest.raises(pkg.CTMError) as e:
        b.ctm_load(state)
    assert e.value.status == pkg.CTM_EINVAL
    a.ctm_free()
    b.ctm_free()
