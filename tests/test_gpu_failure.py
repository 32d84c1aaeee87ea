"""Failure detection on the GPU without a GPU fault.

* A stencil whose wait for its halo tile gives up (the poll limit set to 0 from
  the host, so that no wait can succeed) waits for its copies in flight, sets
  the device flag and returns: the restoration reports AR_ERR_TIMEOUT, the
  context stays usable, and the next call with the default limit returns the
  same iterate as a call that never timed out.
* An allocation failure injected on the host (a fake of the failing
  cudaMallocAsync) makes the call return AR_ERR_ALLOC and leaves the library
  usable.
"""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ar():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0393_gb300 import ar as mod

    mod.lib()
    return mod


def _inputs(n1, n2, seed):
    rng = np.random.default_rng(seed)
    f = rng.uniform(0, 1, (n1, n2)).astype(np.float32)
    g = (f + 0.01 * rng.standard_normal((n1, n2))).astype(np.float32)
    h = rng.uniform(0, 1, (9, 9))
    return torch.from_numpy(g).cuda(), torch.from_numpy(f).cuda(), h / h.sum()


@pytest.mark.parametrize("pc", [True, False])
@pytest.mark.parametrize("stencil", ["fp32", "f16x2"])
def test_stencil_wait_timeout_is_reported_and_recoverable(ar, pc, stencil):
    # n2 % 4 == 0 and 16-byte aligned rows: the TMA stencils (and, preconditioned,
    # the folding reblur) run; f16x2: the tensor-core stencils (producer warp and
    # compute warps, and the folding pair whose ranks exchange the give-up)
    gd, fd, h = _inputs(256, 192, 3)
    want, tr_want, _ = ar.ar_restore(gd, h, 0.1, 1.0, 4, pc, f_true=fd, stencil=stencil)
    want = want.clone()
    try:
        ar.set_stencil_wait_polls(0)
        with pytest.raises(ar.ARError) as ei:
            ar.ar_restore(gd, h, 0.1, 1.0, 4, pc, f_true=fd, stencil=stencil)
        assert ei.value.name == "AR_ERR_TIMEOUT"
        assert "stencil" in str(ei.value)
    finally:
        ar.set_stencil_wait_polls()
    torch.cuda.synchronize()                       # the context is still usable
    got, tr, _ = ar.ar_restore(gd, h, 0.1, 1.0, 4, pc, f_true=fd, stencil=stencil)
    assert torch.equal(got, want)
    np.testing.assert_allclose(tr, tr_want, rtol=1e-12)


def test_static_restore_reports_stencil_timeout(ar):
    gd, fd, h = _inputs(128, 128, 4)
    want, _, _ = ar.ar_restore_plain_static(gd, h, 1.0, 3)
    want = want.clone()
    try:
        ar.set_stencil_wait_polls(0)
        with pytest.raises(ar.ARError) as ei:
            ar.ar_restore_plain_static(gd, h, 1.0, 3)
        assert ei.value.name == "AR_ERR_TIMEOUT"
    finally:
        ar.set_stencil_wait_polls()
    got, _, _ = ar.ar_restore_plain_static(gd, h, 1.0, 3)
    assert torch.equal(got, want)


def test_injected_allocation_failure_then_success(ar):
    """One device allocation of a preconditioned restoration fails, after `skip`
    successful ones (skip 0 is the first scratch buffer; from 4 on they fall in the
    preconditioner's build, from 7 on in its transform plan's operands): the call
    returns AR_ERR_ALLOC, and the next call returns the usual iterate."""
    gd, fd, h = _inputs(96, 96, 5)
    want, _, _ = ar.ar_restore(gd, h, 0.1, 1.0, 3, True)
    want = want.clone()
    for skip in (0, 2, 5, 6, 9, 11):
        try:
            ar.inject_alloc_failures(1, skip=skip)
            with pytest.raises(ar.ARError) as ei:
                ar.ar_restore(gd, h, 0.1, 1.0, 3, True)
            assert ei.value.name == "AR_ERR_ALLOC"
        finally:
            ar.inject_alloc_failures(0)
        got, _, _ = ar.ar_restore(gd, h, 0.1, 1.0, 3, True)
        assert torch.equal(got, want)
    try:
        ar.inject_alloc_failures(1, skip=1)
        with pytest.raises(ar.ARError) as ei:
            ar.ar_symprec_setup(h, 96, 96, 0.1)
        assert ei.value.name == "AR_ERR_ALLOC"
    finally:
        ar.inject_alloc_failures(0)
