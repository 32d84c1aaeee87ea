"""The allocation-free entry point against the allocating one, on the GPU.

ar_restore_plain_static() serves callers that cannot let a library allocate
device memory (the whole GPU already reserved for their own pool, or a
fixed-budget service).  It keeps its scratch in a static device array, so its
result must equal ar_restore(..., precondition=0) on the same inputs; two calls
in a row check that the shared array is correctly reset between calls.  This
file is collected last so that a failure here cannot hide another test's
result in a run that stops at the first failure.
"""

import numpy as np
import pytest
import torch

from paper_1211_0393_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_static_scratch_restore_matches_allocating_restore_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0393_gb300 import ar

    ar.lib()
    h = W.psf_config1()
    n = 96
    rng = np.random.default_rng(7)
    f = rng.uniform(0, 1, (n, n)).astype(np.float32)
    g = (f + 0.01 * rng.standard_normal((n, n))).astype(np.float32)
    gd = torch.from_numpy(g).cuda()
    fd = torch.from_numpy(f).cuda()
    x_ref, tr_ref, best_ref = ar.ar_restore(gd, h, 0.0, 1.0, 12, False, f_true=fd)
    x_ref = x_ref.cpu().numpy().astype(np.float64)
    for call in range(2):
        x, tr, best = ar.ar_restore_plain_static(gd, h, 1.0, 12, f_true=fd)
        x = x.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref)
        assert err <= 1e-5, (call, err)
        np.testing.assert_allclose(tr, tr_ref, rtol=1e-5)
        assert best == best_ref
    with pytest.raises(ar.ARError) as ei:      # larger than the static scratch
        big = torch.zeros(1025, 1024, device="cuda")
        ar.ar_restore_plain_static(big, h, 1.0, 1)
    assert ei.value.name == "AR_ERR_INVALID_ARG"
