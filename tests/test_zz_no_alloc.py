"""The allocation-free entry point against the allocating one, on the GPU.

ar_restore_plain_static() serves callers that cannot let a library allocate
device memory (the whole GPU already reserved for their own pool, or a
fixed-budget service).  It keeps its scratch in a static device array, so its
result must equal ar_restore(..., precondition=0) on the same inputs; two calls
in a row check that the shared array is correctly reset between calls.  A
second test checks that a call allocates nothing: neither from the device's
stream-ordered pool (the pool's high-water mark, read through the driver),
nor through cudaMalloc (free device memory), nor through PyTorch's allocator.
That includes the address lookups of the static scratch and of the stencils'
bounded-wait flag.  This file is collected last so that a failure here cannot
hide another test's result in a run that stops at the first failure.
"""

import ctypes
import gc

import numpy as np
import pytest
import torch

from paper_1211_0393_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# CUmemPool_attribute values (cuda.h)
_USED_MEM_CURRENT = 7
_USED_MEM_HIGH = 8


def _inputs(n=96, seed=7):
    rng = np.random.default_rng(seed)
    f = rng.uniform(0, 1, (n, n)).astype(np.float32)
    g = (f + 0.01 * rng.standard_normal((n, n))).astype(np.float32)
    return torch.from_numpy(g).cuda(), torch.from_numpy(f).cuda()


def test_static_scratch_restore_matches_allocating_restore_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0393_gb300 import ar

    ar.lib()
    h = W.psf_config1()
    gd, fd = _inputs()
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


def _pool_reader():
    """(read(attr) -> int, reset_high()) on the current device's default pool."""
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int(0)
    assert cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0

    def read(attr):
        v = ctypes.c_uint64(0)
        assert cu.cuMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high():
        z = ctypes.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(pool, _USED_MEM_HIGH, ctypes.byref(z)) == 0

    return read, reset_high


def test_static_restore_allocates_nothing():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0393_gb300 import ar

    ar.lib()
    h = W.psf_config1()
    gd, fd = _inputs(80, 11)
    x = torch.empty_like(gd)
    torch.cuda.synchronize()
    read, reset_high = _pool_reader()
    free = []
    for call in range(2):
        gc.collect()
        used = read(_USED_MEM_CURRENT)
        reset_high()
        torch.cuda.reset_peak_memory_stats()
        torch_bytes = torch.cuda.memory_allocated()
        free.append(torch.cuda.mem_get_info()[0])
        # the first call in a process looks up the device addresses of the static
        # scratch and of the stencils' wait flag
        ar.ar_restore_plain_static(gd, h, 1.0, 6, f_true=fd, x_out=x)
        torch.cuda.synchronize()
        assert read(_USED_MEM_HIGH) <= used, (call, "stream-ordered pool grew")
        assert torch.cuda.max_memory_allocated() <= torch_bytes, (call, "torch allocation")
    # the first call may load the library's device code (driver-owned memory);
    # the second may change no free memory at all
    assert torch.cuda.mem_get_info()[0] == free[1]
