"""hm_apply_noalloc: the allocation-free apply gives hm_apply's results.

This entry point serves callers that cannot allocate device memory when they
apply the compressed operator (for example a serving loop whose free device
memory belongs to another framework's caching allocator, or one that must not
wait on cudaMalloc/cudaFree mid-request).  It takes its scratch from one array
held inside the library.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import hm_workloads as W

from gpu_helpers import hm, run_gpu

pytestmark = pytest.mark.gpu


def test_apply_noalloc_matches_apply_on_two_calls():
    import torch
    m = hm()
    w = W.torus_laplace(n=20000, tol=1e-8, r=24)
    comp, _ = run_gpu(w, keep=False)
    X = torch.from_numpy(np.random.default_rng(0).standard_normal((w.n, 2))).cuda()
    for trans in (0, 1):
        a0 = comp.info().device_allocs
        ref = comp.apply(X, trans)
        assert comp.info().device_allocs > a0  # hm_apply allocates its scratch
        for _ in range(2):  # the scratch array keeps the previous call's contents
            # hm_info.device_allocs counts every device allocation the library
            # makes; the binding's output tensor comes from torch, outside it
            a0 = comp.info().device_allocs
            got = comp.apply_noalloc(X, trans)
            assert comp.info().device_allocs == a0, "hm_apply_noalloc allocated device memory"
            assert torch.linalg.norm(got - ref) <= 1e-10 * torch.linalg.norm(ref)
    # a request larger than the scratch array is refused with a clear error
    big = torch.zeros((w.n, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(m.HMError) as ei:
        comp.apply_noalloc(big)
    assert ei.value.status == m.HM_ENOTSUP and "MiB" in str(ei.value)
    # and the context is still usable afterwards
    got = comp.apply_noalloc(X, 0)
    assert torch.linalg.norm(got - comp.apply(X, 0)) <= 1e-10 * torch.linalg.norm(got)
    comp.close()
