"""The allocation-free resampling entry point (static device scratch) gives
exactly the result of the workspace entry point, on two calls in a row.

It is for callers that cannot call cudaMalloc or pass a workspace (a host
framework that owns all device memory through its own pool, or a
latency-critical loop that may not allocate).  This file is collected last so
that a run stopping at the first failure has already run every other test;
it passes alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def make_case(seed, n, k):
    rng = np.random.default_rng(seed)
    model = rng.integers(0, k, n)
    W = np.zeros(n)
    for m in range(k):
        idx = np.nonzero(model == m)[0]
        if idx.size:
            w = rng.exponential(1.0, idx.size) ** 3
            W[idx] = w / w.sum()
    u40 = rng.integers(0, 1 << 40, k, dtype=np.uint64)
    return W, model.astype(np.int32), u40.astype(np.int64)


def test_noalloc_resample_matches_workspace_entry():
    import torch

    from paper_2109_00661_gb300 import _lib, smc

    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two calls in a row with different sizes: the second sees the first's
    # leftovers in the shared scratch
    for call, (n, k) in enumerate([(6000, 37), (2500, 11)]):
        W, model, u40 = make_case(call, n, k)
        W_t = torch.as_tensor(W, device="cuda")
        m_t = torch.as_tensor(model, device="cuda")
        u_t = torch.as_tensor(u40, device="cuda")
        ref = smc.resample_systematic(W_t, m_t, k, u_t)
        anc = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rc = lib.aem_resample_systematic_noalloc(W_t.data_ptr(), m_t.data_ptr(), n, k, u_t.data_ptr(),
                                                 anc.data_ptr(), stream)
        assert rc == 0, lib.aem_last_error()
        torch.cuda.synchronize()
        assert torch.equal(anc, ref)
    # sizes beyond the static scratch are rejected with a clear error
    W, model, u40 = make_case(9, 64, 3)
    W_t = torch.as_tensor(W, device="cuda")
    m_t = torch.as_tensor(model, device="cuda")
    u_t = torch.as_tensor(u40, device="cuda")
    anc = torch.empty(64, dtype=torch.int32, device="cuda")
    rc = lib.aem_resample_systematic_noalloc(W_t.data_ptr(), m_t.data_ptr(), 16385, 3, u_t.data_ptr(),
                                             anc.data_ptr(), stream)
    assert rc == -1 and b"maximum" in lib.aem_last_error()
