"""sptt_gram_noalloc: the Gram kernel with a static device workspace, for
callers that cannot allocate device memory (memory owned by another
allocator, or a path where an allocation may synchronise). Checked through
the C ABI against sptt_gram, which allocates its workspace per call, on two
calls in a row (the second reuses the workspace the first left behind).
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import paper_1812_05961_gb300 as sptt

pytestmark = pytest.mark.gpu


def _call(fn, A, R, G, stream):
    st = fn(ctypes.c_void_p(A.data_ptr()), A.shape[0], R, A.shape[1], ctypes.c_void_p(G.data_ptr()),
            ctypes.c_void_p(stream.cuda_stream))
    assert st == sptt.SPTT_OK, sptt.sptt_last_error()


def test_gram_noalloc_matches_gram_twice(cuda_device):
    lib = sptt.lib()
    stream = torch.cuda.current_stream()
    g = torch.Generator().manual_seed(17)
    for rows, R, ld in ((100_000, 16, 16), (33_333, 61, 64)):   # two calls in a row
        A = (torch.rand(rows, ld, generator=g) - 0.5).to(cuda_device)
        G_ref = torch.empty(R, R, dtype=torch.float64, device=cuda_device)
        G_new = torch.full((R, R), float("nan"), dtype=torch.float64, device=cuda_device)
        _call(lib.sptt_gram, A, R, G_ref, stream)
        _call(lib.sptt_gram_noalloc, A, R, G_new, stream)
        torch.cuda.synchronize()
        ref = G_ref.cpu().numpy()
        new = G_new.cpu().numpy()
        assert np.isfinite(new).all()
        assert np.abs(new - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


def test_gram_noalloc_rejects_rank_beyond_workspace(cuda_device):
    A = torch.zeros(10, 72, device=cuda_device)
    G = torch.zeros(65, 65, dtype=torch.float64, device=cuda_device)
    with pytest.raises(sptt.SpttError) as e:
        sptt.sptt_gram_noalloc(A, 65, G)
    assert e.value.status == sptt.SPTT_ERR_BAD_ARG
