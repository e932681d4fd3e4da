"""sptt_gram_noalloc: the Gram kernel with a static device workspace, for
callers that cannot allocate device memory (memory owned by another
allocator, or a path where an allocation may synchronise). Checked through
the C ABI against sptt_gram, which allocates its workspace per call, and
against numpy's FP64 A^T A, on two calls in a row (the second reuses the
workspace the first left behind). The shapes cover the three kernel
instances (padded rank 16, 32 and 64). This file is collected last on
purpose."""
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
    # rank 16 (padded 16), 29 (padded 32) and 61 (padded 64)
    for rows, R, ld in ((100_000, 16, 16), (50_001, 29, 32), (33_333, 61, 64)):
        A_host = torch.rand(rows, ld, generator=g) - 0.5
        A = A_host.to(cuda_device)
        ref64 = A_host[:, :R].double().numpy()
        ref64 = ref64.T @ ref64
        tol = 1e-5 * max(1.0, np.abs(ref64).max())
        G_ref = torch.empty(R, R, dtype=torch.float64, device=cuda_device)
        _call(lib.sptt_gram, A, R, G_ref, stream)
        for _ in range(2):  # two calls in a row on the shared workspace
            G_new = torch.full((R, R), float("nan"), dtype=torch.float64, device=cuda_device)
            _call(lib.sptt_gram_noalloc, A, R, G_new, stream)
            torch.cuda.synchronize()
            new = G_new.cpu().numpy()
            assert np.isfinite(new).all()
            assert np.abs(new - G_ref.cpu().numpy()).max() <= tol
            assert np.abs(new - ref64).max() <= tol


def test_gram_noalloc_rejects_rank_beyond_workspace(cuda_device):
    A = torch.zeros(10, 72, device=cuda_device)
    G = torch.zeros(65, 65, dtype=torch.float64, device=cuda_device)
    with pytest.raises(sptt.SpttError) as e:
        sptt.sptt_gram_noalloc(A, 65, G)
    assert e.value.status == sptt.SPTT_ERR_UNSUPPORTED
    with pytest.raises(sptt.SpttError) as e:
        sptt.sptt_gram(A, 65, G)
    assert e.value.status == sptt.SPTT_ERR_UNSUPPORTED
