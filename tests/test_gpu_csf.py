"""GPU sort/coalesce + CSF build against the oracle: bit-exact integers and
values (Section III, Section V-C)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1812_05961_gb300 as sptt
from gpu_util import make, to_dev

pytestmark = pytest.mark.gpu

CASES = [
    # dims, nnz, kind
    ((200, 150, 100), 20000, "uniform"),
    ((50, 40, 30, 20), 30000, "uniform"),
    ((12, 9, 7, 5, 3), 2000, "uniform"),
    ((300, 200, 100), 4096 * 3 + 17, "zipf"),        # ragged sort tile
    ((1, 300, 7), 1500, "uniform"),                   # length-1 mode
    ((40, 1, 1), 30, "uniform"),
    ((5000, 4000), 70000, "zipf"),                    # 2 modes, many scan tiles
    ((2_000_000, 500_000, 50_000, 1_000), 50000, "zipf"),  # keys wider than 64 bits
    ((64, 64, 64), 1, "uniform"),
]


def _check_csf(c, ref):
    n = c.nmodes
    assert c.order == ref["order"]
    assert c.nfibs == ref["nfibs"]
    lv = c.levels()
    for l in range(n):
        fptr, fids, vals = lv[l]
        np.testing.assert_array_equal(fids.numpy(), ref["fids"][l])
        if l < n - 1:
            np.testing.assert_array_equal(fptr.numpy(), ref["fptr"][l])
        else:
            np.testing.assert_array_equal(vals.numpy().view(np.uint32), ref["vals"].view(np.uint32))


@pytest.mark.parametrize("case", CASES, ids=[str(i) for i in range(len(CASES))])
def test_csf_bit_exact_every_root(case, cuda_device):
    dims, nnz, kind = case
    t = make(dims, nnz, seed=len(dims) * 7 + nnz % 97, dist=kind, s=1.2)
    inds_np, vals_np = t.numpy()
    di, dv = to_dev(t, cuda_device)
    for root in range(len(dims)):
        ref = oracle.csf(inds_np, vals_np, dims, root)
        c = sptt.Csf(dims, di, dv, root)
        _check_csf(c, ref)


def test_csf_custom_order_and_host_input(cuda_device):
    t = make((30, 20, 10, 8), 3000, seed=3)
    inds_np, vals_np = t.numpy()
    order = [2, 0, 3, 1]
    ref = oracle.csf(inds_np, vals_np, t.dims, 2, order)
    c = sptt.Csf(t.dims, t.inds, t.vals, 2, level_order=order)  # host tensors: copied inside
    _check_csf(c, ref)


@pytest.mark.parametrize("seed", [1, 2])
def test_csf_coalesces_duplicates_bit_exact(seed, cuda_device):
    t = make((20, 15, 10), 9000, seed=seed, dups=True, values="uniform")
    # heavy duplication: also repeat a block of entries many times
    inds_np, vals_np = t.numpy()
    di, dv = to_dev(t, cuda_device)
    for root in range(3):
        ref = oracle.csf(inds_np, vals_np, t.dims, root)
        assert ref["nfibs"][-1] < t.nnz
        _check_csf(sptt.Csf(t.dims, di, dv, root), ref)


def test_csf_empty_tensor(cuda_device):
    dims = (5, 6, 7)
    e = torch.zeros(0, dtype=torch.int32, device=cuda_device)
    c = sptt.Csf(dims, [e, e, e], torch.zeros(0, device=cuda_device), 1)
    assert c.nfibs == [0, 0, 0]
    for l in range(2):
        assert c.levels()[l][0].tolist() == [0]


def test_csf_rejects_bad_input(cuda_device):
    i = torch.tensor([0, 1, 5], dtype=torch.int32, device=cuda_device)
    j = torch.tensor([0, 0, 0], dtype=torch.int32, device=cuda_device)
    v = torch.ones(3, device=cuda_device)
    with pytest.raises(sptt.SpttError) as e:
        sptt.Csf((5, 2), [i, j], v, 0)
    assert e.value.status == sptt.SPTT_ERR_BAD_ARG
    i = torch.tensor([0, -1, 2], dtype=torch.int32, device=cuda_device)
    with pytest.raises(sptt.SpttError):
        sptt.Csf((5, 2), [i, j], v, 0)
    i = torch.tensor([0, 1, 2], dtype=torch.int32, device=cuda_device)
    with pytest.raises(sptt.SpttError):
        sptt.Csf((5, 2), [i, j], v, 0, level_order=[1, 0])
    with pytest.raises(sptt.SpttError):
        sptt.Csf((5, 2), [i, j], v, 2)
