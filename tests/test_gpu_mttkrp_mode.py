"""MTTKRP of every mode from one CSF (Section III; output conflicts as in
Section IV-A / V-D-2) against the oracle's element definition.

Tolerances as for the root-mode MTTKRP: FP32 gathers 1e-5 relative
(Frobenius, and element-wise against the scale sum |v| prod |A|); BF16
gathers 1e-5 against the same BF16-rounded factors.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1812_05961_gb300 as sptt
import tensorgen
from gpu_util import make, rand_factors, rel_fro, to_dev

pytestmark = pytest.mark.gpu


def _check(M, t, F, mode, R, tol=1e-5):
    inds_np, vals_np = t.numpy()
    Fo = [f[:, :R].double().numpy() for f in F]
    Mo, Ma = oracle.mttkrp(inds_np, vals_np, t.dims, Fo, mode, with_abs=True)
    assert rel_fro(M[:, :R], Mo) <= tol
    assert np.all(np.abs(M[:, :R] - Mo) <= tol * Ma + 1e-30)


def _modes(c, t, F, dev, dtype=sptt.SPTT_F32, sched=None):
    tdt = torch.bfloat16 if dtype == sptt.SPTT_BF16 else torch.float32
    fd = [f.to(dev).to(tdt).contiguous() for f in F]
    ld = F[0].shape[1]
    out = []
    for m in range(len(t.dims)):
        o = torch.full((t.dims[m], ld), float("nan"), device=dev)  # must be overwritten
        c.mttkrp_mode(m, fd, out=o, factor_dtype=dtype, sched=sched)
        out.append(o.cpu().double().numpy())
    return out


@pytest.mark.parametrize("dims,nnz,dist", [
    ((200, 150, 100), 20000, "uniform"),
    ((500, 400, 300), 60000, "zipf"),
    ((60, 50, 40, 30), 40000, "zipf"),
    ((20, 18, 16, 14, 12), 30000, "uniform"),
    ((3000, 2500), 50000, "zipf"),
    ((1, 200, 100), 5000, "uniform"),
])
@pytest.mark.parametrize("ld", [4, 16, 64])
@pytest.mark.parametrize("variant", [0, 1])
def test_every_mode_from_one_csf(dims, nnz, dist, ld, variant, cuda_device):
    t = make(dims, nnz, seed=ld + len(dims), dist=dist, s=1.2)
    F = rand_factors(dims, ld, seed=ld)
    di, dv = to_dev(t, cuda_device)
    c = sptt.Csf(t.dims, di, dv, 0)
    for m, M in enumerate(_modes(c, t, F, cuda_device, sched=(128, 256, variant))):
        _check(M, t, F, m, ld)


@pytest.mark.parametrize("root,order", [(1, [1, 0, 2, 3]), (1, [1, 3, 2, 0]), (2, [2, 0, 1, 3]), (3, None)])
def test_custom_level_orders(root, order, cuda_device):
    dims = (100, 80, 60, 40)
    t = make(dims, 30000, seed=4, dist="zipf", s=1.3)
    F = rand_factors(dims, 8, seed=3)
    di, dv = to_dev(t, cuda_device)
    c = sptt.Csf(t.dims, di, dv, root, level_order=order)
    for m, M in enumerate(_modes(c, t, F, cuda_device)):
        _check(M, t, F, m, 8)


@pytest.mark.parametrize("chunk", [16, 64, 4096])
def test_chunk_sizes(chunk, cuda_device):
    dims = (400, 300, 200, 20)
    t = make(dims, 50003, seed=5, dist="zipf", s=1.3)
    F = rand_factors(dims, 16, seed=1)
    di, dv = to_dev(t, cuda_device)
    c = sptt.Csf(t.dims, di, dv, 0)
    for variant in (0, 1, 2):
        for m, M in enumerate(_modes(c, t, F, cuda_device, sched=(chunk, 256, variant))):
            _check(M, t, F, m, 16)


@pytest.mark.parametrize("ld", [8, 16, 32])
def test_bf16_gathers(ld, cuda_device):
    dims = (300, 250, 200, 50)
    t = make(dims, 50000, seed=ld, dist="zipf", s=1.1)
    F = rand_factors(dims, ld, seed=ld, lo=0.0, hi=1.0)
    Fb = [f.to(torch.bfloat16).float() for f in F]
    di, dv = to_dev(t, cuda_device)
    c = sptt.Csf(t.dims, di, dv, 0)
    for m, M in enumerate(_modes(c, t, F, cuda_device, dtype=sptt.SPTT_BF16)):
        _check(M, t, Fb, m, ld)


def _skewed(dims, n, hot_mode, frac, seed):
    # most non-zeros share index 0 of hot_mode: one output row with a very
    # large number of contributions
    g = torch.Generator().manual_seed(seed)
    cols = []
    for m, d in enumerate(dims):
        x = torch.randint(0, d, (n,), generator=g)
        if m == hot_mode:
            x = torch.where(torch.rand(n, generator=g) < frac, torch.zeros_like(x), x)
        cols.append(x)
    key = torch.zeros(n, dtype=torch.int64)
    for m, d in enumerate(dims):
        key = key * d + cols[m]
    _, first = np.unique(key.numpy(), return_index=True)
    keep = torch.from_numpy(np.sort(first))
    inds = [x[keep].int() for x in cols]
    vals = torch.rand(keep.numel(), generator=g)
    return tensorgen.CooTensor(list(dims), inds, vals)


@pytest.mark.parametrize("hot_mode", [0, 1, 2])
def test_hot_rows_at_every_level(hot_mode, cuda_device):
    # ~1.8e5 contributions to one row. Privatised (default): 1e-5. Global
    # reductions only (variant 1) add the row's contributions one by one in
    # FP32, whose error grows like sqrt(n) 2^-24 of the row's scale: checked
    # against 8 sqrt(n) 2^-24 with n the row's contribution count.
    dims = (600, 3000, 400)
    t = _skewed(dims, 300000, hot_mode, 0.6, seed=hot_mode)
    F = rand_factors(dims, 16, seed=2, lo=0.0, hi=1.0)
    di, dv = to_dev(t, cuda_device)
    inds_np, vals_np = t.numpy()
    Fo = [f.double().numpy() for f in F]
    for root in (0, 2):
        c = sptt.Csf(t.dims, di, dv, root)
        dflt = _modes(c, t, F, cuda_device, sched=(64, 256, 0))
        priv = _modes(c, t, F, cuda_device, sched=(64, 256, 2))
        glob = _modes(c, t, F, cuda_device, sched=(64, 256, 1))
        for m in range(3):
            _check(dflt[m], t, F, m, 16)
            _check(priv[m], t, F, m, 16)
            Mo, Ma = oracle.mttkrp(inds_np, vals_np, t.dims, Fo, m, with_abs=True)
            n = np.bincount(inds_np[m], minlength=dims[m]).astype(np.float64)[:, None]
            assert np.all(np.abs(glob[m] - Mo) <= np.maximum(1e-5, 8 * np.sqrt(n) * 2.0 ** -24) * Ma + 1e-30)


def test_more_hot_rows_than_fit(cuda_device):
    # ld 128: 128 rows fit in the per-CTA table; 2000 rows have >= 64 contributions
    dims = (2000, 50, 40)
    t = make(dims, 120000, seed=7, dist="uniform")
    F = rand_factors(dims, 128, seed=5)
    di, dv = to_dev(t, cuda_device)
    c = sptt.Csf(t.dims, di, dv, 1)  # mode 0 is a leaf or middle level
    for m, M in enumerate(_modes(c, t, F, cuda_device)):
        _check(M, t, F, m, 128)


def test_root_mode_matches_root_kernel(cuda_device):
    dims = (300, 200, 100)
    t = make(dims, 30000, seed=1, dist="zipf")
    F = [f.to(cuda_device) for f in rand_factors(dims, 16, seed=1)]
    di, dv = to_dev(t, cuda_device)
    c = sptt.Csf(t.dims, di, dv, 1)
    a = c.mttkrp(F).cpu()
    b = c.mttkrp_mode(1, F).cpu()
    assert torch.allclose(a, b, rtol=1e-6, atol=1e-6)


def test_rejects_bad_arguments(cuda_device):
    dims = (10, 10, 10)
    t = make(dims, 100, seed=1)
    di, dv = to_dev(t, cuda_device)
    c = sptt.Csf(dims, di, dv, 0)
    F = [torch.rand(d, 8, device=cuda_device) for d in dims]
    out = torch.empty(10, 8, device=cuda_device)
    for mode, kw in ((3, {}), (-1, {}), (1, dict(sched=(64, 256, 3))), (1, dict(sched=(24, 256, 0))),
                     (1, dict(factor_dtype=7))):
        with pytest.raises(sptt.SpttError):
            c.mttkrp_mode(mode, F, out=out, **kw)
