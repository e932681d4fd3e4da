"""GPU MTTKRP over CSF against the oracle's element definition (Section III).

Tolerances: FP32 gathers 1e-5 relative (Frobenius, and element-wise against
the scale sum |v| prod |A|); BF16 gathers 2e-2 relative against the FP32
factors and 1e-5 against the same BF16-rounded factors.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1812_05961_gb300 as sptt
from gpu_util import make, rand_factors, rel_fro, to_dev

pytestmark = pytest.mark.gpu


def _run(t, root, F, dev, dtype=sptt.SPTT_F32, sched=None, level_order=None):
    di, dv = to_dev(t, dev)
    c = sptt.Csf(t.dims, di, dv, root, level_order=level_order)
    tdt = torch.bfloat16 if dtype == sptt.SPTT_BF16 else torch.float32
    fd = [f.to(dev).to(tdt).contiguous() for f in F]
    ld = F[0].shape[1]
    out = torch.full((t.dims[root], ld), float("nan"), device=dev)  # must be overwritten
    c.mttkrp(fd, out=out, factor_dtype=dtype, sched=sched)
    return out.cpu().double().numpy()


def _check(M, t, F, root, R, tol):
    inds_np, vals_np = t.numpy()
    Fo = [f[:, :R].double().numpy() for f in F]
    Mo, Ma = oracle.mttkrp(inds_np, vals_np, t.dims, Fo, root, with_abs=True)
    assert rel_fro(M[:, :R], Mo) <= tol
    assert np.all(np.abs(M[:, :R] - Mo) <= tol * Ma + 1e-30)
    return Mo


@pytest.mark.parametrize("dims,nnz,dist", [
    ((200, 150, 100), 20000, "uniform"),
    ((500, 400, 300), 60000, "zipf"),
    ((60, 50, 40, 30), 40000, "zipf"),
    ((20, 18, 16, 14, 12), 30000, "uniform"),
    ((3000, 2500), 50000, "zipf"),
    ((1, 200, 100), 5000, "uniform"),
])
@pytest.mark.parametrize("ld", [4, 8, 16, 32, 64, 128])
def test_mttkrp_fp32_all_roots(dims, nnz, dist, ld, cuda_device):
    t = make(dims, nnz, seed=ld + len(dims), dist=dist, s=1.2)
    F = rand_factors(dims, ld, seed=ld)
    for root in range(len(dims)):
        M = _run(t, root, F, cuda_device)
        _check(M, t, F, root, ld, 1e-5)


@pytest.mark.parametrize("R,ld", [(1, 4), (5, 8), (35, 36), (35, 40), (61, 64)])
def test_mttkrp_padded_rank(R, ld, cuda_device):
    dims = (300, 200, 100)
    t = make(dims, 30000, seed=R, dist="zipf")
    F = rand_factors(dims, R, seed=R, ld=ld)
    for root in range(3):
        M = _run(t, root, F, cuda_device)
        _check(M, t, F, root, R, 1e-5)
        assert not M[:, R:].any()


@pytest.mark.parametrize("chunk", [16, 32, 128, 512, 4096])
@pytest.mark.parametrize("block", [64, 256])
@pytest.mark.parametrize("variant", list(range(16)))
def test_mttkrp_schedules_agree(chunk, block, variant, cuda_device):
    dims = (400, 300, 200, 20)
    t = make(dims, 50003, seed=5, dist="zipf", s=1.3)
    F = rand_factors(dims, 16, seed=1)
    for root in range(4):
        M = _run(t, root, F, cuda_device, sched=(chunk, block, variant))
        _check(M, t, F, root, 16, 1e-5)


@pytest.mark.parametrize("variant", list(range(16)))
@pytest.mark.parametrize("nm", [2, 3, 4, 5])
def test_mttkrp_variants_every_order(variant, nm, cuda_device):
    dims = (290, 170, 50, 30, 10)[:nm]
    t = make(dims, 20011, seed=nm, dist="zipf", s=1.2)
    for dtype, ld in ((sptt.SPTT_F32, 8), (sptt.SPTT_BF16, 16)):
        F = rand_factors(dims, ld, seed=nm + ld)
        if dtype == sptt.SPTT_BF16:
            F = [f.to(torch.bfloat16).float() for f in F]
        for root in range(nm):
            M = _run(t, root, F, cuda_device, dtype=dtype, sched=(64, 128, variant))
            _check(M, t, F, root, ld, 1e-5)


@pytest.mark.parametrize("ld", [8, 16, 32, 64])
def test_mttkrp_bf16_gathers(ld, cuda_device):
    dims = (300, 250, 200, 50)
    t = make(dims, 50000, seed=ld, dist="zipf", s=1.1)
    F = rand_factors(dims, ld, seed=ld, lo=0.0, hi=1.0)
    Fb = [f.to(torch.bfloat16).float() for f in F]  # the values the kernel gathers
    for root in range(4):
        M = _run(t, root, F, cuda_device, dtype=sptt.SPTT_BF16)
        _check(M, t, Fb, root, ld, 1e-5)
        inds_np, vals_np = t.numpy()
        Mo = oracle.mttkrp(inds_np, vals_np, dims, [f.double().numpy() for f in F], root)
        assert rel_fro(M, Mo) <= 2e-2


def test_mttkrp_heavy_single_slice(cuda_device):
    # one slice holding most non-zeros: split across many chunks + atomics
    dims = (50, 3000, 400)
    g = torch.Generator().manual_seed(9)
    n = 200000
    i = torch.where(torch.rand(n, generator=g) < 0.9, torch.zeros(n, dtype=torch.int64),
                    torch.randint(0, 50, (n,), generator=g))
    j = torch.randint(0, 3000, (n,), generator=g)
    k = torch.randint(0, 400, (n,), generator=g)
    import tensorgen
    t = tensorgen.CooTensor(list(dims), [i.int(), j.int(), k.int()], torch.rand(n, generator=g))
    F = rand_factors(dims, 16, seed=2, lo=0.0, hi=1.0)
    for root in range(3):
        M = _run(t, root, F, cuda_device)
        _check(M, t, F, root, 16, 1e-5)


@pytest.mark.parametrize("variant", [7, 8, 10, 12])
@pytest.mark.parametrize("dtype,ld", [(sptt.SPTT_F32, 4), (sptt.SPTT_F32, 12), (sptt.SPTT_F32, 24),
                                      (sptt.SPTT_F32, 64), (sptt.SPTT_F32, 128), (sptt.SPTT_BF16, 8),
                                      (sptt.SPTT_BF16, 24), (sptt.SPTT_BF16, 32), (sptt.SPTT_BF16, 256)])
def test_wide_segments_any_ld(variant, dtype, ld, cuda_device):
    # 32-byte segments where ld allows them (F32 ld % 8, BF16 ld % 16), the
    # 16-byte walk otherwise; the result is the same either way
    dims = (700, 300, 90)
    t = make(dims, 40000, seed=ld, dist="zipf", s=1.2)
    F = rand_factors(dims, ld, seed=ld + 1)
    if dtype == sptt.SPTT_BF16:
        F = [f.to(torch.bfloat16).float() for f in F]
    for root in range(3):
        M = _run(t, root, F, cuda_device, dtype=dtype, sched=(64, 256, variant))
        _check(M, t, F, root, ld, 1e-5)


@pytest.mark.parametrize("variant", [7, 8, 10, 12])
def test_wide_segments_misaligned_factor(variant, cuda_device):
    # a factor that is 16- but not 32-byte aligned runs the 16-byte walk
    dims = (500, 400, 60)
    t = make(dims, 30000, seed=2, dist="zipf", s=1.1)
    F = rand_factors(dims, 16, seed=4)
    di, dv = to_dev(t, cuda_device)
    c = sptt.Csf(dims, di, dv, 0)
    base = torch.zeros(dims[1] * 16 + 4, device=cuda_device)
    shifted = base[4:].view(dims[1], 16)
    shifted.copy_(F[1].to(cuda_device))
    assert shifted.data_ptr() % 32 == 16
    fd = [F[0].to(cuda_device), shifted, F[2].to(cuda_device)]
    M = c.mttkrp(fd, sched=(64, 256, variant)).cpu().double().numpy()
    _check(M, t, F, 0, 16, 1e-5)


def test_mttkrp_custom_level_order(cuda_device):
    dims = (100, 80, 60, 40)
    t = make(dims, 20000, seed=4)
    F = rand_factors(dims, 8, seed=3)
    for order in ([1, 0, 2, 3], [1, 3, 2, 0], [1, 2, 0, 3]):
        M = _run(t, 1, F, cuda_device, level_order=order)
        _check(M, t, F, 1, 8, 1e-5)


def test_mttkrp_rejects_bad_arguments(cuda_device):
    dims = (10, 10, 10)
    t = make(dims, 100, seed=1)
    di, dv = to_dev(t, cuda_device)
    c = sptt.Csf(dims, di, dv, 0)
    F = [torch.rand(d, 8, device=cuda_device) for d in dims]
    out = torch.empty(10, 8, device=cuda_device)
    for bad in (dict(sched=(24, 256, 0)), dict(sched=(64, 512, 0)), dict(sched=(64, 256, 16)),
                dict(factor_dtype=7)):
        with pytest.raises(sptt.SpttError):
            c.mttkrp(F, out=out, **bad)
    with pytest.raises(sptt.SpttError):  # ld 6 is not a multiple of 4
        c.mttkrp([torch.rand(d, 6, device=cuda_device) for d in dims],
                 out=torch.empty(10, 6, device=cuda_device))
    with pytest.raises(sptt.SpttError):  # BF16 needs ld % 8 == 0
        c.mttkrp([torch.rand(d, 4, device=cuda_device).bfloat16() for d in dims],
                 out=torch.empty(10, 4, device=cuda_device), factor_dtype=sptt.SPTT_BF16)


def test_staged_variant_reports_no_timeout_and_matches_default(cuda_device):
    dims = (3000, 900, 200)
    t = make(dims, 300000, seed=6, dist="zipf", s=1.3)
    di, dv = to_dev(t, cuda_device)
    c = sptt.Csf(dims, di, dv, 0)
    F = [torch.rand(d, 16, device=cuda_device) for d in dims]
    ref = c.mttkrp(F).clone()
    for variant in (6, 8, 6, 8):
        got = c.mttkrp(F, sched=(64, 256, variant, 0))
        assert sptt.lib().sptt_csf_check(c.handle, torch.cuda.current_stream().cuda_stream) == 0
        assert torch.allclose(got, ref, rtol=1e-5, atol=1e-5)
