"""GPU CP-ALS (Algorithm 1) against the oracle: |delta fit| <= 1e-4 per
iteration, matching initial factors, solve branches, error paths."""
import numpy as np
import pytest
import torch

import oracle
import paper_1812_05961_gb300 as sptt
from gpu_util import make, rel_fro, to_dev

pytestmark = pytest.mark.gpu


def test_philox_init_matches_oracle_bit_for_bit(cuda_device):
    t = make((37, 23, 11), 500, seed=1)
    di, dv = to_dev(t, cuda_device)
    for R in (1, 3, 8, 13):
        cpd = sptt.Cpd(t.dims, di, dv, R, seed=12345).init()
        for m, d in enumerate(t.dims):
            got = cpd.factor(m).numpy()  # factors are not normalised before the first iteration
            want = oracle.init_factor(12345, m, d, R).astype(np.float32)
            np.testing.assert_array_equal(got, want)


def test_gram_matches_numpy(cuda_device):
    g = torch.Generator().manual_seed(0)
    for rows, R, ld in ((1000, 8, 8), (777, 13, 16), (5000, 64, 64), (3, 32, 32), (0, 4, 4)):
        A = torch.rand(rows, ld, generator=g) - 0.5
        G = sptt.sptt_gram(A.to(cuda_device), R).cpu().numpy()
        ref = A[:, :R].double().numpy()
        ref = ref.T @ ref
        assert np.abs(G - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("dims,nnz,R,iters,dist", [
    # the small uniform workload: 200 x 150 x 100, 20,000 distinct uniform
    # coordinates, values U(0,1), R = 8, 10 iterations
    ((200, 150, 100), 20000, 8, 10, "uniform"),
    ((200, 150, 100), 20000, 8, 10, "zipf"),
    ((300, 250, 200), 40000, 16, 6, "zipf"),
    ((60, 50, 40, 30), 30000, 12, 6, "uniform"),
    ((20, 18, 16, 14, 12), 20000, 8, 5, "uniform"),
    ((400, 300), 20000, 10, 6, "uniform"),
])
def test_cpd_als_fit_matches_oracle(dims, nnz, R, iters, dist, cuda_device):
    t = make(dims, nnz, seed=nnz % 101 + R, dist=dist, s=1.1)
    inds_np, vals_np = t.numpy()
    di, dv = to_dev(t, cuda_device)
    cpd = sptt.Cpd(dims, di, dv, R, seed=7).init()
    cpd.iterate(iters)
    fits = cpd.fit_history()
    ref = oracle.cpd_als(inds_np, vals_np, dims, R, iters, seed=7)
    assert len(fits) == iters
    np.testing.assert_allclose(fits, ref["fits"], atol=1e-4, rtol=0)
    assert cpd.solve_branch() == (0, iters * len(dims))


def test_first_iteration_factors_match_oracle(cuda_device):
    dims = (120, 90, 70)
    t = make(dims, 15000, seed=3)
    inds_np, vals_np = t.numpy()
    di, dv = to_dev(t, cuda_device)
    R = 10
    cpd = sptt.Cpd(dims, di, dv, R, seed=99).init()
    cpd.iterate(1)
    ref = oracle.cpd_als(inds_np, vals_np, dims, R, 1, seed=99)
    for m in range(3):
        assert rel_fro(cpd.factor(m).numpy(), ref["factors"][m]) < 1e-4
        G = cpd.gram(m).numpy()
        Gr = ref["factors"][m].T @ ref["factors"][m]
        assert np.abs(G - Gr).max() < 1e-4
    np.testing.assert_allclose(cpd.lam().numpy(), ref["lam"], rtol=1e-4)


def test_explicit_init_and_one_shot(cuda_device):
    dims = (80, 60, 40)
    t = make(dims, 8000, seed=8)
    inds_np, vals_np = t.numpy()
    R = 6
    g = torch.Generator().manual_seed(1)
    init = [torch.rand(d, R, generator=g) for d in dims]
    di, dv = to_dev(t, cuda_device)
    cpd = sptt.Cpd(dims, di, dv, R).init(init)
    cpd.iterate(4)
    ref = oracle.cpd_als(inds_np, vals_np, dims, R, 4, init=[x.double().numpy() for x in init])
    np.testing.assert_allclose(cpd.fit_history(), ref["fits"], atol=1e-4)
    # one-shot call with host inputs and host outputs
    outs = [torch.empty(d, R) for d in dims]
    lam = torch.empty(R, dtype=torch.float64)
    fit, iters = sptt.sptt_cpd_als(dims, t.inds, t.vals, R, 4, factors_out=outs, lambda_out=lam, seed=0)
    ref0 = oracle.cpd_als(inds_np, vals_np, dims, R, 4, seed=0)
    assert iters == 4 and abs(fit - ref0["fits"][-1]) < 1e-4
    for m in range(3):
        assert rel_fro(outs[m].numpy(), ref0["factors"][m]) < 1e-3


def test_exact_recovery_fp32(cuda_device):
    rng = np.random.default_rng(101)
    dims = (10, 9, 8)
    fac = []
    for d in dims:
        Q, _ = np.linalg.qr(rng.standard_normal((d, 3)))
        fac.append(Q + 0.1)
    X = np.einsum("r,ir,jr,kr->ijk", np.array([3.0, 2.0, 1.5]), *fac).astype(np.float32)
    coords = np.indices(dims).reshape(3, -1)
    inds = [torch.from_numpy(c.astype(np.int32)).to(cuda_device) for c in coords]
    vals = torch.from_numpy(X.reshape(-1)).to(cuda_device)
    fit, iters = sptt.sptt_cpd_als(dims, inds, vals, 3, 500, tol=1e-10, seed=1)
    assert fit >= 1 - 1e-5, fit


def test_tol_stops_like_oracle(cuda_device):
    dims = (50, 40, 30)
    t = make(dims, 5000, seed=2)
    inds_np, vals_np = t.numpy()
    di, dv = to_dev(t, cuda_device)
    cpd = sptt.Cpd(dims, di, dv, 5, seed=3).init()
    done = cpd.iterate(200, tol=1e-3)
    ref = oracle.cpd_als(inds_np, vals_np, dims, 5, 200, tol=1e-3, seed=3)
    assert abs(done - ref["iters"]) <= 1
    assert done < 200


def test_pseudo_inverse_branch(cuda_device):
    # a zero column in one initial factor makes V singular for the other modes
    dims = (30, 25, 20)
    t = make(dims, 3000, seed=4)
    inds_np, vals_np = t.numpy()
    R = 4
    g = torch.Generator().manual_seed(2)
    init = [torch.rand(d, R, generator=g) for d in dims]
    init[2][:, 1] = 0.0
    di, dv = to_dev(t, cuda_device)
    cpd = sptt.Cpd(dims, di, dv, R).init(init)
    cpd.iterate(3)
    ref = oracle.cpd_als(inds_np, vals_np, dims, R, 3, init=[x.double().numpy() for x in init])
    npinv, ntot = cpd.solve_branch()
    assert npinv > 0 and ntot == 9
    np.testing.assert_allclose(cpd.fit_history(), ref["fits"], atol=1e-4)


def test_rank_larger_than_mode(cuda_device):
    dims = (6, 40, 30)
    t = make(dims, 2000, seed=6)
    inds_np, vals_np = t.numpy()
    di, dv = to_dev(t, cuda_device)
    cpd = sptt.Cpd(dims, di, dv, 9, seed=4).init()
    cpd.iterate(3)
    ref = oracle.cpd_als(inds_np, vals_np, dims, 9, 3, seed=4)
    np.testing.assert_allclose(cpd.fit_history(), ref["fits"], atol=1e-4)


def test_error_paths(cuda_device):
    dims = (10, 10, 10)
    t = make(dims, 100, seed=1)
    di, dv = to_dev(t, cuda_device)
    with pytest.raises(sptt.SpttError) as e:
        sptt.Cpd(dims, di, dv, 65)
    assert e.value.status == sptt.SPTT_ERR_UNSUPPORTED
    with pytest.raises(sptt.SpttError) as e:
        sptt.Cpd(dims, di, dv, 0)
    assert e.value.status == sptt.SPTT_ERR_BAD_ARG
    z = torch.zeros(0, dtype=torch.int32, device=cuda_device)
    with pytest.raises(sptt.SpttError):
        sptt.Cpd(dims, [z, z, z], torch.zeros(0, device=cuda_device), 4)
    # an injected allocation failure surfaces as OOM and leaves the library usable
    for k in (1, 3, 7, 20):
        sptt.sptt_debug_fail_alloc_after(k)
        try:
            with pytest.raises(sptt.SpttError) as e:
                sptt.Cpd(dims, di, dv, 4, seed=1).init().iterate(2)
            assert e.value.status == sptt.SPTT_ERR_OOM
        finally:
            sptt.sptt_debug_fail_alloc_after(0)
    cpd = sptt.Cpd(dims, di, dv, 4, seed=1).init()
    cpd.iterate(2)
    assert 0.0 < cpd.fit()[0] <= 1.0


def test_profile_timers(cuda_device):
    dims = (100, 80, 60)
    t = make(dims, 5000, seed=2)
    di, dv = to_dev(t, cuda_device)
    cpd = sptt.Cpd(dims, di, dv, 8, seed=1, profile=1).init()
    cpd.iterate(3)
    tm = cpd.timers()
    assert tm["mttkrp"][1] == 9 and tm["cpd_fit"][1] == 3
    assert all(v[0] > 0 for v in tm.values())


def test_graph_replay_matches_stream_launches(cuda_device):
    dims = (150, 120, 90, 40)
    t = make(dims, 30000, seed=12)
    di, dv = to_dev(t, cuda_device)
    a = sptt.Cpd(dims, di, dv, 12, seed=2).init()
    b = sptt.Cpd(dims, di, dv, 12, seed=2, use_graph=1).init()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):  # graphs need a non-default stream
        c = sptt.Cpd(dims, di, dv, 12, seed=2, use_graph=1).init()
        l0 = sptt.sptt_debug_launch_count()
        c.iterate(5)
        l1 = sptt.sptt_debug_launch_count()
    a.iterate(5)
    b.iterate(5)
    fa, fc = a.fit_history(), c.fit_history()
    np.testing.assert_allclose(fc, fa, atol=1e-9)
    np.testing.assert_allclose(b.fit_history(), fa, atol=1e-9)
    assert l1 - l0 >= 5 * (4 * 6 + 1)  # every replayed kernel is counted


@pytest.mark.parametrize("csf_mode", [1, 2])
@pytest.mark.parametrize("dims,nnz,R,iters", [
    ((200, 150, 100), 20000, 8, 6),
    ((60, 50, 40, 30), 30000, 12, 5),
    ((20, 18, 16, 14, 12), 20000, 8, 4),
    ((400, 300), 20000, 10, 5),
])
def test_one_csf_for_all_modes_matches_oracle(csf_mode, dims, nnz, R, iters, cuda_device):
    # the non-root modes' MTTKRPs from the one CSF (sptt_mttkrp_mode's kernels)
    t = make(dims, nnz, seed=nnz % 97 + R, dist="zipf", s=1.2)
    inds_np, vals_np = t.numpy()
    di, dv = to_dev(t, cuda_device)
    one = sptt.Cpd(dims, di, dv, R, seed=5, csf_mode=csf_mode).init()
    one.iterate(iters)
    per_mode = sptt.Cpd(dims, di, dv, R, seed=5).init()
    per_mode.iterate(iters)
    ref = oracle.cpd_als(inds_np, vals_np, dims, R, iters, seed=5)
    np.testing.assert_allclose(one.fit_history(), ref["fits"], atol=1e-4, rtol=0)
    np.testing.assert_allclose(one.fit_history(), per_mode.fit_history(), atol=1e-5, rtol=0)


def test_one_csf_graph_and_bf16(cuda_device):
    dims = (150, 120, 90, 40)
    t = make(dims, 30000, seed=21, dist="zipf", s=1.3)
    di, dv = to_dev(t, cuda_device)
    a = sptt.Cpd(dims, di, dv, 16, seed=3, csf_mode=1).init()
    a.iterate(4)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = sptt.Cpd(dims, di, dv, 16, seed=3, csf_mode=1, use_graph=1).init()
        g.iterate(4)
    torch.cuda.synchronize()
    np.testing.assert_allclose(g.fit_history(), a.fit_history(), atol=1e-6)
    b = sptt.Cpd(dims, di, dv, 16, seed=3, csf_mode=1, precision=sptt.SPTT_BF16).init()
    b.iterate(4)
    b.refine(1)
    c = sptt.Cpd(dims, di, dv, 16, seed=3, precision=sptt.SPTT_BF16).init()
    c.iterate(4)
    c.refine(1)
    assert abs(b.fit()[0] - c.fit()[0]) <= 1e-4
    with pytest.raises(sptt.SpttError):
        sptt.Cpd(dims, di, dv, 16, seed=3, csf_mode=1, plan=1)
