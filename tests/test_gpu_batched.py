"""Batched CP-ALS (one persistent launch for many tensors) against the oracle
and the single-tensor path; graph replay; the bounded grid barrier."""
import numpy as np
import pytest
import torch

import oracle
import paper_1812_05961_gb300 as sptt
import tensorgen

pytestmark = pytest.mark.gpu


def _batch(count, seed, dim_hi=300, nnz_hi=6000, dev="cuda"):
    g = torch.Generator().manual_seed(seed)
    out = []
    for t in range(count):
        n = 3 if torch.rand(1, generator=g).item() < 0.5 else 4
        dims = [int(torch.randint(8, dim_hi, (1,), generator=g)) for _ in range(n)]
        space = int(np.prod(dims))
        nnz = min(int(torch.randint(50, nnz_hi, (1,), generator=g)), space // 2)
        x = tensorgen.batch_member(dims, max(nnz, 1), seed=seed * 1000 + t)
        out.append((dims, [i.to(dev) for i in x.inds], x.vals.to(dev), x))
    return out


def test_batched_fits_match_oracle_per_tensor(cuda_device):
    items = _batch(24, seed=3)
    R, iters = 8, 5
    b = sptt.Batch([(d, i, v) for d, i, v, _ in items], R, seed=100).init()
    b.run(iters)
    for t, (dims, _, _, x) in enumerate(items):
        inds_np, vals_np = x.numpy()
        ref = oracle.cpd_als(inds_np, vals_np, dims, R, iters, seed=100 + t)
        np.testing.assert_allclose(b.fit_history(t), ref["fits"], atol=1e-4, err_msg="tensor %d" % t)
    for t in (0, 7):
        dims, _, _, x = items[t]
        inds_np, vals_np = x.numpy()
        ref = oracle.cpd_als(inds_np, vals_np, dims, R, iters, seed=100 + t)
        for m in range(len(dims)):
            F = b.factor(t, m).numpy()
            assert np.linalg.norm(F - ref["factors"][m]) <= 1e-3 * max(1.0, np.linalg.norm(ref["factors"][m]))


@pytest.mark.parametrize("R", [8, 16])
def test_autotuned_batch_fits_match_oracle_per_tensor(R, cuda_device):
    # plan 1: the batch times its walk x chunk candidates on itself, keeps the
    # fastest and must still give every tensor the oracle's fits
    items = _batch(24, seed=13)
    iters = 5
    b = sptt.Batch([(d, i, v) for d, i, v, _ in items], R, seed=100, plan=1).init()
    (chunk, _, variant, _), ms, n = b.schedule()
    assert n >= 3 and ms > 0 and chunk in (64, 128, 256) and variant in (4, 7)
    b.run(iters)
    for t, (dims, _, _, x) in enumerate(items):
        inds_np, vals_np = x.numpy()
        ref = oracle.cpd_als(inds_np, vals_np, dims, R, iters, seed=100 + t)
        np.testing.assert_allclose(b.fit_history(t), ref["fits"], atol=1e-4, err_msg="tensor %d" % t)


def test_batched_matches_single_tensor_path_and_continues(cuda_device):
    items = _batch(10, seed=5)
    R = 16
    b = sptt.Batch([(d, i, v) for d, i, v, _ in items], R, seed=7).init()
    b.run(3)
    b.run(2)  # a second launch continues from the factors of the first
    for t, (dims, inds, vals, _) in enumerate(items):
        c = sptt.Cpd(dims, inds, vals, R, seed=7 + t).init()
        c.iterate(5)
        np.testing.assert_allclose(b.fit_history(t), c.fit_history(), atol=1e-6)
        np.testing.assert_allclose(b.lam(t).numpy(), c.lam().numpy(), rtol=1e-4)


@pytest.mark.parametrize("R", [16, 24])
def test_batched_large_skewed_tensors_match_single_path(R, cuda_device):
    # tensors of many solve tiles and many chunks, with power-law slices
    # that span CTAs, next to tiny ones; R = 24 takes the 32-wide kernel
    specs = [((6000, 900, 300), 250000, 1.3), ((40, 30, 20), 500, 1.0), ((12000, 500, 80, 30), 180000, 1.2),
             ((3000, 2000, 1000), 120000, 1.1), ((50, 5000, 60), 90000, 1.4)]
    items = []
    for k, (dims, nnz, s_) in enumerate(specs):
        x = tensorgen.sample_unique(list(dims), nnz, 40 + k, "cpu", dist="zipf", s=s_, values="uniform")
        items.append((list(dims), [i.to(cuda_device) for i in x.inds], x.vals.to(cuda_device)))
    b = sptt.Batch(items, R, seed=11).init()
    b.run(4)
    for t, (dims, inds, vals) in enumerate(items):
        c = sptt.Cpd(dims, inds, vals, R, seed=11 + t).init()
        c.iterate(4)
        np.testing.assert_allclose(b.fit_history(t), c.fit_history(), atol=1e-5, err_msg="tensor %d" % t)
        for m in range(len(dims)):
            Fb, Fc = b.factor(t, m), c.factor(m)
            assert torch.linalg.norm(Fb - Fc) <= 1e-3 * max(1.0, float(torch.linalg.norm(Fc)))


def test_batched_record_sources_agree(cuda_device):
    # the batched MTTKRP walks - 32-byte rows on packed leaf records in the
    # 1-CTA-per-SM kernel (the default at R = 16), 16-byte rows on packed
    # records (schedule variant 4) and on the separate leaf arrays (variant
    # 3) - add the same products in the same order per output element; only
    # the order of the split-slice atomics differs
    items = _batch(16, seed=13, dim_hi=2000, nnz_hi=40000)
    R = 16
    runs = []
    for sched in (None, (0, 0, 4, 0), (0, 0, 3, 0)):
        kw = {} if sched is None else {"sched": sched}
        b = sptt.Batch([(d, i, v) for d, i, v, _ in items], R, seed=21, **kw).init()
        b.run(4)
        runs.append(b)
    assert runs[0].info()[0] * 2 == runs[1].info()[0] == runs[2].info()[0]  # 1 against 2 CTAs per SM
    for other in runs[1:]:
        for t in range(len(items)):
            np.testing.assert_allclose(runs[0].fit_history(t), other.fit_history(t), atol=1e-6,
                                       err_msg="tensor %d" % t)
            for m in range(len(items[t][0])):
                Fa, Fb = runs[0].factor(t, m), other.factor(t, m)
                assert torch.linalg.norm(Fa - Fb) <= 1e-4 * max(1.0, float(torch.linalg.norm(Fb)))


def test_batched_graph_replay(cuda_device):
    items = _batch(12, seed=9)
    R = 8
    ref = sptt.Batch([(d, i, v) for d, i, v, _ in items], R, seed=1).init()
    ref.run(4)
    ref.run(4)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = sptt.Batch([(d, i, v) for d, i, v, _ in items], R, seed=1, use_graph=1).init()
        g.run(4)   # first run: direct launch
        g.run(4)   # captured, then replayed
        l0 = sptt.sptt_debug_launch_count()
        g.run(4)
        assert sptt.sptt_debug_launch_count() - l0 == 3
    for t in range(len(items)):
        np.testing.assert_allclose(g.fit_history(t)[:8], ref.fit_history(t), atol=1e-6)


def test_batched_barrier_timeout_is_reported_and_recoverable(cuda_device):
    items = _batch(6, seed=11)
    R = 8
    b = sptt.Batch([(d, i, v) for d, i, v, _ in items], R, seed=4).init()
    grid, _, _ = b.info()
    assert grid >= 2
    sptt.sptt_debug_batch_stall(b.handle, 1, 50_000_000)  # CTA 1 never arrives; waits end after 50 ms
    with pytest.raises(sptt.SpttError) as e:
        b.run(2)
    assert e.value.status == sptt.SPTT_ERR_TIMEOUT
    sptt.sptt_debug_batch_stall(b.handle, -1, 0)
    b.init()
    b.run(3)
    for t, (dims, _, _, x) in enumerate(items):
        inds_np, vals_np = x.numpy()
        ref = oracle.cpd_als(inds_np, vals_np, dims, R, 3, seed=4 + t)
        np.testing.assert_allclose(b.fit_history(t), ref["fits"], atol=1e-4)


def test_batched_rejects_unsupported(cuda_device):
    items = _batch(2, seed=2)
    with pytest.raises(sptt.SpttError) as e:
        sptt.Batch([(d, i, v) for d, i, v, _ in items], 33)
    assert e.value.status == sptt.SPTT_ERR_UNSUPPORTED
    x = tensorgen.sample_unique([5, 4, 3, 3, 2], 50, seed=1)
    with pytest.raises(sptt.SpttError) as e:
        sptt.Batch([(x.dims, [i.cuda() for i in x.inds], x.vals.cuda())], 8)
    assert e.value.status == sptt.SPTT_ERR_UNSUPPORTED


def test_batched_rejects_a_chunk_that_is_not_a_power_of_two(cuda_device):
    # the walk's batches tile a chunk exactly: power-of-two chunks of at least 16 leaves
    items = _batch(2, seed=3)
    for chunk in (100, 8, 8192):
        with pytest.raises(sptt.SpttError) as e:
            sptt.Batch([(d, i, v) for d, i, v, _ in items], 8, sched=(chunk, 256, 4, 0))
        assert e.value.status == sptt.SPTT_ERR_BAD_ARG, chunk
