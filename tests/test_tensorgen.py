"""The seeded input generators: determinism, uniqueness, ranges, skew."""
import numpy as np
import torch

import tensorgen


def _keys(t):
    c = np.stack([x.numpy().astype(np.int64) for x in t.inds], 1)
    return [tuple(r) for r in c]


def test_uniform_unique_is_deterministic_and_distinct():
    a = tensorgen.sample_unique([20, 15, 10], 1500, seed=5)
    b = tensorgen.sample_unique([20, 15, 10], 1500, seed=5)
    c = tensorgen.sample_unique([20, 15, 10], 1500, seed=6)
    for x, y in zip(a.inds, b.inds):
        assert torch.equal(x, y)
    assert torch.equal(a.vals, b.vals)
    assert not all(torch.equal(x, y) for x, y in zip(a.inds, c.inds))
    k = _keys(a)
    assert len(set(k)) == 1500
    for m, d in enumerate(a.dims):
        assert a.inds[m].dtype == torch.int32
        assert int(a.inds[m].min()) >= 0 and int(a.inds[m].max()) < d
    assert a.vals.dtype == torch.float32 and float(a.vals.min()) >= 0 and float(a.vals.max()) < 1
    # not handed over in sorted order
    assert k != sorted(k)


def test_zipf_is_skewed_and_wide_keys_work():
    # 4 modes whose index space exceeds 2^63 (two key words)
    dims = [2_000_000, 500_000, 50_000, 1_000]
    t = tensorgen.sample_unique(dims, 20000, seed=3, dist="zipf", s=1.2, values="uniform")
    assert len(set(_keys(t))) == 20000
    counts = np.bincount(t.inds[3].numpy(), minlength=1000)
    top = np.sort(counts)[::-1]
    assert top[:10].sum() > 0.2 * counts.sum()     # heavy head
    assert (counts > 0).sum() > 100                # but a long tail too


def test_full_space_and_duplicates():
    t = tensorgen.sample_unique([3, 2, 2], 12, seed=1)
    assert sorted(_keys(t)) == [(i, j, k) for i in range(3) for j in range(2) for k in range(2)]
    d = tensorgen.sample_with_duplicates([5, 4, 3], 200, seed=2)
    assert len(set(_keys(d))) < 200


def test_batch_specs():
    specs = tensorgen.batch_tensor_specs(64, seed=4)
    assert len(specs) == 64
    for dims, nnz in specs:
        assert len(dims) in (3, 4)
        assert all(100 <= d <= 200_000 for d in dims)
        assert 1 <= nnz <= 2_000_000
    t = tensorgen.batch_member(specs[0][0], min(specs[0][1], 3000), seed=9)
    assert len(set(_keys(t))) == t.nnz


def test_scheduler_specs_follow_the_log_uniform_law_in_two_strata():
    # the training draw: tensor k of a stratum is the same whatever the count,
    # the strata split n in the law's proportion, every nnz is inside its
    # stratum's range (or capped at a quarter of the index space)
    from paper_1812_05961_gb300 import train_scheduler as ts
    lo, hi, split = 1e5, 2e8, 2e7
    below, above = ts.strata(2000, lo, hi, split)
    assert (below, above) == (1394, 606)
    assert ts.strata(10, lo, hi, 1e9) == (10, 0) and ts.strata(10, lo, hi, 1.0) == (0, 10)
    a = ts.tensor_specs(50, 21, split, lo)
    assert ts.tensor_specs(20, 21, split, lo) == a[:20]
    specs = ts.specs_for(200, 77, lo, hi, split)
    assert len(specs) == 200
    for k, (dims, nnz, s, R, seed) in enumerate(specs):
        space = 1.0
        for d in dims:
            space *= d
        top = split if k < 139 else hi
        bot = lo if k < 139 else split
        assert 3 <= len(dims) <= 5 and R in (8, 16, 32, 64) and 0.8 <= s <= 1.5
        assert nnz <= top and (nnz >= bot or nnz >= min(space / 4, bot) - 1 or nnz == 1000)


def test_zipf_table_is_built_on_the_host():
    # the same table whatever the device it is asked for (a fixed-order sum)
    t = tensorgen._zipf_table(1000, 1.1, "cpu")
    assert t.dtype == torch.float64 and t[-1] == 1.0 and bool((t[1:] >= t[:-1]).all())
