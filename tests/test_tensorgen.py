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
