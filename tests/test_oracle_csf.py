"""Pins for the oracle's sort/coalesce and CSF construction (Section III,
Section V-C "Sort").

  * a CSF worked out by hand for a 7-non-zero tensor;
  * expanding the CSF back to coordinates gives the coalesced, sorted COO;
  * structural invariants (fptr strictly increasing, last entry = child count,
    fids strictly increasing within a parent);
  * coalescing against a plain dictionary sum.
"""
import numpy as np
import pytest

import oracle


def test_csf_hand_worked_example():
    # Non-zeros (i, j, k) -> v, given unsorted; root mode 0, order (0, 1, 2)
    coords = [(2, 0, 1), (0, 1, 0), (0, 0, 3), (2, 0, 0), (0, 1, 2), (2, 2, 1), (0, 0, 1)]
    vals = np.array([1, 2, 3, 4, 5, 6, 7], np.float32)
    inds = [np.array([c[m] for c in coords], np.int32) for m in range(3)]
    dims = (3, 3, 4)
    c = oracle.csf(inds, vals, dims, root=0, order=[0, 1, 2])
    # sorted: (0,0,1)7 (0,0,3)3 (0,1,0)2 (0,1,2)5 (2,0,0)4 (2,0,1)1 (2,2,1)6
    # slices:  i=0 | i=2                  -> fids0 = [0, 2]
    # fibers:  (0,0) (0,1) | (2,0) (2,2)  -> fids1 = [0, 1, 0, 2], fptr0 = [0, 2, 4]
    # leaves:  k = 1 3 | 0 2 | 0 1 | 1    -> fptr1 = [0, 2, 4, 6, 7]
    assert c["nfibs"] == [2, 4, 7]
    np.testing.assert_array_equal(c["fids"][0], [0, 2])
    np.testing.assert_array_equal(c["fptr"][0], [0, 2, 4])
    np.testing.assert_array_equal(c["fids"][1], [0, 1, 0, 2])
    np.testing.assert_array_equal(c["fptr"][1], [0, 2, 4, 6, 7])
    np.testing.assert_array_equal(c["fids"][2], [1, 3, 0, 2, 0, 1, 1])
    np.testing.assert_array_equal(c["vals"], [7, 3, 2, 5, 4, 1, 6])
    # rooted at mode 2 with order (2, 0, 1)
    c2 = oracle.csf(inds, vals, dims, root=2, order=[2, 0, 1])
    # sorted by (k, i, j): (0:0,1)2 (0:2,0)4 | (1:0,0)7 (1:2,0)1 (1:2,2)6 | (2:0,1)5 | (3:0,0)3
    np.testing.assert_array_equal(c2["fids"][0], [0, 1, 2, 3])
    np.testing.assert_array_equal(c2["fptr"][0], [0, 2, 4, 5, 6])
    np.testing.assert_array_equal(c2["fids"][1], [0, 2, 0, 2, 0, 0])
    np.testing.assert_array_equal(c2["fptr"][1], [0, 1, 2, 3, 5, 6, 7])
    np.testing.assert_array_equal(c2["fids"][2], [1, 0, 0, 0, 2, 1, 0])
    np.testing.assert_array_equal(c2["vals"], [2, 4, 7, 1, 6, 5, 3])


def _expand(c):
    """CSF back to per-level coordinate columns, by walking the tree."""
    n = len(c["order"])
    nnz = c["nfibs"][-1]
    cols = [np.zeros(nnz, np.int64) for _ in range(n)]
    cols[n - 1][:] = c["fids"][n - 1]
    # owner at level l of each leaf
    owner = np.arange(nnz)
    for l in range(n - 2, -1, -1):
        fptr = c["fptr"][l]
        parent = np.searchsorted(fptr, owner, side="right") - 1
        cols[l][:] = c["fids"][l][parent]
        owner = parent
    return cols


def _check_invariants(c):
    n = len(c["order"])
    for l in range(n - 1):
        fptr = c["fptr"][l]
        assert fptr[0] == 0
        assert fptr[-1] == c["nfibs"][l + 1]
        assert np.all(np.diff(fptr) > 0), "every fiber has at least one child"
        child = c["fids"][l + 1]
        for f in range(c["nfibs"][l]):
            seg = child[fptr[f]:fptr[f + 1]]
            assert np.all(np.diff(seg) > 0)
    assert np.all(np.diff(c["fids"][0]) > 0)


@pytest.mark.parametrize("dims,nnz", [((12, 9, 7), 200), ((5, 6, 4, 3), 150), ((4, 3, 5, 2, 3), 90),
                                      ((1, 7, 1), 5), ((30, 1, 2), 40)])
@pytest.mark.parametrize("root", [0, 1, 2])
def test_csf_round_trip_and_invariants(dims, nnz, root):
    rng = np.random.default_rng(nnz + root)
    inds = [rng.integers(0, d, nnz).astype(np.int32) for d in dims]
    vals = rng.random(nnz).astype(np.float32)
    c = oracle.csf(inds, vals, dims, root=root)
    assert c["order"][0] == root
    _check_invariants(c)
    s_inds, s_vals = oracle.coalesce(inds, vals, dims, c["order"])
    cols = _expand(c)
    for l, m in enumerate(c["order"]):
        np.testing.assert_array_equal(cols[l], s_inds[m])
    np.testing.assert_array_equal(c["vals"], s_vals)


def test_default_order_ascending_length_ties_by_mode():
    assert oracle.default_order([50, 10, 30, 10], 0) == [0, 1, 3, 2]
    assert oracle.default_order([50, 10, 30, 10], 3) == [3, 1, 2, 0]


def test_coalesce_sums_duplicates_like_a_dictionary():
    rng = np.random.default_rng(21)
    dims = (4, 3, 5)
    n = 300
    inds = [rng.integers(0, d, n).astype(np.int32) for d in dims]
    vals = rng.standard_normal(n).astype(np.float32)
    acc = {}
    for k in range(n):
        key = tuple(int(inds[m][k]) for m in range(3))
        acc[key] = acc.get(key, 0.0) + float(vals[k])
    order = [1, 2, 0]
    s_inds, s_vals = oracle.coalesce(inds, vals, dims, order)
    keys = sorted(acc, key=lambda t: (t[1], t[2], t[0]))
    assert len(keys) == len(s_vals)
    for u, key in enumerate(keys):
        assert tuple(int(s_inds[m][u]) for m in range(3)) == key
        assert s_vals[u] == np.float32(acc[key])


def test_coalesce_rejects_out_of_range():
    with pytest.raises(ValueError):
        oracle.coalesce([np.array([0, 3], np.int32), np.array([0, 0], np.int32)],
                        np.ones(2, np.float32), (3, 1))


def test_csf_empty_tensor():
    c = oracle.csf([np.zeros(0, np.int32)] * 3, np.zeros(0, np.float32), (3, 4, 5), root=1)
    assert c["nfibs"] == [0, 0, 0]
    for f in c["fptr"]:
        np.testing.assert_array_equal(f, [0])
