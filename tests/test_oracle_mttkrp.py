"""Pins for the oracle's MTTKRP (Section III) and its generator.

Each check is chosen so that a plausible slip in the oracle (a dropped factor,
a wrong index, the root factor multiplied in, a transposed operand) fails at
least one of them:
  * brute force: explicit mode-n unfolding X_(n) times an explicit Khatri-Rao
    matrix, both built by their textbook definitions (Kolda & Bader 2009);
  * the rank-1 closed form M = a * ((b^T B) .* (c^T C));
  * linearity in the tensor and in each factor;
  * all-ones factors give the row sums of the unfolding;
  * the Philox stream against numpy's independent Philox4x64-10.
"""
import numpy as np
import pytest

import oracle


def _dense_to_coo(X):
    idx = np.nonzero(X)
    return [i.astype(np.int32) for i in idx], X[idx].astype(np.float32)


def _unfold(X, n):
    """Mode-n unfolding with the first remaining index varying fastest."""
    return np.moveaxis(X, n, 0).reshape(X.shape[n], -1, order="F")


def _khatri_rao(mats):
    """Column-wise Kronecker product of mats[0] (slowest) ... mats[-1] (fastest)."""
    R = mats[0].shape[1]
    cols = []
    for r in range(R):
        c = np.array([1.0])
        for A in mats:
            c = np.kron(c, A[:, r])
        cols.append(c)
    return np.stack(cols, 1)


def _krp_for_mode(factors, n):
    # X_(n) columns put the lowest remaining mode fastest, so the Khatri-Rao
    # product runs from the highest remaining mode down to the lowest.
    others = [factors[m] for m in reversed(range(len(factors))) if m != n]
    return _khatri_rao(others)


@pytest.mark.parametrize("dims", [(6, 5, 4), (4, 4, 4, 4), (3, 2, 4, 2, 3), (1, 5, 3)])
@pytest.mark.parametrize("density", [1.0, 0.35])
def test_mttkrp_matches_unfolding_times_khatri_rao(dims, density):
    rng = np.random.default_rng(hash((dims, density)) % 2**32)
    X = rng.standard_normal(dims).astype(np.float32)
    X[rng.random(dims) > density] = 0.0
    inds, vals = _dense_to_coo(X)
    R = 5
    factors = [rng.standard_normal((d, R)) for d in dims]
    for n in range(len(dims)):
        want = _unfold(X.astype(np.float64), n) @ _krp_for_mode(factors, n)
        got = oracle.mttkrp(inds, vals, dims, factors, n)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


def test_mttkrp_rank1_closed_form():
    rng = np.random.default_rng(7)
    a, b, c = rng.random(6), rng.random(5), rng.random(4)
    X = np.einsum("i,j,k->ijk", a, b, c).astype(np.float32)
    inds, vals = _dense_to_coo(X)
    R = 3
    B, C = rng.random((5, R)), rng.random((4, R))
    got = oracle.mttkrp(inds, vals, X.shape, [None, B, C], 0)
    # X was rounded to float32, so compare against the closed form of that X
    want = np.outer(a, (b @ B) * (c @ C))
    np.testing.assert_allclose(got, want, rtol=2e-7)
    X64 = X.astype(np.float64)
    exact = np.einsum("ijk,jr,kr->ir", X64, B, C)
    np.testing.assert_allclose(got, exact, rtol=1e-12)


def test_mttkrp_linearity():
    rng = np.random.default_rng(11)
    dims = (7, 6, 5, 3)
    R = 4

    def rand_coo(n):
        return ([rng.integers(0, d, n).astype(np.int32) for d in dims],
                rng.standard_normal(n).astype(np.float32))

    i1, v1 = rand_coo(60)
    i2, v2 = rand_coo(45)
    F = [rng.standard_normal((d, R)) for d in dims]
    for n in range(4):
        m1 = oracle.mttkrp(i1, v1, dims, F, n)
        m2 = oracle.mttkrp(i2, v2, dims, F, n)
        m12 = oracle.mttkrp([np.concatenate([a, b]) for a, b in zip(i1, i2)],
                            np.concatenate([v1, v2]), dims, F, n)
        np.testing.assert_allclose(m12, m1 + m2, rtol=1e-12, atol=1e-12)
        for m in range(4):
            if m == n:
                continue
            G = [f.copy() for f in F]
            G[m] = rng.standard_normal((dims[m], R))
            H = [f.copy() for f in F]
            H[m] = 2.5 * F[m] - 0.5 * G[m]
            mF = oracle.mttkrp(i1, v1, dims, F, n)
            mG = oracle.mttkrp(i1, v1, dims, G, n)
            mH = oracle.mttkrp(i1, v1, dims, H, n)
            np.testing.assert_allclose(mH, 2.5 * mF - 0.5 * mG, rtol=1e-10, atol=1e-10)


def test_mttkrp_all_ones_factors_give_row_sums():
    rng = np.random.default_rng(3)
    dims = (9, 8, 7)
    X = rng.random(dims).astype(np.float32)
    X[X < 0.6] = 0
    inds, vals = _dense_to_coo(X)
    R = 3
    F = [np.ones((d, R)) for d in dims]
    for n in range(3):
        rows = _unfold(X.astype(np.float64), n).sum(1)
        got = oracle.mttkrp(inds, vals, dims, F, n)
        for r in range(R):
            np.testing.assert_allclose(got[:, r], rows, rtol=1e-12)


def test_mttkrp_root_factor_is_ignored_and_rows_mask():
    rng = np.random.default_rng(5)
    dims = (10, 6, 4)
    inds = [rng.integers(0, d, 50).astype(np.int32) for d in dims]
    vals = rng.random(50).astype(np.float32)
    F = [rng.random((d, 2)) for d in dims]
    G = [f.copy() for f in F]
    G[0] = rng.random((10, 2)) * 100
    full = oracle.mttkrp(inds, vals, dims, F, 0)
    np.testing.assert_array_equal(full, oracle.mttkrp(inds, vals, dims, G, 0))
    rows = [1, 4, 7]
    part = oracle.mttkrp(inds, vals, dims, F, 0, rows=rows)
    np.testing.assert_array_equal(part[rows], full[rows])
    others = np.setdiff1d(np.arange(10), rows)
    assert not part[others].any()


def test_mttkrp_abs_bounds_value():
    rng = np.random.default_rng(9)
    dims = (5, 6, 7)
    inds = [rng.integers(0, d, 80).astype(np.int32) for d in dims]
    vals = rng.standard_normal(80).astype(np.float32)
    F = [rng.standard_normal((d, 3)) for d in dims]
    M, Ma = oracle.mttkrp(inds, vals, dims, F, 1, with_abs=True)
    assert np.all(np.abs(M) <= Ma * (1 + 1e-12) + 1e-300)
    Fa = [np.abs(f) for f in F]
    np.testing.assert_allclose(Ma, oracle.mttkrp(inds, np.abs(vals), dims, Fa, 1), rtol=1e-12)


def test_philox_matches_numpy_philox4x64():
    # numpy's Philox(counter=c) emits philox(c + 1) first (it increments the
    # counter before each block), an independent implementation of the same
    # published generator.
    for key in ([0, 0], [7, 9], [2**64 - 1, 12345]):
        for c0 in (0, 5, 2**40 + 3):
            bg = np.random.Philox(counter=np.array([c0, 0, 0, 0], np.uint64),
                                  key=np.array(key, np.uint64))
            want = bg.random_raw(4)
            got = oracle.philox4x64([(c0 + 1) % 2**64, 0, 0, 0], key)
            np.testing.assert_array_equal(got, want)


def test_init_factor_is_u01_from_stream():
    A = oracle.init_factor(42, 1, 50, 7)
    assert A.shape == (50, 7)
    assert np.all(A > 0) and np.all(A < 1)
    # element e uses word e % 4 of philox((e // 4, 0, 0, 0), (seed, mode))
    for e in (0, 3, 4, 17, 349):
        w = oracle.philox4x64([e // 4, 0, 0, 0], [42, 1])[e % 4]
        m = int(w) >> 41
        assert A.reshape(-1)[e] == (m + 0.5) / 2**23
    # float32-exact
    np.testing.assert_array_equal(A.astype(np.float32).astype(np.float64), A)
    assert abs(A.mean() - 0.5) < 0.06
    B = oracle.init_factor(42, 2, 50, 7)
    assert not np.array_equal(A, B)
