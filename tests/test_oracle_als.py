"""Pins for the oracle's dense algebra and CP-ALS (Algorithm 1).

  * Gram, Cholesky, eigen and pseudo-inverse against numpy/LAPACK (an
    independent third implementation) and their defining residuals;
  * the normal-equation solve through its residual A V = M;
  * normalisation: unit columns, lambda = numpy column norms, zero columns;
  * the fit formula against an explicit dense |X - Xhat| on tiny tensors;
  * exact recovery of a fully observed rank-3 tensor (fit -> 1);
  * the residual never increases from one full iteration to the next.
"""
import numpy as np
import pytest

import oracle


def test_gram_matches_numpy():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((37, 6))
    np.testing.assert_allclose(oracle.gram(A), A.T @ A, rtol=1e-13, atol=1e-13)


def _spd(n, rng, cond=100.0):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    w = np.geomspace(1.0, 1.0 / cond, n)
    return (Q * w) @ Q.T


@pytest.mark.parametrize("n", [1, 3, 8, 33])
def test_cholesky_matches_lapack(n):
    rng = np.random.default_rng(n)
    V = _spd(n, rng)
    L = oracle.cholesky(V)
    assert L is not None
    np.testing.assert_allclose(L @ L.T, V, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(L, np.linalg.cholesky(V), rtol=1e-10, atol=1e-12)
    assert np.all(np.triu(L, 1) == 0)


def test_cholesky_rejects_singular_and_indefinite():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((5, 2))
    assert oracle.cholesky(x @ x.T) is None           # rank 2 PSD
    V = np.eye(3)
    V[2, 2] = -1
    assert oracle.cholesky(V) is None
    Z = np.zeros((4, 4))
    assert oracle.cholesky(Z) is None


def test_sym_eig_and_pinv_match_numpy():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((7, 4))
    V = x @ x.T  # rank 4 of 7
    w, Q = oracle.sym_eig(V)
    np.testing.assert_allclose((Q * w) @ Q.T, V, atol=1e-11)
    np.testing.assert_allclose(Q.T @ Q, np.eye(7), atol=1e-12)
    np.testing.assert_allclose(np.sort(w), np.linalg.eigvalsh(V), atol=1e-11)
    P = oracle.pinv_sym(V)
    np.testing.assert_allclose(P, np.linalg.pinv(V, hermitian=True), rtol=1e-8, atol=1e-10)
    # Penrose conditions
    np.testing.assert_allclose(V @ P @ V, V, atol=1e-10)
    np.testing.assert_allclose(P @ V @ P, P, atol=1e-10)


def test_solve_normals_residual_and_branches():
    rng = np.random.default_rng(4)
    V = _spd(6, rng, cond=1e4)
    M = rng.standard_normal((20, 6))
    A, b = oracle.solve_normals(M, V)
    assert b == 0
    np.testing.assert_allclose(A @ V, M, rtol=1e-10, atol=1e-10)
    x = rng.standard_normal((6, 3))
    S = x @ x.T
    A2, b2 = oracle.solve_normals(M, S)
    assert b2 == 1
    np.testing.assert_allclose(A2, M @ np.linalg.pinv(S, hermitian=True), rtol=1e-7, atol=1e-9)


def test_normalize():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((10, 4))
    A[:, 2] = 0
    B, lam = oracle.normalize(A)
    np.testing.assert_allclose(lam, np.linalg.norm(A, axis=0), rtol=1e-14)
    assert lam[2] == 0 and not B[:, 2].any()
    for r in (0, 1, 3):
        assert abs(np.linalg.norm(B[:, r]) - 1) < 1e-14
        np.testing.assert_allclose(B[:, r] * lam[r], A[:, r], rtol=1e-14)


def _dense(dims, inds, vals):
    X = np.zeros(dims)
    np.add.at(X, tuple(inds), vals.astype(np.float64))
    return X


def _reconstruct(factors, lam):
    R = lam.shape[0]
    X = 0
    for r in range(R):
        t = lam[r]
        for A in factors:
            t = np.multiply.outer(t, A[:, r])
        X = X + t
    return X


@pytest.mark.parametrize("dims", [(6, 5, 4), (4, 3, 5, 3)])
def test_fit_formula_equals_explicit_residual(dims):
    rng = np.random.default_rng(len(dims))
    nnz = 40
    inds = [rng.integers(0, d, nnz).astype(np.int32) for d in dims]
    vals = rng.random(nnz).astype(np.float32)
    inds, vals = oracle.coalesce(inds, vals, dims)
    R = 3
    res = oracle.cpd_als(inds, vals, dims, R, max_iters=4, seed=9)
    X = _dense(dims, inds, vals)
    Xh = _reconstruct(res["factors"], res["lam"])
    explicit = 1 - np.linalg.norm(X - Xh) / np.linalg.norm(X)
    assert abs(res["fits"][-1] - explicit) < 1e-9


def _lowrank_dense(dims, R, rng):
    # well-conditioned factors: orthonormal columns plus a positive shift
    fac = []
    for d in dims:
        Q, _ = np.linalg.qr(rng.standard_normal((d, R)))
        fac.append(Q + 0.1)
    lam = np.array([3.0, 2.0, 1.5])[:R]
    return _reconstruct(fac, lam)


# Seed 3 is left out on purpose: from its initial factors ALS settles in a
# local minimum (fit 0.697), which an independent numpy restatement of
# Algorithm 1 from the same start reaches too. Seeds 1, 2, 4 reach fit 1.
@pytest.mark.parametrize("seed", [1, 2, 4])
def test_exact_recovery_of_fully_observed_rank3(seed):
    rng = np.random.default_rng(100 + seed)
    dims = (10, 9, 8)
    X = _lowrank_dense(dims, 3, rng).astype(np.float32)
    coords = np.indices(dims).reshape(3, -1)
    inds = [c.astype(np.int32) for c in coords]
    vals = X.reshape(-1)
    res = oracle.cpd_als(inds, vals, dims, 3, max_iters=500, tol=1e-12, seed=seed)
    assert res["fits"][-1] >= 1 - 1e-6, res["fits"][-5:]


def test_residual_non_increasing():
    rng = np.random.default_rng(8)
    dims = (15, 12, 10)
    nnz = 600
    inds = [rng.integers(0, d, nnz).astype(np.int32) for d in dims]
    vals = rng.random(nnz).astype(np.float32)
    inds, vals = oracle.coalesce(inds, vals, dims)
    res = oracle.cpd_als(inds, vals, dims, 4, max_iters=25, seed=4)
    normx = np.sqrt(np.sum(vals.astype(np.float64) ** 2))
    resid = (1 - res["fits"]) * normx
    assert np.all(np.diff(resid) <= 1e-12 * normx), resid
    assert np.all(res["fits"] <= 1.0)


def test_mode_update_is_one_step_of_als():
    """One call of the mode update equals a literal numpy restatement of
    one mode update of Algorithm 1 (Hadamard of Grams, solve, normalise)."""
    rng = np.random.default_rng(12)
    dims = (8, 7, 6)
    nnz = 120
    inds = [rng.integers(0, d, nnz).astype(np.int32) for d in dims]
    vals = rng.random(nnz).astype(np.float32)
    inds, vals = oracle.coalesce(inds, vals, dims)
    R = 3
    F = [rng.random((d, R)) for d in dims]
    G = [f.T @ f for f in F]
    A1, lam, G1, M, b = oracle.als_mode_update(inds, vals, dims, F, G, 1)
    X = _dense(dims, inds, vals)
    Mw = np.einsum("ijk,ir,kr->jr", X, F[0], F[2])
    np.testing.assert_allclose(M, Mw, rtol=1e-12)
    V = G[0] * G[2]
    Aw = np.linalg.solve(V, Mw.T).T
    lw = np.linalg.norm(Aw, axis=0)
    np.testing.assert_allclose(lam, lw, rtol=1e-10)
    np.testing.assert_allclose(A1, Aw / lw, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(G1, (Aw / lw).T @ (Aw / lw), rtol=1e-9, atol=1e-12)
    assert b == 0


def test_tol_stops_early_and_history_length():
    rng = np.random.default_rng(13)
    dims = (10, 9, 8)
    X = _lowrank_dense(dims, 3, rng).astype(np.float32)
    coords = np.indices(dims).reshape(3, -1)
    res = oracle.cpd_als([c.astype(np.int32) for c in coords], X.reshape(-1), dims, 3,
                         max_iters=400, tol=1e-4, seed=1)
    assert res["iters"] < 400
    assert len(res["fits"]) == res["iters"]
    assert abs(res["fits"][-1] - res["fits"][-2]) < 1e-4
