"""The oracle's threaded form against its single loop.

With T > 1 threads the MTTKRP sums each thread's share of the non-zeros into
a private copy of M and adds the copies in thread order, so only the FP64
summation order differs from the literal loop (results agree to rounding).
The row-independent loops of the solve, the normalisation and the Gram keep
every output's own summation order, so a CP-ALS run differs from the
single-thread one only through the MTTKRP's rounding.
"""
import numpy as np
import pytest

import oracle
import tensorgen


@pytest.fixture()
def threads4():
    prev = oracle.threads()
    got = oracle.set_threads(4)
    yield got
    oracle.set_threads(prev)


def _tensor(dims, nnz, seed):
    t = tensorgen.sample_unique(dims, nnz, seed, "cpu", dist="zipf", s=1.1)
    return t.numpy()


def test_threaded_mttkrp_equals_single_loop_to_rounding(threads4):
    dims = [700, 500, 300, 40]
    inds, vals = _tensor(dims, 60000, 5)
    g = np.random.default_rng(2)
    F = [g.uniform(-1, 1, (d, 12)) for d in dims]
    for mode in range(4):
        oracle.set_threads(1)
        M1, A1 = oracle.mttkrp(inds, vals, dims, F, mode, with_abs=True)
        oracle.set_threads(threads4)
        M4, A4 = oracle.mttkrp(inds, vals, dims, F, mode, with_abs=True)
        # every element is a sum of the same terms; only their order differs
        assert np.all(np.abs(M4 - M1) <= 1e-12 * A1 + 1e-300)
        np.testing.assert_allclose(A4, A1, rtol=1e-12, atol=0)


def test_threaded_dense_steps_are_bit_identical(threads4):
    g = np.random.default_rng(3)
    A = g.uniform(-1, 1, (5000, 24))
    oracle.set_threads(1)
    G1 = oracle.gram(A)
    oracle.set_threads(threads4)
    G4 = oracle.gram(A)
    np.testing.assert_array_equal(G1, G4)


def test_threaded_cpd_als_follows_the_single_thread_run(threads4):
    dims = [300, 200, 100]
    inds, vals = _tensor(dims, 30000, 7)
    oracle.set_threads(1)
    r1 = oracle.cpd_als(inds, vals, dims, 8, 8, seed=4)
    oracle.set_threads(threads4)
    r4 = oracle.cpd_als(inds, vals, dims, 8, 8, seed=4)
    np.testing.assert_allclose(r4["fits"], r1["fits"], rtol=0, atol=1e-10)
    for a, b in zip(r4["factors"], r1["factors"]):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-8)


def test_set_threads_reports_the_count_in_effect():
    prev = oracle.threads()
    try:
        assert oracle.set_threads(0) == 1
        n = oracle.set_threads(3)
        assert n in (1, 3)  # 1 when compiled without OpenMP
        assert oracle.threads() == n
    finally:
        oracle.set_threads(prev)
