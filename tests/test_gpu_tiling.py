"""Mode tiling (opts.leaf_tile_rows): each mode's non-zeros split by their
leaf-mode index into tiles whose leaf rows fit the shared-memory table, the
MTTKRP summed over the tiles (linearity in the non-zeros), against the FP64
oracle (Algorithm 1) and against the untiled path."""
import numpy as np
import pytest
import torch

import oracle
import paper_1812_05961_gb300 as sptt
from gpu_util import make, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,nnz,R,rows", [
    ((300, 250, 200), 40000, 16, 37),   # 3 modes: the shortest other mode at the leaves, 6 tiles
    ((500, 90, 400), 30000, 8, 64),     # tiles of very uneven fill (Zipf leaf indices)
    ((60, 50, 40, 30), 30000, 12, 7),   # 4 modes: ascending order, the longest other mode tiled
    ((20, 18, 16, 14, 12), 20000, 8, 5),
])
def test_tiled_cpals_fits_match_oracle(dims, nnz, R, rows, cuda_device):
    t = make(dims, nnz, seed=nnz % 97 + R, dist="zipf", s=1.2)
    inds_np, vals_np = t.numpy()
    di, dv = to_dev(t, cuda_device)
    iters = 5
    cpd = sptt.Cpd(dims, di, dv, R, seed=7, leaf_tile_rows=rows).init()
    cpd.iterate(iters)
    ref = oracle.cpd_als(inds_np, vals_np, dims, R, iters, seed=7)
    np.testing.assert_allclose(cpd.fit_history(), ref["fits"], atol=1e-4, rtol=0)
    for m in range(len(dims)):
        F = cpd.factor(m).numpy()
        assert np.linalg.norm(F - ref["factors"][m]) <= 1e-3 * max(1.0, np.linalg.norm(ref["factors"][m]))


@pytest.mark.parametrize("precision", [sptt.SPTT_F32, sptt.SPTT_BF16])
def test_tiled_matches_untiled_path_and_graph_replay(precision, cuda_device):
    dims = (3000, 1200, 700)
    t = make(dims, 200000, seed=3, dist="zipf", s=1.1)
    di, dv = to_dev(t, cuda_device)
    R = 16
    runs = {}
    for name, kw in (("untiled", {}), ("tiled", {"leaf_tile_rows": 128}),
                     ("tiled_graph", {"leaf_tile_rows": 128, "use_graph": 1}), ("auto", {"leaf_tile_rows": -1})):
        c = sptt.Cpd(dims, di, dv, R, seed=2, precision=precision, **kw).init()
        c.iterate(6)
        runs[name] = np.asarray(c.fit_history())
        del c
    tol = 1e-5 if precision == sptt.SPTT_F32 else 2e-4
    for name in ("tiled", "tiled_graph", "auto"):
        np.testing.assert_allclose(runs[name], runs["untiled"], atol=tol, rtol=0, err_msg=name)
    np.testing.assert_array_equal(runs["tiled"], runs["tiled_graph"])


def test_tiling_rejects_bad_options(cuda_device):
    dims = (40, 30, 20)
    t = make(dims, 2000, seed=1)
    di, dv = to_dev(t, cuda_device)
    for kw in ({"leaf_tile_rows": 100000}, {"leaf_tile_rows": -2}, {"leaf_tile_rows": 8, "csf_mode": 1},
               {"leaf_tile_rows": 8, "plan": 1}):
        with pytest.raises(sptt.SpttError) as e:
            sptt.Cpd(dims, di, dv, 16, **kw)
        assert e.value.status == sptt.SPTT_ERR_BAD_ARG, kw
