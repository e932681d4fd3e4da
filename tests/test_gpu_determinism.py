"""Run-to-run determinism, the race check of the CUDA path.

Every reduction of the path adds in a fixed order (the Gram and post-solve
partial sums, the FP64 block totals), and an output row that only one lane
group touches is stored or added once; the one source of run-to-run
variation is the order in which the chunks of a split slice add their
partials with atomics, and those go into FP64 rows, where the sum of FP32
partials of similar magnitude is exact. So with every slice inside one chunk
(one chunk per tensor) two runs must agree bit for bit, which a race between
lane groups, a missing barrier or an unordered reduction would break; with
split slices and positive factors (partials of one sign) too; with factors
of both signs to 1e-7.
"""
import numpy as np
import pytest
import torch

import paper_1812_05961_gb300 as sptt
from gpu_util import make, rand_factors, rel_fro, to_dev

pytestmark = pytest.mark.gpu

ONE_CHUNK = (4096, 256, 0)  # chunk of 4096 leaves: a tensor of <= 4096 non-zeros is one chunk


@pytest.mark.parametrize("dims", [(300, 200, 100), (40, 30, 20, 10)])
def test_mttkrp_of_one_chunk_is_bitwise_repeatable(dims, cuda_device):
    t = make(dims, 4000, seed=3, dist="zipf", s=1.2)
    F = [f.to(cuda_device) for f in rand_factors(dims, 16, seed=2)]
    di, dv = to_dev(t, cuda_device)
    for root in range(len(dims)):
        c = sptt.Csf(dims, di, dv, root)
        runs = [c.mttkrp(F, sched=ONE_CHUNK).clone() for _ in range(3)]
        for r in runs[1:]:
            assert torch.equal(r, runs[0]), "root %d" % root


def test_gram_is_bitwise_repeatable(cuda_device):
    g = torch.Generator().manual_seed(5)
    A = torch.rand(200003, 16, generator=g).to(cuda_device)
    runs = [sptt.sptt_gram(A, 16).clone() for _ in range(3)]
    for r in runs[1:]:
        assert torch.equal(r, runs[0])


def test_cpals_of_one_chunk_tensors_is_bitwise_repeatable(cuda_device):
    dims = (120, 90, 60)
    t = make(dims, 3500, seed=8, dist="zipf", s=1.1)
    di, dv = to_dev(t, cuda_device)
    runs = []
    for _ in range(2):
        c = sptt.Cpd(dims, di, dv, 8, seed=4, sched=ONE_CHUNK + (0,)).init()
        c.iterate(6)
        runs.append((np.asarray(c.fit_history()), [c.factor(m) for m in range(3)], c.lam()))
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    for a, b in zip(runs[0][1], runs[1][1]):
        assert torch.equal(a, b)
    assert torch.equal(runs[0][2], runs[1][2])


def test_mttkrp_with_split_slices_repeats_to_tolerance(cuda_device):
    # power-law slices spanning many chunks: their partials meet in atomics
    dims = (2000, 800, 300)
    t = make(dims, 200000, seed=6, dist="zipf", s=1.3)
    F = [f.to(cuda_device) for f in rand_factors(dims, 16, seed=7)]
    di, dv = to_dev(t, cuda_device)
    for root in range(3):
        c = sptt.Csf(dims, di, dv, root)
        a = c.mttkrp(F).cpu().double().numpy()
        b = c.mttkrp(F).cpu().double().numpy()
        assert rel_fro(a, b) <= 1e-7


@pytest.mark.parametrize("dtype", [sptt.SPTT_F32, sptt.SPTT_BF16])
def test_mttkrp_with_split_slices_and_positive_factors_is_bitwise_repeatable(dtype, cuda_device):
    dims = (2000, 800, 300)
    t = make(dims, 200000, seed=6, dist="zipf", s=1.3)
    tdt = torch.bfloat16 if dtype == sptt.SPTT_BF16 else torch.float32
    F = [f.to(cuda_device).to(tdt) for f in rand_factors(dims, 16, seed=7, lo=0.0, hi=1.0)]
    di, dv = to_dev(t, cuda_device)
    for root in range(3):
        c = sptt.Csf(dims, di, dv, root)
        runs = [c.mttkrp(F, factor_dtype=dtype).clone() for _ in range(3)]
        for r in runs[1:]:
            assert torch.equal(r, runs[0]), "root %d" % root


def test_bf16_cpals_with_split_slices_is_bitwise_repeatable(cuda_device):
    # the mixed path's trajectory no longer depends on the order of the
    # split-slice atomics (BF16 rounding of the factor copies used to amplify it)
    dims = (3000, 1000, 400)
    t = make(dims, 300000, seed=9, dist="zipf", s=1.2)
    di, dv = to_dev(t, cuda_device)
    runs = []
    for _ in range(2):
        c = sptt.Cpd(dims, di, dv, 16, seed=2, precision=sptt.SPTT_BF16).init()
        c.iterate(12)
        c.refine(1)
        runs.append((np.asarray(c.fit_history()), [c.factor(m) for m in range(3)]))
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    for a, b in zip(runs[0][1], runs[1][1]):
        assert torch.equal(a, b)
