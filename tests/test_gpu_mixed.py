"""Mixed-precision CP-ALS (BF16 factor gathers with FP32 accumulation, FP64
Grams / normal equations, then one FP32 refinement sweep) against the FP64
oracle (Algorithm 1).

The tensor is a scaled-down form of the 4-mode power-law workload:
8,000 x 2,000 x 500 x 100, 300,000 distinct Zipf(1.2) coordinates per mode,
values U(0,1), rank 64. The runs are compared after the same number of
iterations from the same initial factors, as the workload states its run (25
BF16 iterations + one FP32 sweep against 26 iterations). A stop on the fit
change (Algorithm 1's |fit - fit_prev| < tol) is not a usable common point at
this rank: the fit still gains 1e-5 per iteration after ~110 iterations, and
the per-iteration change of a BF16-gathered fit is noisier than that (with
tol = 1e-5 the mixed run stopped after 25 iterations, FP32 after 82 and the
oracle after 111; at 82 iterations FP32 and the oracle agreed to 6e-6).

Stated per result: fit of the mixed path and of the FP32 path against the
oracle (|delta fit| <= 1e-4), and each factor's relative error against the
oracle's. From the same state, the refinement sweep itself agrees with one
FP64 iteration of the oracle to 1e-5 in fit.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_1812_05961_gb300 as sptt
import tensorgen
from gpu_util import rel_fro

pytestmark = pytest.mark.gpu

DIMS = (8000, 2000, 500, 100)
NNZ = 300_000
R = 64
ITERS = 26  # the mixed run: 25 BF16 iterations + 1 FP32 refinement sweep
SEED = 3


def _oracle(inds, vals, iters, init=None):
    prev = oracle.threads()
    oracle.set_threads(os.cpu_count() or 1)
    try:
        return oracle.cpd_als(inds, vals, DIMS, R, iters, seed=SEED, init=init)
    finally:
        oracle.set_threads(prev)


@pytest.fixture(scope="module")
def case():
    t = tensorgen.sample_unique(DIMS, NNZ, 31, "cpu", dist="zipf", s=1.2, values="uniform")
    inds, vals = t.numpy()
    return t, _oracle(inds, vals, ITERS)


def _cpd(t, dev, precision):
    di = [x.to(dev) for x in t.inds]
    dv = t.vals.to(dev)
    return sptt.Cpd(DIMS, di, dv, R, seed=SEED, precision=precision).init()


def test_mixed_and_fp32_cpals_match_fp64_oracle(case, cuda_device):
    t, ref = case
    fits_o = np.asarray(ref["fits"])
    report = {"oracle_fit": float(fits_o[-1])}
    for name, prec in (("fp32", sptt.SPTT_F32), ("mixed", sptt.SPTT_BF16)):
        cpd = _cpd(t, cuda_device, prec)
        if prec == sptt.SPTT_BF16:
            cpd.iterate(ITERS - 1)
            cpd.refine(1)
        else:
            cpd.iterate(ITERS)
        fits = np.asarray(cpd.fit_history())
        errs = [rel_fro(cpd.factor(m).numpy(), ref["factors"][m]) for m in range(len(DIMS))]
        report[name] = {"fit": float(fits[-1]), "delta_fit": float(fits[-1] - fits_o[-1]),
                        "max_delta_fit_per_iter": float(np.abs(fits - fits_o).max()),
                        "factor_rel_err": [float("%.3e" % e) for e in errs]}
        if prec == sptt.SPTT_F32:
            # every iteration of the FP32 path tracks the oracle
            np.testing.assert_allclose(fits, fits_o, atol=1e-4, rtol=0)
        del cpd
        torch.cuda.empty_cache()
    print("mixed precision vs FP64 oracle after %d iterations:" % ITERS, report)
    assert abs(report["fp32"]["delta_fit"]) <= 1e-4, report
    assert abs(report["mixed"]["delta_fit"]) <= 1e-4, report


def test_refinement_sweep_equals_one_fp64_iteration_from_the_same_state(case, cuda_device):
    # the BF16 run's factors before the refinement sweep seed one oracle
    # iteration; the GPU's FP32 sweep from that state must land on its fit
    t, _ = case
    cpd = _cpd(t, cuda_device, sptt.SPTT_BF16)
    cpd.iterate(ITERS - 1)
    before = [cpd.factor(m) for m in range(len(DIMS))]
    cpd.refine(1)
    fit = cpd.fit()[0]
    inds, vals = t.numpy()
    one = _oracle(inds, vals, 1, init=[f.double().numpy() for f in before])
    errs = [rel_fro(cpd.factor(m).numpy(), one["factors"][m]) for m in range(len(DIMS))]
    print("refinement sweep vs one FP64 iteration: fit %.8f vs %.8f, factor rel. err %s"
          % (fit, one["fits"][-1], ["%.2e" % e for e in errs]))
    assert abs(fit - float(one["fits"][-1])) <= 1e-5, (fit, one["fits"])
    assert max(errs) <= 1e-2, errs
