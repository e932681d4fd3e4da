"""Checkpoint / resume of a CP-ALS run: a run stopped, saved, restored into
a fresh handle and continued follows the uninterrupted run."""
import numpy as np
import pytest
import torch

import paper_1812_05961_gb300 as sptt
from gpu_util import make, rel_fro, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,R,kw,tol", [
    ((300, 250, 200), 16, {}, 1e-7),
    ((60, 50, 40, 30), 12, dict(csf_mode=1), 1e-7),
    ((200, 150, 100), 8, dict(precision=sptt.SPTT_BF16), 1e-5),
])
def test_resume_continues_the_run(dims, R, kw, tol, cuda_device):
    # The restored state is the saved one byte for byte. From equal states
    # one iteration of each handle agrees to the run-to-run spread of the
    # split-slice atomics (which BF16 gathers amplify: an FP32 ulp can flip
    # a BF16 rounding); the FP32 runs also follow the uninterrupted run.
    t = make(dims, 30000, seed=len(dims) + R, dist="zipf", s=1.2)
    di, dv = to_dev(t, cuda_device)
    a = sptt.Cpd(dims, di, dv, R, seed=4, **kw).init()
    a.iterate(3)
    ckp = a.save()
    b = sptt.Cpd(dims, di, dv, R, seed=99, **kw).init()  # another start: everything comes from the checkpoint
    b.load(ckp)
    assert b.save() == ckp
    assert b.fit()[1] == 3
    a.iterate(1)
    b.iterate(1)
    assert abs(a.fit()[0] - b.fit()[0]) <= tol
    if kw.get("precision", sptt.SPTT_F32) == sptt.SPTT_F32:
        full = sptt.Cpd(dims, di, dv, R, seed=4, **kw).init()
        full.iterate(6)
        b.iterate(2)
        np.testing.assert_allclose(b.fit_history(), full.fit_history(), atol=tol, rtol=0)
        for m in range(len(dims)):
            assert rel_fro(b.factor(m).numpy(), full.factor(m).numpy()) <= 1e-4
        np.testing.assert_allclose(b.lam().numpy(), full.lam().numpy(), rtol=1e-4)


def test_load_rewinds_and_rejects_bad_buffers(cuda_device):
    dims = (120, 90, 70)
    t = make(dims, 15000, seed=3)
    di, dv = to_dev(t, cuda_device)
    a = sptt.Cpd(dims, di, dv, 10, seed=1).init()
    a.iterate(2)
    ckp = a.save()
    f2 = a.fit()[0]
    a.iterate(3)
    a.load(ckp)  # back to iteration 2
    assert a.fit() == (pytest.approx(f2, abs=0), 2)
    bad = bytearray(ckp)
    bad[-3] ^= 0x40  # payload byte: checksum mismatch
    for data in (bytes(bad), ckp[:-8], b"NOTACKPT" + ckp[8:]):
        with pytest.raises(sptt.SpttError):
            a.load(data)
    other_rank = sptt.Cpd(dims, di, dv, 11, seed=1).init()
    with pytest.raises(sptt.SpttError):
        other_rank.load(ckp)
    other_shape = sptt.Cpd((121, 90, 70), di, dv, 10, seed=1).init()
    with pytest.raises(sptt.SpttError):
        other_shape.load(ckp)
