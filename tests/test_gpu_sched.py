"""The schedule machinery: MLP kernels against the FP64 oracle MLP, training,
features, autotuner, planned CP-ALS, and the learned scheduler's regret
against the fixed default on held-out tensors."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_1812_05961_gb300 as sptt
from paper_1812_05961_gb300 import schedtrain
import tensorgen

pytestmark = pytest.mark.gpu

NIN, NH, NOUT = 16, 64, 16
# the held-out claim: the learned choice's mean regret is at most GAIN_FACTOR
# times the fixed default's and at most GAIN_ABS (regret = time of the chosen
# schedule over the autotuner's best, minus 1)
GAIN_FACTOR = 0.5
GAIN_ABS = 0.15


def test_mlp_forward_and_gradient_match_oracle(cuda_device):
    m = sptt.Mlp(seed=3)
    P, mu, sd = sptt.sptt_mlp_get(m.handle)
    assert mu.abs().max() == 0 and (sd == 1).all()  # untrained: no standardisation
    g = torch.Generator().manual_seed(0)
    X = torch.randn(77, NIN, generator=g)
    T = torch.randn(77, NOUT, generator=g)
    Y = sptt.sptt_mlp_forward(m.handle, X.to(cuda_device)).cpu().double().numpy()
    Yo = oracle.mlp_forward(P.double().numpy(), X.double().numpy(), NIN, NH, NOUT)
    assert np.abs(Y - Yo).max() <= 1e-5 * max(1.0, np.abs(Yo).max())
    L, G = sptt.sptt_mlp_loss_grad(m.handle, X.to(cuda_device), T.to(cuda_device))
    Lo, Go = oracle.mlp_loss_grad(P.double().numpy(), X.double().numpy(), T.double().numpy(), NIN, NH, NOUT)
    assert abs(L - Lo) <= 1e-5 * abs(Lo)
    G = G.double().numpy()
    assert np.linalg.norm(G - Go) <= 1e-4 * np.linalg.norm(Go)
    assert np.abs(G - Go).max() <= 1e-4 * np.abs(Go).max()


def test_mlp_training_fits_a_smooth_target(cuda_device):
    g = torch.Generator().manual_seed(1)
    X = torch.randn(512, NIN, generator=g) * 3 + 5
    W = torch.randn(NIN, NOUT, generator=g)
    T = torch.tanh(((X - 5) / 3) @ W / 4)
    m = sptt.Mlp(seed=2)
    hist = sptt.sptt_mlp_train(m.handle, X.to(cuda_device), T.to(cuda_device), 600, 3e-3)
    assert hist[-1] < 0.1 * hist[0], (float(hist[0]), float(hist[-1]))
    _, mu, sd = sptt.sptt_mlp_get(m.handle)
    np.testing.assert_allclose(mu.numpy(), X.mean(0).numpy(), rtol=1e-3, atol=1e-3)
    np.testing.assert_allclose(sd.numpy(), X.std(0, unbiased=False).numpy(), rtol=1e-3)


def test_features_match_a_host_restatement(cuda_device):
    t = tensorgen.sample_unique([300, 200, 50], 30000, seed=4, dist="zipf", s=1.3)
    inds_np, vals_np = t.numpy()
    c = sptt.Csf(t.dims, [x.to(cuda_device) for x in t.inds], t.vals.to(cuda_device), 1)
    f = sptt.sptt_csf_features(c.handle, 16)
    fb = sptt.sptt_csf_features(c.handle, 16, sptt.SPTT_BF16)
    ref = oracle.csf(inds_np, vals_np, t.dims, 1)
    sizes = np.diff(ref["fptr"][1][ref["fptr"][0]])  # leaves per slice (3 modes)
    nnz = ref["nfibs"][-1]
    # a row of 16 FP32 values is 64 bytes (BF16: 32)
    assert abs(f[0] - math.log2(nnz)) < 1e-5 and f[1] == 3 and abs(f[2] - 6) < 1e-6 and abs(fb[2] - 5) < 1e-6
    assert abs(f[13] - math.log2(t.dims[ref["order"][2]] * 64)) < 1e-5
    assert abs(fb[13] - math.log2(t.dims[ref["order"][2]] * 32)) < 1e-5
    assert abs(f[6] - math.log2(ref["nfibs"][0])) < 1e-5
    assert abs(f[10] - math.log2(sizes.max())) < 1e-5
    assert abs(f[11] - sizes[sizes >= 1024].sum() / nnz) < 1e-6
    assert abs(f[12] - (sizes == 1).mean()) < 1e-6


def test_autotune_and_planned_cpd(cuda_device):
    t = tensorgen.sample_unique([2000, 800, 300], 200000, seed=5, dist="zipf", s=1.2)
    di = [x.to(cuda_device) for x in t.inds]
    dv = t.vals.to(cuda_device)
    ms = sptt.sptt_autotune(t.dims, di, dv, 0, 16)
    assert len(ms) == 16 and all(x > 0 for x in ms)
    cands = sptt.sptt_sched_candidates(t.nnz)
    for dt in (sptt.SPTT_F32, sptt.SPTT_BF16):
        for root in range(3):
            d = sptt.sptt_sched_default(t.dims, root, 16, dt, t.nnz)
            assert any(c[0] == d[0] and c[2] == d[2] and c[3] == d[3] for c in cands), d
    base = sptt.Cpd(t.dims, di, dv, 16, seed=1).init()
    base.iterate(4)
    tuned = sptt.Cpd(t.dims, di, dv, 16, seed=1, plan=1).init()
    tuned.iterate(4)
    np.testing.assert_allclose(tuned.fit_history(), base.fit_history(), atol=1e-6)
    m = sptt.Mlp(seed=0)
    learned = sptt.Cpd(t.dims, di, dv, 16, seed=1, plan=2, mlp=m).init()
    learned.iterate(4)
    np.testing.assert_allclose(learned.fit_history(), base.fit_history(), atol=1e-6)
    per_mode = [cands[int(np.argmax(ms))]] * 3  # the slowest one still gives the same numbers
    other = sptt.Cpd(t.dims, di, dv, 16, seed=1, mode_sched=per_mode).init()
    other.iterate(4)
    np.testing.assert_allclose(other.fit_history(), base.fit_history(), atol=1e-6)


def test_training_on_sweeps_fits_the_timings(cuda_device):
    # the library's training kernels on autotuner sweeps of a few generated
    # tensors: the loss falls and the fitted model beats the fixed rule on
    # the tensors it saw
    from paper_1812_05961_gb300 import train_scheduler
    ds = train_scheduler.sweep(train_scheduler.tensor_specs(12, seed=5, nnz_max=2e6), cuda_device)
    model, hist = schedtrain.train(ds, steps=1500, lr=3e-3)
    assert float(hist[-1]) < 0.5 * float(hist[0])
    r_model = schedtrain.summarize(schedtrain.regret(ds, model))
    r_default = schedtrain.summarize(schedtrain.regret(ds))
    assert r_model["mean"] < r_default["mean"], (r_model, r_default)


def test_shipped_scheduler_gains_over_the_fixed_default_on_held_out(cuda_device):
    # the model the package ships (trained by train_scheduler.py on the
    # autotuner's timings of 2,000 generated tensors, nnz log-uniform in
    # [1e5, 2e8]) against the library's
    # fixed default rule, on tensors of the same distribution it never saw
    # (another seed), timed now by the exhaustive autotuner
    from paper_1812_05961_gb300 import train_scheduler
    model = train_scheduler.load()
    held = train_scheduler.sweep(train_scheduler.tensor_specs(40, seed=4242), cuda_device)
    r_model = schedtrain.summarize(schedtrain.regret(held, model))
    r_default = schedtrain.summarize(schedtrain.regret(held))
    print("held-out regret: learned %s, default %s" % (r_model, r_default))
    assert r_model["mean"] <= GAIN_FACTOR * r_default["mean"], (r_model, r_default)
    assert r_model["mean"] <= GAIN_ABS, (r_model, r_default)


# On tensors of 2e7-2e8 non-zeros the fixed rule (the 32-byte FP32 walk and
# the table kernels from its size thresholds) is already within a few percent
# of the best schedule, and the learned choice and the rule trade places from
# one held-out set to the next; no gain is claimed there, only that the
# learned choice stays within LARGE_MARGIN of the rule and within GAIN_ABS of
# the best.
LARGE_MARGIN = 0.03


def test_shipped_scheduler_on_held_out_large_tensors(cuda_device):
    from paper_1812_05961_gb300 import train_scheduler
    model = train_scheduler.load()
    held = train_scheduler.sweep(train_scheduler.tensor_specs(24, seed=4343, nnz_max=2e8, nnz_min=2e7), cuda_device)
    r_model = schedtrain.summarize(schedtrain.regret(held, model))
    r_default = schedtrain.summarize(schedtrain.regret(held))
    print("held-out regret (2e7-2e8 non-zeros): learned %s, default %s" % (r_model, r_default))
    assert r_model["mean"] <= r_default["mean"] + LARGE_MARGIN, (r_model, r_default)
    assert r_model["mean"] <= GAIN_ABS, (r_model, r_default)
