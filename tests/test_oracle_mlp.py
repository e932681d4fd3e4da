"""Pins for the oracle's scheduler MLP: forward against a numpy restatement,
gradient against central finite differences of the loss."""
import numpy as np

import oracle

NIN, NH, NOUT = 16, 64, 16


def _split(P):
    i = 0
    out = []
    for shape in ((NH, NIN), (NH,), (NH, NH), (NH,), (NOUT, NH), (NOUT,)):
        k = int(np.prod(shape))
        out.append(P[i:i + k].reshape(shape))
        i += k
    return out


def test_mlp_forward_matches_numpy():
    rng = np.random.default_rng(0)
    P = rng.standard_normal(oracle.mlp_nparams(NIN, NH, NOUT)) * 0.2
    x = rng.standard_normal((7, NIN))
    W1, b1, W2, b2, W3, b3 = _split(P)
    h1 = np.maximum(x @ W1.T + b1, 0)
    h2 = np.maximum(h1 @ W2.T + b2, 0)
    want = h2 @ W3.T + b3
    np.testing.assert_allclose(oracle.mlp_forward(P, x, NIN, NH, NOUT), want, rtol=1e-12, atol=1e-12)


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    P = rng.standard_normal(oracle.mlp_nparams(NIN, NH, NOUT)) * 0.3
    x = rng.standard_normal((5, NIN))
    t = rng.standard_normal((5, NOUT))
    L, G = oracle.mlp_loss_grad(P, x, t, NIN, NH, NOUT)
    y = oracle.mlp_forward(P, x, NIN, NH, NOUT)
    assert abs(L - np.mean((y - t) ** 2)) < 1e-12
    idx = rng.choice(P.size, 200, replace=False)
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (oracle.mlp_loss_grad(Pp, x, t, NIN, NH, NOUT)[0] - oracle.mlp_loss_grad(Pm, x, t, NIN, NH, NOUT)[0]) / (2 * h)
        assert abs(fd - G[i]) <= 1e-6 * max(1.0, abs(G[i])), (i, fd, G[i])
