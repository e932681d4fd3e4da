"""Training and evaluation of the learned MTTKRP scheduler.

Orchestration only: the timings come from the library's autotuner
(sptt_autotune), the statistics from sptt_csf_features, the fixed rule the
network is measured against from sptt_sched_default, and the network is
trained and run by the library's own MLP kernels (sptt_mlp_train,
sptt_mlp_predict). The caller supplies the tensors.

Target of the regression: for each (tensor, root mode, rank, gather type)
sample and each candidate schedule k, log2(time_k / min_j time_j), so 0 marks
the best.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence

import torch

from . import (SPTT_BF16, SPTT_F32, Csf, Mlp, sptt_autotune, sptt_csf_features, sptt_level_order,
               sptt_mlp_predict, sptt_mlp_train, sptt_sched_candidates, sptt_sched_default)


@dataclass
class Sample:
    features: List[float]
    times_ms: List[float]
    default: int            # candidate index of the library's default schedule
    label: str = ""
    rank: int = 16
    dtype: int = SPTT_F32
    dims: List[int] = field(default_factory=list)
    nnz: int = 0


@dataclass
class Dataset:
    samples: List[Sample] = field(default_factory=list)

    def tensors(self, device):
        X = torch.tensor([s.features for s in self.samples], dtype=torch.float32, device=device)
        T = torch.tensor([[math.log2(t / min(s.times_ms)) for t in s.times_ms] for s in self.samples],
                         dtype=torch.float32, device=device)
        return X, T


def default_index(dims, root: int, rank: int, dtype: int, nnz: int) -> int:
    """Candidate index of the schedule the library uses when given none."""
    d = sptt_sched_default(dims, root, rank, dtype, nnz)
    for i, c in enumerate(sptt_sched_candidates(nnz)):
        if c[0] == d[0] and c[2] == d[2] and c[3] == d[3]:
            return i
    raise RuntimeError("the default schedule %r is not a candidate" % (d,))


def sweep_tensor(dims, inds, vals, rank: int, dtypes: Sequence[int] = (SPTT_F32, SPTT_BF16), reps: int = 3,
                 label: str = ""):
    """One sample per root mode and gather type: the statistics of the CSF
    the library would build by default, the time of every candidate
    schedule, and which candidate is the default."""
    out = []
    nnz = int(vals.numel())
    for dtype in dtypes:
        for root in range(len(dims)):
            d = sptt_sched_default(dims, root, rank, dtype, nnz)
            csf = Csf(dims, inds, vals, root, level_order=sptt_level_order(dims, root, d[3]))
            feats = sptt_csf_features(csf.handle, rank, dtype)
            csf.close()
            ms = sptt_autotune(dims, inds, vals, root, rank, dtype, reps)
            out.append(Sample(feats, ms, default_index(dims, root, rank, dtype, nnz),
                              "%s root %d R %d %s" % (label, root, rank, "bf16" if dtype == SPTT_BF16 else "f32"),
                              rank, dtype, [int(x) for x in dims], nnz))
    return out


def train(ds: Dataset, steps: int = 2000, lr: float = 3e-3, seed: int = 0, device="cuda"):
    """Fits a fresh MLP to the dataset; returns (model, loss history)."""
    X, T = ds.tensors(device)
    m = Mlp(seed)
    hist = sptt_mlp_train(m.handle, X, T, steps, lr)
    return m, hist


def regret(ds: Dataset, model=None, fixed: int = None):
    """Per-sample time of the chosen schedule over the best one, minus 1:
    choices from the model, a fixed candidate index, or (neither) the
    library's default for each sample."""
    if model is not None:
        choice, _ = sptt_mlp_predict(model.handle, [s.features for s in ds.samples])
    elif fixed is not None:
        choice = [fixed] * len(ds.samples)
    else:
        choice = [s.default for s in ds.samples]
    return [s.times_ms[k] / min(s.times_ms) - 1.0 for s, k in zip(ds.samples, choice)]


def summarize(r: Sequence[float]):
    xs = sorted(r)
    n = len(xs)
    return {"mean": sum(xs) / n, "median": xs[n // 2], "p90": xs[min(n - 1, int(0.9 * n))], "n": n}
