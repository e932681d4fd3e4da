"""Training and evaluation of the learned MTTKRP scheduler.

Orchestration only: the timings come from the library's autotuner
(sptt_autotune), the statistics from sptt_csf_features, and the network is
trained and run by the library's own MLP kernels (sptt_mlp_train,
sptt_mlp_predict). The caller supplies the tensors.

Target of the regression: for each (tensor, root mode, rank) sample and each
candidate schedule k, log2(time_k / min_j time_j), so 0 marks the best.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence

import torch

from . import (SPTT_F32, Csf, Mlp, sptt_autotune, sptt_csf_features, sptt_mlp_predict, sptt_mlp_train,
               sptt_sched_candidates)


@dataclass
class Sample:
    features: List[float]
    times_ms: List[float]
    label: str = ""
    rank: int = 16


@dataclass
class Dataset:
    samples: List[Sample] = field(default_factory=list)

    def tensors(self, device):
        X = torch.tensor([s.features for s in self.samples], dtype=torch.float32, device=device)
        T = torch.tensor([[math.log2(t / min(s.times_ms)) for t in s.times_ms] for s in self.samples],
                         dtype=torch.float32, device=device)
        return X, T


def sweep_tensor(dims, inds, vals, rank: int, dtype: int = SPTT_F32, reps: int = 3, label: str = ""):
    """One sample per root mode: the default CSF's statistics and the time of
    every candidate schedule."""
    out = []
    for root in range(len(dims)):
        csf = Csf(dims, inds, vals, root)
        feats = sptt_csf_features(csf.handle, rank)
        csf.close()
        ms = sptt_autotune(dims, inds, vals, root, rank, dtype, reps)
        out.append(Sample(feats, ms, "%s root %d R %d" % (label, root, rank), rank))
    return out


def train(ds: Dataset, steps: int = 2000, lr: float = 3e-3, seed: int = 0, device="cuda"):
    """Fits a fresh MLP to the dataset; returns (model, loss history)."""
    X, T = ds.tensors(device)
    m = Mlp(seed)
    hist = sptt_mlp_train(m.handle, X, T, steps, lr)
    return m, hist


def default_index(rank: int = 16, dtype: int = SPTT_F32, nnz: int = 1 << 30, sms: int = 152) -> int:
    """Index of the candidate closest to the library's default schedule:
    ascending order, the default variant for the gather type and rank (for
    BF16 gathers the candidate with the same walk shape: 4 for the default
    11, 7 for the default 10), and the default chunk (128, halved while
    nnz / chunk < 256 per SM; the candidates have 64 and 128)."""
    ld = (rank + 7) // 8 * 8
    variant = (4 if ld <= 16 else 7) if dtype != SPTT_F32 else 7
    chunk = 128
    while chunk > 16 and nnz // chunk < sms * 256:
        chunk //= 2
    chunk = 128 if chunk >= 128 else 64
    for i, c in enumerate(sptt_sched_candidates()):
        if c[0] == chunk and c[2] == variant and c[3] == 0:
            return i
    return 0


def regret(ds: Dataset, model=None, fixed: int = None):
    """Per-sample time of the chosen schedule over the best one, minus 1:
    choices from the model, or the fixed candidate index (None: the
    library's default for each sample's rank)."""
    if model is not None:
        choice, _ = sptt_mlp_predict(model.handle, [s.features for s in ds.samples])
    elif fixed is not None:
        choice = [fixed] * len(ds.samples)
    else:
        choice = [default_index(s.rank, nnz=int(round(2.0 ** s.features[0]))) for s in ds.samples]
    return [s.times_ms[k] / min(s.times_ms) - 1.0 for s, k in zip(ds.samples, choice)]


def summarize(r: Sequence[float]):
    xs = sorted(r)
    n = len(xs)
    return {"mean": sum(xs) / n, "median": xs[n // 2], "p90": xs[min(n - 1, int(0.9 * n))], "n": n}
