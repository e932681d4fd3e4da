"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

import tensorgen


def make(dims, nnz, seed, dist="uniform", s=1.1, values="uniform", dups=False):
    if dups:
        return tensorgen.sample_with_duplicates(dims, nnz, seed, values=values)
    return tensorgen.sample_unique(dims, nnz, seed, "cpu", dist=dist, s=s, values=values)


def to_dev(t, dev):
    return [x.to(dev) for x in t.inds], t.vals.to(dev)


def rand_factors(dims, R, seed, ld=None, lo=-1.0, hi=1.0):
    g = torch.Generator().manual_seed(seed)
    ld = ld or R
    out = []
    for d in dims:
        f = torch.zeros(d, ld)
        f[:, :R] = lo + (hi - lo) * torch.rand(d, R, generator=g)
        out.append(f)
    return out


def rel_fro(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)
