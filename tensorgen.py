"""Seeded synthetic sparse tensors (COO) for tests and benchmarks.

This module only draws inputs; it holds none of the decomposition's
arithmetic, and both the CUDA path and the CPU oracle consume what it makes.
Everything is generated with torch on the requested device from a
``torch.Generator`` seeded by the caller, so a (seed, device) pair always
yields the same tensor.

Recipes (the shapes and distributions of the workloads in the design notes):
  * ``uniform``: coordinates uniform over the index space, values U(0,1).
  * ``zipf``: per mode, a rank k ~ Zipf(s) truncated to [1, I_m] (inverse-CDF
    table), mapped through a seeded random permutation of the mode's indices;
    values lognormal(0,1) or U(0,1).
  * ``batch``: many small tensors with log-uniform mode lengths and nnz, 30%
    of coordinates drawn from a Zipf(1.1) hot set.
"Unique" generators resample colliding coordinates until exactly ``nnz``
distinct ones exist, then shuffle them, so the non-zeros arrive unsorted.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import torch


@dataclass
class CooTensor:
    dims: List[int]
    inds: List[torch.Tensor]          # per mode, int32 [nnz]
    vals: torch.Tensor                # float32 [nnz]
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.vals.shape[0])

    @property
    def nmodes(self) -> int:
        return len(self.dims)

    def to(self, device) -> "CooTensor":
        return CooTensor(list(self.dims), [x.to(device) for x in self.inds], self.vals.to(device),
                         dict(self.meta))

    def numpy(self):
        return [x.cpu().numpy() for x in self.inds], self.vals.cpu().numpy()


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _key_words(dims):
    """Group modes (from the last) into int64 words of at most 62 bits."""
    words, cur, bits = [], [], 0
    for m in reversed(range(len(dims))):
        b = max(1, math.ceil(math.log2(max(int(dims[m]), 2))))
        if cur and bits + b > 62:
            words.append(cur)
            cur, bits = [], 0
        cur.append(m)
        bits += b
    words.append(cur)
    return words  # words[0] = least significant group


def _unique_coords(coords: torch.Tensor, dims) -> torch.Tensor:
    """Distinct rows of coords [n, N] (int64), in lexicographic order."""
    if coords.shape[0] == 0:
        return coords
    words = _key_words(dims)
    keys = []
    for grp in words:
        k = torch.zeros(coords.shape[0], dtype=torch.int64, device=coords.device)
        for m in reversed(grp):  # most significant mode of the group first
            k = k * int(dims[m]) + coords[:, m]
        keys.append(k)
    perm = torch.arange(coords.shape[0], device=coords.device)
    for k in keys:  # least significant word first; stable sorts give lexicographic order
        _, p = torch.sort(k[perm], stable=True)
        perm = perm[p]
    c = coords[perm]
    new = torch.ones(c.shape[0], dtype=torch.bool, device=c.device)
    new[1:] = (c[1:] != c[:-1]).any(dim=1)
    return c[new]


def _zipf_table(n: int, s: float, device) -> torch.Tensor:
    # built on the CPU, whose cumulative sum adds in a fixed order (a GPU
    # scan's float64 rounding varied from run to run, and with it a few
    # drawn coordinates), then moved to the device
    k = torch.arange(1, n + 1, dtype=torch.float64)
    w = k.pow(-float(s))
    cdf = torch.cumsum(w, 0)
    return (cdf / cdf[-1]).to(device)


def _draw_mode(n_samples, I, dist, s, perm, table, g, device):
    if dist == "uniform":
        return torch.randint(0, int(I), (n_samples,), generator=g, device=device, dtype=torch.int64)
    u = torch.rand(n_samples, generator=g, device=device, dtype=torch.float64)
    r = torch.searchsorted(table, u, right=True).clamp_(max=int(I) - 1)
    return perm[r]


def _values(n, values, g, device):
    if values == "uniform":
        return torch.rand(n, generator=g, device=device, dtype=torch.float32)
    if values == "lognormal":
        return torch.exp(torch.randn(n, generator=g, device=device, dtype=torch.float32))
    if values == "ones":
        return torch.ones(n, device=device, dtype=torch.float32)
    raise ValueError(values)


def sample_unique(dims, nnz: int, seed: int, device="cpu", dist: str = "uniform",
                  s: float = 1.1, values: str = "uniform", shuffle: bool = True) -> CooTensor:
    """``nnz`` distinct coordinates drawn per mode from ``dist`` ("uniform" or
    "zipf" with exponent ``s``), values from ``values``."""
    dims = [int(d) for d in dims]
    space = 1
    for d in dims:
        space *= d
    if nnz > space:
        raise ValueError("nnz %d exceeds the index space %d" % (nnz, space))
    g = _gen(seed, device)
    perms, tables = [], []
    for I in dims:
        if dist == "zipf":
            perms.append(torch.randperm(I, generator=g, device=device))
            tables.append(_zipf_table(I, s, device))
        else:
            perms.append(None)
            tables.append(None)
    have = torch.zeros((0, len(dims)), dtype=torch.int64, device=device)
    want = nnz
    rounds = 0
    while have.shape[0] < nnz:
        deficit = nnz - have.shape[0]
        n_draw = int(deficit * 1.25) + 1024 if rounds else nnz
        cols = [_draw_mode(n_draw, dims[m], dist, s, perms[m], tables[m], g, device)
                for m in range(len(dims))]
        fresh = torch.stack(cols, dim=1)
        have = _unique_coords(torch.cat([have, fresh], 0), dims)
        rounds += 1
        if rounds > 200:
            raise RuntimeError("could not reach %d distinct coordinates" % want)
    if have.shape[0] > nnz:
        keep = torch.randperm(have.shape[0], generator=g, device=device)[:nnz]
        have = have[keep]
    if shuffle:
        have = have[torch.randperm(have.shape[0], generator=g, device=device)]
    vals = _values(nnz, values, g, device)
    inds = [have[:, m].to(torch.int32).contiguous() for m in range(len(dims))]
    return CooTensor(dims, inds, vals, {"dist": dist, "s": s, "values": values, "seed": seed,
                                        "resample_rounds": rounds})


def sample_with_duplicates(dims, nnz: int, seed: int, device="cpu", values: str = "uniform",
                           dup_frac: float = 0.3) -> CooTensor:
    """Uniform coordinates where about ``dup_frac`` of the entries repeat an
    earlier coordinate (for coalescing tests)."""
    dims = [int(d) for d in dims]
    g = _gen(seed, device)
    n_base = max(1, nnz - int(nnz * dup_frac))
    cols = [torch.randint(0, d, (n_base,), generator=g, device=device, dtype=torch.int64)
            for d in dims]
    base = torch.stack(cols, 1)
    extra = base[torch.randint(0, n_base, (nnz - n_base,), generator=g, device=device)]
    c = torch.cat([base, extra], 0)
    c = c[torch.randperm(c.shape[0], generator=g, device=device)]
    vals = _values(nnz, values, g, device)
    return CooTensor(dims, [c[:, m].to(torch.int32).contiguous() for m in range(len(dims))], vals,
                     {"dist": "uniform+dups", "seed": seed})


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def small_uniform(seed: int = 1, device="cpu") -> CooTensor:
    """200 x 150 x 100, 20,000 distinct uniform coordinates, values U(0,1)."""
    return sample_unique([200, 150, 100], 20000, seed, device, "uniform", values="uniform")


def powerlaw3(seed: int = 2, device="cpu", nnz: int = 100_000_000,
              dims=(480_000, 18_000, 2_000), s: float = 1.1) -> CooTensor:
    """3-mode power-law tensor, the shape of the NETFLIX tensor of Table I:
    480,000 x 18,000 x 2,000, 1e8 distinct non-zeros, Zipf(1.1) per mode then
    a random permutation, values lognormal(0,1)."""
    return sample_unique(list(dims), nnz, seed, device, "zipf", s=s, values="lognormal")


def powerlaw4(seed: int = 3, device="cpu", nnz: int = 150_000_000,
              dims=(2_000_000, 500_000, 50_000, 1_000), s: float = 1.2) -> CooTensor:
    """4-mode power-law tensor 2e6 x 5e5 x 5e4 x 1e3, 1.5e8 distinct non-zeros,
    Zipf(1.2) per mode, values U(0,1)."""
    return sample_unique(list(dims), nnz, seed, device, "zipf", s=s, values="uniform")


def batch_tensor_specs(count: int = 512, seed: int = 4, nnz_max: int = 2_000_000):
    """Shapes of the batched workload: 3 or 4 modes (50/50), mode lengths
    log-uniform in [100, 200,000], nnz log-uniform in [1,000, nnz_max] capped
    at the index space. Returns a list of (dims, nnz)."""
    g = _gen(seed, "cpu")
    specs = []
    for _ in range(count):
        n = 3 if torch.rand(1, generator=g).item() < 0.5 else 4
        dims = [int(round(math.exp(math.log(100) + torch.rand(1, generator=g).item()
                                   * (math.log(200_000) - math.log(100))))) for _ in range(n)]
        nnz = int(round(math.exp(math.log(1000) + torch.rand(1, generator=g).item()
                                 * (math.log(nnz_max) - math.log(1000)))))
        space = 1
        for d in dims:
            space *= d
        specs.append((dims, min(nnz, space)))
    return specs


def batch_member(dims, nnz: int, seed: int, device="cpu", hot_frac: float = 0.3,
                 s: float = 1.1) -> CooTensor:
    """One tensor of the batched workload: distinct coordinates, 70% uniform
    and 30% from a Zipf(1.1) hot set (per-mode Zipf then permutation), values
    U(0,1)."""
    dims = [int(d) for d in dims]
    n_hot = int(round(nnz * hot_frac))
    hot = sample_unique(dims, n_hot, seed * 2 + 1, device, "zipf", s=s, values="uniform",
                        shuffle=False) if n_hot else None
    g = _gen(seed * 2 + 2, device)
    have = torch.stack([x.to(torch.int64) for x in hot.inds], 1) if hot else \
        torch.zeros((0, len(dims)), dtype=torch.int64, device=device)
    rounds = 0
    while have.shape[0] < nnz:
        deficit = nnz - have.shape[0]
        fresh = torch.stack([torch.randint(0, d, (int(deficit * 1.25) + 64,), generator=g,
                                           device=device, dtype=torch.int64) for d in dims], 1)
        have = _unique_coords(torch.cat([have, fresh], 0), dims)
        rounds += 1
        if rounds > 200:
            raise RuntimeError("could not reach %d distinct coordinates" % nnz)
    if have.shape[0] > nnz:
        have = have[torch.randperm(have.shape[0], generator=g, device=device)[:nnz]]
    have = have[torch.randperm(have.shape[0], generator=g, device=device)]
    vals = _values(nnz, "uniform", g, device)
    return CooTensor(dims, [have[:, m].to(torch.int32).contiguous() for m in range(len(dims))],
                     vals, {"dist": "batch", "seed": seed})
