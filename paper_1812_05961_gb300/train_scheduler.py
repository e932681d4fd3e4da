"""Train the learned MTTKRP scheduler and write the model the package ships.

    python -m paper_1812_05961_gb300.train_scheduler [--tensors 2000] [--nnz-range 1e5 2e8]
        [--split 2e7] [--samples FILE ...] [--out FILE]

Steps, all on the GPU through the library: generate seeded synthetic tensors
(3-5 modes, mode lengths log-uniform in [1e2, 1e7], nnz log-uniform in the
`--nnz-range` capped at a quarter of the index space, Zipf exponent
U(0.8, 1.5) per tensor, rank drawn from {8, 16, 32, 64}); time every
candidate schedule of every root mode under both gather types with the
exhaustive autotuner (sptt_autotune); fit the MLP to log2(time / best time)
with the library's training kernels (sptt_mlp_train); write the parameters
and the feature standardisation to a JSON file (default: sched_model.json
next to this file), which default_scheduler() loads. `--samples` reads
timed samples written earlier by `--dump` in place of sweeping again.

The tensors are drawn in two strata of the log-uniform law, below and above
`--split` (seeds `--seed` and `--seed` + 1), in the proportion the law gives
them (for [1e5, 2e8] split at 2e7: 1,394 and 606 of 2,000), so that a set can
be extended on either side without redrawing the other. tensor_specs(n, seed,
...) draws tensor k identically whatever n is.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
MODEL = os.path.join(HERE, "sched_model.json")


def tensor_specs(n: int, seed: int, nnz_max: float = 2e7, nnz_min: float = 1e5):
    """(dims, nnz, zipf s, rank, tensor seed) of n generated tensors."""
    import numpy as np
    g = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nm = int(g.integers(3, 6))
        dims = [int(math.exp(g.uniform(math.log(100), math.log(1e7)))) for _ in range(nm)]
        space = float(np.prod(dims, dtype=np.float64))
        nnz = int(min(math.exp(g.uniform(math.log(nnz_min), math.log(nnz_max))), space / 4))
        s = float(g.uniform(0.8, 1.5))
        R = int(g.choice([8, 16, 32, 64]))
        out.append((dims, max(nnz, 1000), s, R, seed * 100000 + i))
    return out


def strata(n: int, lo: float, hi: float, split: float):
    """Tensors below and above split of n drawn log-uniform in [lo, hi]."""
    below = int(round(n * math.log(split / lo) / math.log(hi / lo))) if lo < split < hi else (n if split >= hi else 0)
    return below, n - below


def specs_for(n: int, seed: int, lo: float = 1e5, hi: float = 2e8, split: float = 2e7):
    """The stratified draw of n tensors: specs below split (seed), then above (seed + 1)."""
    below, above = strata(n, lo, hi, split)
    return tensor_specs(below, seed, min(split, hi), lo) + tensor_specs(above, seed + 1, hi, max(split, lo))


def sweep(specs, device, log=None):
    """The autotuner's timings of every spec (schedtrain samples)."""
    import torch

    import tensorgen

    from . import schedtrain
    ds = schedtrain.Dataset()
    t0 = time.time()
    for k, (dims, nnz, s, R, sd) in enumerate(specs):
        while True:
            try:
                t = tensorgen.sample_unique(dims, nnz, sd, device, "zipf", s=s, values="uniform")
                break
            except RuntimeError:  # too concentrated for that many distinct coordinates: halve
                nnz //= 2
        ds.samples += schedtrain.sweep_tensor(t.dims, t.inds, t.vals, R, reps=3, label="t%d" % k)
        del t
        torch.cuda.empty_cache()
        if log and (k + 1) % 100 == 0:
            log("%d tensors, %d samples, %.0f s" % (k + 1, len(ds.samples), time.time() - t0))
    return ds


def dump(ds, path: str):
    with open(path, "w") as f:
        json.dump([{"features": x.features, "times_ms": x.times_ms, "default": x.default, "label": x.label,
                    "rank": x.rank, "dtype": x.dtype, "dims": x.dims, "nnz": x.nnz} for x in ds.samples], f)


def read_samples(path: str):
    from . import schedtrain
    with open(path) as f:
        rows = json.load(f)
    return [schedtrain.Sample(r["features"], r["times_ms"], r["default"], r.get("label", ""), r.get("rank", 16),
                              r.get("dtype", 0), r.get("dims", []), r.get("nnz", 0)) for r in rows]


def save(model, path: str, meta: dict):
    from . import sptt_mlp_get
    P, mu, sd = sptt_mlp_get(model.handle)
    with open(path, "w") as f:
        json.dump({"params": [float(x) for x in P], "mu": [float(x) for x in mu], "sd": [float(x) for x in sd],
                   "meta": meta}, f)


def load(path: str = MODEL):
    """An Mlp holding the parameters stored at path."""
    import torch

    from . import Mlp, sptt_mlp_set
    with open(path) as f:
        d = json.load(f)
    m = Mlp(0)
    sptt_mlp_set(m.handle, torch.tensor(d["params"], dtype=torch.float32), torch.tensor(d["mu"], dtype=torch.float32),
                 torch.tensor(d["sd"], dtype=torch.float32))
    return m


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--tensors", type=int, default=2000)
    p.add_argument("--nnz-range", type=float, nargs=2, default=(1e5, 2e8), metavar=("MIN", "MAX"))
    p.add_argument("--split", type=float, default=2e7, help="stratum boundary of the nnz draw")
    p.add_argument("--samples", nargs="*", default=None, help="timed samples (--dump files) to train on instead")
    p.add_argument("--seed", type=int, default=21)
    p.add_argument("--steps", type=int, default=6000)
    p.add_argument("--lr", type=float, default=3e-3)
    p.add_argument("--out", default=MODEL)
    p.add_argument("--dump", default=None, help="also write the timed samples to this JSON file")
    a = p.parse_args(argv)
    import torch

    from . import schedtrain
    dev = torch.device("cuda")
    lo, hi = a.nnz_range
    if a.samples:
        ds = schedtrain.Dataset([x for path in a.samples for x in read_samples(path)])
    else:
        ds = sweep(specs_for(a.tensors, a.seed, lo, hi, a.split), dev, log=lambda s: print(s, flush=True))
    if a.dump:
        dump(ds, a.dump)
    model, hist = schedtrain.train(ds, steps=a.steps, lr=a.lr)
    r_model = schedtrain.summarize(schedtrain.regret(ds, model))
    r_default = schedtrain.summarize(schedtrain.regret(ds))
    meta = {"tensors": a.tensors, "strata": list(strata(a.tensors, lo, hi, a.split)), "nnz_range": [lo, hi],
            "split": a.split, "samples": len(ds.samples), "seed": a.seed, "steps": a.steps, "lr": a.lr,
            "loss_first_last": [float(hist[0]), float(hist[-1])],
            "train_regret_learned": r_model, "train_regret_default": r_default}
    save(model, a.out, meta)
    print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(HERE))
    main()
