"""Leaf counts of trees built on Sec. 5's simulation shape (the analogue of
Fig. 2): the trivariate normal with mean 0, unit variances and common
correlation rho, mapped into (0,1)^3 by the normal CDF (the paper scales the
data into the unit cube, Sec. 2), N points, cyclic keys, depths 6-10.

Two split rules are compared on the same points:
  - the subset-median rule of this library (r = 64 subsets by index mod 64);
  - the paper's Fourier-moment estimator (Sec. 3, Eq. (kd:eq:b)) with J
    harmonics per coordinate (the paper's worked example uses the J-vector
    (3, 5), i.e. 15 harmonics).
A depth-10 tree gives every shallower depth, because a level's splits do not
depend on the depth the build stops at: the count of a depth-D leaf is the
sum of the 2^(10 - D) depth-10 leaves below it. The paper reads a tree's
accuracy from how close its leaf counts are to N / 2^D (Sec. 4); this prints
their spread in log2 units beside that ideal.

    python -m paper_2201_08288_gb300.fig2_study [--n N] [--J 15 ...] [--json out.json]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np


def leaf_stats(offs10: np.ndarray, depth: int) -> dict:
    counts = np.diff(offs10).reshape(1 << depth, -1).sum(axis=1).astype(np.float64)
    lg = np.log2(np.maximum(counts, 1.0))
    q = np.quantile(lg, [0.0, 0.25, 0.5, 0.75, 1.0])
    return {"log2_min": q[0], "log2_q25": q[1], "log2_median": q[2], "log2_q75": q[3], "log2_max": q[4],
            "max_rel_dev": float(np.max(np.abs(counts / (counts.sum() / counts.size) - 1.0)))}


def main() -> None:
    import torch
    from paper_2201_08288_gb300 import kdt, workloads
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=3_000_000_000)
    ap.add_argument("--rho", type=float, nargs="+", default=[0.0, 0.25, 0.5, 0.75])
    ap.add_argument("--J", type=int, nargs="+", default=[15])
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--json", default=None)
    args = ap.parse_args()
    dev = torch.device("cuda:0")
    rows = []
    for rho in args.rho:
        t0 = time.perf_counter()
        pts = workloads.mvn_probit_device(args.n, 3, rho, args.seed, dev)
        torch.cuda.synchronize()
        gen_s = time.perf_counter() - t0
        rules = [("median_r64", dict(r=64, subset_mode=0, depth=10))]
        rules += [(f"fourier_J{j}", dict(depth=10, fourier_j=j)) for j in args.J]
        for name, kw in rules:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            t = kdt.kdt_build(pts, **kw)
            torch.cuda.synchronize()
            build_s = time.perf_counter() - t0
            offs = t.node_offsets.cpu().numpy()
            del t
            torch.cuda.empty_cache()
            for depth in range(6, 11):
                rows.append({"rho": rho, "rule": name, "depth": depth, "n": args.n,
                             "log2_ideal": math.log2(args.n / (1 << depth)), "build_s": build_s, "gen_s": gen_s,
                             **leaf_stats(offs, depth)})
                r = rows[-1]
                print(f"rho={rho:<5} {name:12s} D={depth:2d} ideal 2^{r['log2_ideal']:.5f}  "
                      f"min 2^{r['log2_min']:.5f} q25 2^{r['log2_q25']:.5f} med 2^{r['log2_median']:.5f} "
                      f"q75 2^{r['log2_q75']:.5f} max 2^{r['log2_max']:.5f}  max |c/mean-1| {r['max_rel_dev']:.2e}  "
                      f"(build {build_s:.2f} s)", flush=True)
        del pts
        torch.cuda.empty_cache()
    if args.json:
        with open(args.json, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
