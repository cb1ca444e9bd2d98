"""Seeded synthetic inputs shaped like the paper's simulation study and the
benchmark configurations.

This module holds no arithmetic of the method: it only draws points and
subset ids. Both the CUDA path and the CPU oracle consume what it returns.
Host versions use numpy's PCG64; device versions use torch's CUDA generator
(a different stream with the same distribution, used where the input is too
large to draw on the host in reasonable time).

Points are float32 structure-of-arrays, shape [d, n].
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# ---------------------------------------------------------------- host (numpy)


def uniform(n: int, d: int, seed: int) -> np.ndarray:
    """i.i.d. U[0, 1)^d."""
    rng = np.random.default_rng(seed)
    return rng.random((d, n), dtype=np.float32)


def gaussian_mixture(n: int, d: int, k: int, sd: float, seed: int) -> np.ndarray:
    """k isotropic Gaussians, centres U[0,1)^d, standard deviation sd, equal weights."""
    rng = np.random.default_rng(seed)
    centres = rng.random((k, d))
    comp = rng.integers(0, k, size=n)
    x = centres[comp].T + sd * rng.standard_normal((d, n))
    return x.astype(np.float32)


def student_t_snapped(n: int, d: int, df: float, snap_frac: float, grid: int, seed: int) -> np.ndarray:
    """Per-coordinate Student-t(df), drawn in float64 and rounded to float32;
    each value independently with probability snap_frac is replaced by
    rint(x * grid) / grid (float32 arithmetic, round-half-even)."""
    rng = np.random.default_rng(seed)
    out = np.empty((d, n), np.float32)
    step = 1 << 22
    for j in range(d):
        for b in range(0, n, step):
            e = min(n, b + step)
            x = rng.standard_t(df, size=e - b).astype(np.float32)
            snap = rng.random(e - b) < snap_frac
            g = np.float32(grid)
            x[snap] = np.rint(x[snap] * g) / g
            out[j, b:e] = x
    return out


def mvn_common_corr(n: int, d: int, rho: float, seed: int) -> np.ndarray:
    """Multivariate normal, mean 0, unit variances, common correlation rho
    (the simulation study of Sec. 5)."""
    rng = np.random.default_rng(seed)
    cov = np.full((d, d), rho) + (1.0 - rho) * np.eye(d)
    chol = np.linalg.cholesky(cov)
    z = rng.standard_normal((d, n))
    return (chol @ z).astype(np.float32)


def mvn_probit(n: int, d: int, rho: float, seed: int) -> np.ndarray:
    """Host version of mvn_probit_device's recipe (a different random stream)."""
    from scipy.special import ndtr
    z = mvn_common_corr(n, d, rho, seed).astype(np.float64)
    return np.clip(ndtr(z), 2.0 ** -24, 1.0 - 2.0 ** -24).astype(np.float32)


def uniform_open(n: int, d: int, seed: int) -> np.ndarray:
    """Uniform on the open cube (0,1)^d: k / 2^24 with k uniform on
    1 .. 2^24 - 1 (exact in float32, never 0 or 1)."""
    rng = np.random.default_rng(seed)
    return (rng.integers(1, 1 << 24, size=(d, n)) / float(1 << 24)).astype(np.float32)


def explicit_sids(n: int, r: int, seed: int) -> np.ndarray:
    """Subset ids uniform on [0, r); uint8 when r <= 256 else uint16."""
    rng = np.random.default_rng(seed)
    dt = np.uint8 if r <= 256 else np.uint16
    return rng.integers(0, r, size=n).astype(dt)


# ------------------------------------------------------------- device (torch)


def uniform_device(n: int, d: int, seed: int, device="cuda"):
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    return torch.rand((d, n), generator=g, device=device, dtype=torch.float32)


def gaussian_mixture_device(n: int, d: int, k: int, sd: float, seed: int, device="cuda"):
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    centres = torch.rand((k, d), generator=g, device=device, dtype=torch.float64)
    comp = torch.randint(0, k, (n,), generator=g, device=device)
    x = torch.randn((d, n), generator=g, device=device, dtype=torch.float32)
    x.mul_(sd).add_(centres[comp].T.to(torch.float32))
    return x


def student_t_snapped_device(n: int, d: int, df: float, snap_frac: float, grid: int, seed: int,
                             device="cuda"):
    """Student-t as Z / sqrt(V/df), V ~ chi^2_df = 2 Gamma(df/2), in float64 per chunk."""
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    out = torch.empty((d, n), device=device, dtype=torch.float32)
    step = 1 << 24
    for j in range(d):
        for b in range(0, n, step):
            e = min(n, b + step)
            m = e - b
            z = torch.randn(m, generator=g, device=device, dtype=torch.float64)
            # chi-square(df) for integer df as a sum of squared normals
            v = torch.zeros(m, device=device, dtype=torch.float64)
            for _ in range(int(df)):
                w = torch.randn(m, generator=g, device=device, dtype=torch.float64)
                v.add_(w * w)
            x = (z / torch.sqrt(v / df)).to(torch.float32)
            snap = torch.rand(m, generator=g, device=device) < snap_frac
            gr = torch.tensor(float(grid), device=device, dtype=torch.float32)
            x = torch.where(snap, torch.round(x * gr) / gr, x)
            out[j, b:e] = x
    return out


def mvn_common_corr_device(n: int, d: int, rho: float, seed: int, device="cuda"):
    """Multivariate normal, mean 0, unit variances, common correlation rho, drawn
    on the device (float64 Cholesky factor applied to float64 normals)."""
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    cov = np.full((d, d), rho) + (1.0 - rho) * np.eye(d)
    chol = torch.from_numpy(np.linalg.cholesky(cov)).to(device)
    out = torch.empty((d, n), device=device, dtype=torch.float32)
    step = 1 << 24
    for b in range(0, n, step):
        e = min(n, b + step)
        z = torch.randn((d, e - b), generator=g, device=device, dtype=torch.float64)
        out[:, b:e] = (chol @ z).to(torch.float32)
    return out


def uniform_open_device(n: int, d: int, seed: int, device="cuda"):
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    k = torch.randint(1, 1 << 24, (d, n), generator=g, device=device, dtype=torch.int32)
    return k.to(torch.float32) / float(1 << 24)


def mvn_probit_device(n: int, d: int, rho: float, seed: int, device="cuda"):
    """Sec. 5's trivariate normal mapped into (0,1)^d coordinate by coordinate
    by the standard normal CDF (in float64), clamped to [2^-24, 1 - 2^-24]."""
    import torch
    x = mvn_common_corr_device(n, d, rho, seed, device)
    out = torch.empty_like(x)
    step = 1 << 24
    lo, hi = 2.0 ** -24, 1.0 - 2.0 ** -24
    for b in range(0, n, step):
        e = min(n, b + step)
        z = x[:, b:e].to(torch.float64)
        out[:, b:e] = (0.5 * torch.erfc(-z / np.sqrt(2.0))).clamp_(lo, hi).to(torch.float32)
    return out


def explicit_sids_device(n: int, r: int, seed: int, device="cuda"):
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    dt = torch.uint8 if r <= 256 else torch.int16
    return torch.randint(0, r, (n,), generator=g, device=device).to(dt)


# --------------------------------------------------------- named configurations


@dataclass
class TreeSpec:
    """One build request: data recipe plus build parameters."""
    name: str
    n: int
    d: int
    dist: str                 # "uniform" | "mixture16" | "mixture8" | "student_t" | "mvn"
    seed: int
    r: int
    subset_mode: int          # 0 mod, 1 contiguous, 2 explicit
    key_rule: int             # 0 cyclic, 1 widest spread
    depth: int = 0            # > 0 fixed depth; 0 leaf mode
    leaf_size: int = 1
    max_levels: int = 24
    sid_seed: Optional[int] = None
    rho: float = 0.0
    fourier_j: int = 0        # > 0: the Fourier-moment estimator with J harmonics
    extra: dict = field(default_factory=dict)

    def points(self) -> np.ndarray:
        if self.dist == "uniform":
            return uniform(self.n, self.d, self.seed)
        if self.dist == "mixture16":
            return gaussian_mixture(self.n, self.d, 16, 0.05, self.seed)
        if self.dist == "mixture8":
            return gaussian_mixture(self.n, self.d, 8, 0.05, self.seed)
        if self.dist == "student_t":
            return student_t_snapped(self.n, self.d, 3.0, 0.1, 256, self.seed)
        if self.dist == "mvn":
            return mvn_common_corr(self.n, self.d, self.rho, self.seed)
        if self.dist == "uniform_open":
            return uniform_open(self.n, self.d, self.seed)
        if self.dist == "mvn_probit":
            return mvn_probit(self.n, self.d, self.rho, self.seed)
        raise ValueError(self.dist)

    def points_device(self, device="cuda"):
        if self.dist == "uniform":
            return uniform_device(self.n, self.d, self.seed, device)
        if self.dist == "mixture16":
            return gaussian_mixture_device(self.n, self.d, 16, 0.05, self.seed, device)
        if self.dist == "mixture8":
            return gaussian_mixture_device(self.n, self.d, 8, 0.05, self.seed, device)
        if self.dist == "student_t":
            return student_t_snapped_device(self.n, self.d, 3.0, 0.1, 256, self.seed, device)
        if self.dist == "mvn":
            return mvn_common_corr_device(self.n, self.d, self.rho, self.seed, device)
        if self.dist == "uniform_open":
            return uniform_open_device(self.n, self.d, self.seed, device)
        if self.dist == "mvn_probit":
            return mvn_probit_device(self.n, self.d, self.rho, self.seed, device)
        raise ValueError(self.dist)

    def sids(self):
        if self.subset_mode != 2:
            return None
        return explicit_sids(self.n, self.r, self.sid_seed if self.sid_seed is not None else self.seed + 1)

    def sids_device(self, device="cuda"):
        if self.subset_mode != 2:
            return None
        return explicit_sids_device(self.n, self.r,
                                    self.sid_seed if self.sid_seed is not None else self.seed + 1, device)

    def levels(self) -> int:
        return self.depth


def config1(n: int = 65536) -> TreeSpec:
    """Uniform [0,1)^3, r=8 subsets by index mod 8, cyclic keys, depth 10."""
    return TreeSpec("plain_uniform_n65536_d3_r8_depth10", n, 3, "uniform", 0, 8, 0, 0, depth=10)


def config2(n: int = 1 << 24, depth: int = 16) -> TreeSpec:
    """16-Gaussian mixture in [0,1)^3 (sd 0.05), r=64 contiguous subsets, cyclic, depth 16."""
    return TreeSpec(f"plain_mixture16_n{n}_d3_r64contig_depth{depth}", n, 3, "mixture16", 0, 64, 1, 0,
                    depth=depth)


def config3(n: int = 1 << 27, depth: int = 20) -> TreeSpec:
    """Student-t(3) in 8-D with 10% of values on a 1/256 grid, r=256 random
    explicit subsets, widest-spread keys, depth 20."""
    return TreeSpec(f"plain_studentt_n{n}_d8_r256explicit_widest_depth{depth}", n, 8, "student_t", 0,
                    256, 2, 1, depth=depth, sid_seed=1)


def paper_mvn_fourier(n: int, rho: float, depth: int, J: int, seed: int = 0) -> TreeSpec:
    """Sec. 5's shape for the paper's own estimator: the trivariate normal with
    common correlation rho mapped into (0,1)^3 by the normal CDF, cyclic keys,
    splits by the Fourier-moment estimator with J harmonics."""
    return TreeSpec(f"paper_mvn_fourier_rho{rho}_n{n}_depth{depth}_J{J}", n, 3, "mvn_probit", seed, 1, 0, 0,
                    depth=depth, rho=rho, fourier_j=J)


def leaf_mode_levels(n: int) -> int:
    """Output capacity (levels) requested for a leaf-mode tree of n points:
    two levels more than a perfectly balanced tree down to one point."""
    return int(min(30, max(4, int(np.ceil(np.log2(max(n, 2)))) + 2)))


def config4_batch(num_trees: int = 4096, n_lo: float = 8.0, n_hi: float = 20.0) -> list[TreeSpec]:
    """Independent trees: n = floor(2^U(8,20)), d in {2,3,8,16}, half uniform
    half 8-cluster mixture, r in {4,16,64} by index mod r, cyclic, leaf <= 32.
    Tree i draws its parameters and its points from seed i."""
    out = []
    for i in range(num_trees):
        rng = np.random.default_rng(i)
        n = int(np.floor(2.0 ** rng.uniform(n_lo, n_hi)))
        d = int(rng.choice([2, 3, 8, 16]))
        dist = "uniform" if rng.random() < 0.5 else "mixture8"
        r = int(rng.choice([4, 16, 64]))
        out.append(TreeSpec(f"batch{i}", n, d, dist, 1_000_000 + i, r, 0, 0, depth=0, leaf_size=32,
                            max_levels=leaf_mode_levels(n)))
    return out


def config5_stream(num_requests: int = 20000, rate: float = 100.0, n_lo: float = 10.0,
                   n_hi: float = 24.0, seed: int = 2):
    """Poisson stream of build requests: n = floor(2^U(10,24)), d in {3,16},
    half uniform half 8-cluster mixture, r=32 by index mod 32, leaf <= 64.
    Returns (arrival_times_seconds, specs)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=num_requests)
    t = np.cumsum(gaps)
    specs = []
    for i in range(num_requests):
        n = int(np.floor(2.0 ** rng.uniform(n_lo, n_hi)))
        d = int(rng.choice([3, 16]))
        dist = "uniform" if rng.random() < 0.5 else "mixture8"
        specs.append(TreeSpec(f"req{i}", n, d, dist, 2_000_000 + i, 32, 0, 0, depth=0, leaf_size=64,
                              max_levels=leaf_mode_levels(n)))
    return t, specs


def paper_mvn(n: int, rho: float, depth: int, seed: int = 0) -> TreeSpec:
    """Sec. 5 shape: trivariate normal, common correlation rho; r=64 by index
    mod 64, cyclic keys."""
    return TreeSpec(f"paper_mvn_rho{rho}_n{n}_depth{depth}", n, 3, "mvn", seed, 64, 0, 0, depth=depth,
                    rho=rho)
