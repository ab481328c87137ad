"""Seeded synthetic diagonal-GMM workloads (numpy PCG64).

This module only draws random numbers: it holds none of the method's
arithmetic and is the one piece of code that both the oracle-side tests and
the CUDA-side tests/bench use.  Every workload is a diagonal Gaussian mixture:
labels ~ Categorical(w), x = mu_label + sigma_label * z, z ~ N(0, I), stored
as float32 [N][D] (one sample per row).

Workloads (shapes of the paper's experiments, Sec. 5, and of the benchmark):
  c1   N=100000,   D=10,  G=8     w~Dir(1),   mu~U[-5,5], sigma~U[0.5,2]
  c2   N=2000000,  D=60,  G=256   w~Dir(0.5); speech-like 20 base dims with
       mu~N(0, 2^2), sigma~U[0.3,3], then 20 "delta" dims (mu = mu_base/2 +
       N(0, 0.5^2), sigma = sigma_base/2) and 20 "delta-delta" dims
       (mu = mu_base/4 + N(0, 0.25^2), sigma = sigma_base/4)
  c3   N=10000000, D=128, G=1024  w~Dir(1), mu~N(0, 3^2), sigma log-uniform
       on [0.1, 10]
  batched fit j: N log-uniform on [1000, 200000], D in {13,39,64},
       G in {8,16,32,64,128}, distributions of c1, seed 40000+j
  fig1 the two-cluster example program of Sec. 4.1 (Fig. 1): D=5, N=10000,
       mean1 = (1..5), mean2 = mean1 + 2, unit noise, pattern 1,1,2
  initialiser sets: c1-style mixtures at (D, G), P points each drawn on the
       GPU by draw_sets_torch (many sets of 4096 points are too slow to draw
       with numpy)
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Mixture:
    hefts: np.ndarray   # [G]
    means: np.ndarray   # [G][D]
    stds: np.ndarray    # [G][D]


def _draw(rng, mix: Mixture, N: int, chunk: int = 1 << 20):
    G, D = mix.means.shape
    X = np.empty((N, D), np.float32)
    labels = np.empty(N, np.int32)
    cdf = np.cumsum(mix.hefts)
    cdf /= cdf[-1]
    for s in range(0, N, chunk):
        n = min(chunk, N - s)
        lab = np.searchsorted(cdf, rng.random(n), side="right").astype(np.int32)
        lab = np.minimum(lab, G - 1)
        z = rng.standard_normal((n, D), dtype=np.float32)
        X[s:s + n] = mix.means[lab].astype(np.float32) + mix.stds[lab].astype(np.float32) * z
        labels[s:s + n] = lab
    return X, labels


def mixture_c1(rng, D: int, G: int) -> Mixture:
    w = rng.dirichlet(np.ones(G))
    mu = rng.uniform(-5.0, 5.0, (G, D))
    sd = rng.uniform(0.5, 2.0, (G, D))
    return Mixture(w, mu, sd)


def mixture_c2(rng, D: int = 60, G: int = 256) -> Mixture:
    assert D % 3 == 0
    b = D // 3
    w = rng.dirichlet(np.full(G, 0.5))
    mu_b = rng.normal(0.0, 2.0, (G, b))
    sd_b = rng.uniform(0.3, 3.0, (G, b))
    mu = np.concatenate([mu_b, 0.5 * mu_b + rng.normal(0.0, 0.5, (G, b)),
                         0.25 * mu_b + rng.normal(0.0, 0.25, (G, b))], axis=1)
    sd = np.concatenate([sd_b, 0.5 * sd_b, 0.25 * sd_b], axis=1)
    return Mixture(w, mu, sd)


def mixture_c3(rng, D: int = 128, G: int = 1024) -> Mixture:
    w = rng.dirichlet(np.ones(G))
    mu = rng.normal(0.0, 3.0, (G, D))
    sd = np.exp(rng.uniform(np.log(0.1), np.log(10.0), (G, D)))
    return Mixture(w, mu, sd)


def make(kind: str, N: int | None = None, D: int | None = None, G: int | None = None,
         seed: int | None = None):
    """Return (X float32 [N][D], labels int32 [N], Mixture) for a workload."""
    if kind == "c1":
        N, D, G = N or 100000, D or 10, G or 8
        rng = np.random.default_rng(1001 if seed is None else seed)
        mix = mixture_c1(rng, D, G)
    elif kind == "c2":
        N, D, G = N or 2000000, D or 60, G or 256
        rng = np.random.default_rng(1002 if seed is None else seed)
        mix = mixture_c2(rng, D, G)
    elif kind == "c3":
        N, D, G = N or 10000000, D or 128, G or 1024
        rng = np.random.default_rng(1003 if seed is None else seed)
        mix = mixture_c3(rng, D, G)
    elif kind == "fig1":
        N, D = N or 10000, D or 5
        X = np.empty((N, D), np.float32)
        rng = np.random.default_rng(7 if seed is None else seed)
        m1 = np.arange(1, D + 1, dtype=np.float64)
        m2 = m1 + 2.0
        lab = np.array([0 if (i % 3) < 2 else 1 for i in range(N)], np.int32)
        X[:] = (np.where(lab[:, None] == 0, m1, m2) + rng.standard_normal((N, D))).astype(np.float32)
        mix = Mixture(np.array([2 / 3, 1 / 3]), np.stack([m1, m2]), np.ones((2, D)))
        return X, lab, mix
    else:
        raise ValueError(kind)
    X, lab = _draw(rng, mix, N)
    return X, lab, mix


def separated(N: int, D: int, G: int, seed: int, gap: float = 12.0):
    """Well-separated mixture: component means on a lattice >= gap std apart."""
    rng = np.random.default_rng(seed)
    w = rng.dirichlet(np.full(G, 5.0))
    mu = np.zeros((G, D))
    for g in range(G):
        mu[g, g % D] = gap * (1 + g // D) * (1 if g % 2 == 0 else -1)
    mu += rng.uniform(-1, 1, (G, D))
    sd = rng.uniform(0.5, 1.0, (G, D))
    mix = Mixture(w, mu, sd)
    X, lab = _draw(rng, mix, N)
    return X, lab, mix


def batched_fit(j: int, n_lo: int = 1000, n_hi: int = 200000):
    """Fit j of the batched workload: its own seeded c1-style mixture."""
    rng = np.random.default_rng(40000 + j)
    N = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
    D = int(rng.choice([13, 39, 64]))
    G = int(rng.choice([8, 16, 32, 64, 128]))
    mix = mixture_c1(rng, D, G)
    X, lab = _draw(rng, mix, N)
    return X, lab, mix


def draw_sets_torch(mixtures, P: int, seed: int, device="cuda"):
    """P points of each of the given mixtures, drawn on `device` with a torch
    generator seeded `seed`: labels ~ Categorical(w), x = mu + sigma z.
    Returns a float32 tensor [len(mixtures)][P][D]."""
    import torch
    gen = torch.Generator(device=device).manual_seed(int(seed))
    w = torch.tensor(np.stack([m.hefts for m in mixtures]), dtype=torch.float64, device=device)
    mu = torch.tensor(np.stack([m.means for m in mixtures]), dtype=torch.float32, device=device)
    sd = torch.tensor(np.stack([m.stds for m in mixtures]), dtype=torch.float32, device=device)
    B, G, D = mu.shape
    lab = torch.multinomial(w, P, replacement=True, generator=gen)          # [B][P]
    z = torch.randn((B, P, D), generator=gen, device=device, dtype=torch.float32)
    idx = lab.unsqueeze(-1).expand(B, P, D)
    return torch.gather(mu, 1, idx) + torch.gather(sd, 1, idx) * z


def seeds_subset(X: np.ndarray, G: int, seed: int):
    """Pick G distinct rows uniformly (numpy RNG); used to give both sides the
    same explicit starting means in step-level parity tests."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(X.shape[0], size=G, replace=False)
    return np.asarray(X[idx], dtype=np.float64)
