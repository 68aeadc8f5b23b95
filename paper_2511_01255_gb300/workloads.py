"""Seeded synthetic inputs shaped like the paper's design problems.

This module only draws inputs (problem sizes, phase mismatches, random genes,
sign words, relaxed parameters); it holds none of the method's arithmetic, so
both the CUDA path's tests and the oracle's tests may use it.

The paper's own workloads (PPLN at given pump wavelengths, Sec. 5) need
dispersion data it does not give, so the mismatches here are synthetic
kappa = dk * w values in the same range (coherence lengths of 0.65-4 domain
widths), with N spanning the paper's 660-13200 domains and up to 1e5.
"""
import math

import numpy as np

TWO_PI = 2.0 * math.pi

# (name, N, kappa1, kappa2, NP, G, F, CR, compensated)
SMALL = dict(name="n16_np32_g200", N=16, kappa1=TWO_PI / 7.0, kappa2=TWO_PI / 1.6, NP=32,
             G=200, F=0.5, CR=0.9, compensated=0, seed=1)
PAPER_SCALE = dict(name="n1000_np256_g2000", N=1000, kappa1=TWO_PI / 6.9, kappa2=TWO_PI / 1.55,
                   NP=256, G=2000, F=0.5, CR=0.9, compensated=1, seed=1)
PRECISION = dict(name="n100000_np1024_g500", N=100000, kappa1=TWO_PI / 6.9,
                 kappa2=TWO_PI / 1.55, NP=1024, G=500, F=0.5, CR=0.9, compensated=1, seed=1)
RELAXED = dict(name="b4096_n4096", B=4096, N=4096, kappa1=TWO_PI / 6.9, kappa2=TWO_PI / 1.55,
               seed=1)


def batched_instances(n=512, seed=1):
    """Independent instances: N ~ U[500, 8000], kappa1 ~ U[2pi/8, 2pi/6],
    kappa2 ~ U[2pi/2, 2pi/1.3], NP uniform over {64, 128, 256, 512}, G = 1000."""
    rng = np.random.default_rng(seed)
    N = rng.integers(500, 8001, n)
    k1 = rng.uniform(TWO_PI / 8.0, TWO_PI / 6.0, n)
    k2 = rng.uniform(TWO_PI / 2.0, TWO_PI / 1.3, n)
    NP = rng.choice([64, 128, 256, 512], n)
    return [dict(N=int(N[i]), kappa1=float(k1[i]), kappa2=float(k2[i]), NP=int(NP[i]), G=1000,
                 F=0.5, CR=0.9, compensated=0, seed=seed) for i in range(n)]


def random_genes(NP, N, seed=0, ld=None):
    """Genes U(-1, 1) as float32 [NP, ld] (columns beyond N are zero)."""
    rng = np.random.default_rng(seed)
    ld = N if ld is None else ld
    X = np.zeros((NP, ld), dtype=np.float32)
    X[:, :N] = rng.uniform(-1.0, 1.0, (NP, N)).astype(np.float32)
    return X


def pack_signs(X, N):
    """Bit (j % 32) of word j // 32 set where gene j is negative."""
    NP = X.shape[0]
    W = (N + 31) // 32
    neg = np.zeros((NP, W * 32), dtype=np.uint64)
    neg[:, :N] = (X[:, :N] < 0).astype(np.uint64)
    words = (neg.reshape(NP, W, 32) << np.arange(32, dtype=np.uint64)).sum(axis=2)
    return words.astype(np.uint32)


def alternating(N):
    return np.where(np.arange(N) % 2 == 0, 1.0, -1.0).astype(np.float32)


def relaxed_theta(B, N, seed=1):
    """theta ~ N(0, 1), float32 [B, N]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((B, N)).astype(np.float32)


def two_tone_signs(N, kappa1, kappa2):
    """A +-1 row (float32 [N]) whose sign follows cos(kappa1 j) + cos(kappa2 j)
    (+1 where the sum is zero): a sequence carrying both phase-mismatch
    frequencies, so that both integrals of the cascade grow with the length and
    |d_eff| is a sizeable fraction of L^2/2 (about 0.07 at the paper-scale
    mismatches) instead of the ~N of a random row."""
    j = np.arange(N, dtype=np.float64)
    s = np.cos(kappa1 * j) + np.cos(kappa2 * j)
    return np.where(s < 0.0, -1.0, 1.0).astype(np.float32)


# The multi-wavelength designs of Sec. 5: a 9 mm crystal of 3 um domains (N = 3000),
# NP = 5000 and 1000 iterations (the paper's experimental protocol); synthetic
# mismatches stand in for the PPLN dispersion the paper does not give.
DESIGN_THG3 = dict(name="multi_thg_k3_n3000_np5000_g1000", N=3000, NP=5000, G=1000, F=0.5, CR=0.9,
                   seed=1, kind=2, G0=2.0e6, beta=0.5,
                   kappas=[(TWO_PI / 6.5, TWO_PI / 1.4), (TWO_PI / 6.9, TWO_PI / 1.55),
                           (TWO_PI / 7.4, TWO_PI / 1.7)])
DESIGN_SHG5 = dict(name="multi_shg_k5_n3000_np5000_g1000", N=3000, NP=5000, G=1000, F=0.5, CR=0.9,
                   seed=1, kind=3, G0=2.0e3, beta=0.5,
                   kappas=[(TWO_PI / x, 0.0) for x in (2.1, 2.6, 3.2, 3.7, 4.4)])
