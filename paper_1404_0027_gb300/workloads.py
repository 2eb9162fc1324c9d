"""Seeded synthetic inputs shared by the tests, the oracle runs and the benchmark.

This module only draws random inputs (numpy PCG64) with the shapes and value
distributions of the paper's workloads and of the scaled-up service workloads;
it holds none of the selection method's arithmetic.  Both the CUDA path and the
CPU oracle receive the arrays built here.

Workloads
---------
* ``plain_uniform``   -- one propensity vector, M=1024, alpha ~ 1 - U[0,1) (FP64).
* ``skewed``          -- M=1029 (the size of the iron-homeostasis model the paper
                         motivates with, Introduction), alpha FP32 lognormal(0, 2)
                         with exactly round(0.3 M) zero entries at seeded positions.
* ``batched_uneven``  -- B realizations, M_b log-uniform in [64, 16384], alpha FP32
                         Exponential(1), K_b selections each.
* ``wide_range``      -- M=2^20, alpha FP32 = 10^U(-6, 6) (twelve decades).
* ``gaussian_paper``  -- the paper's test propensities (Section "Test and validation"):
                         D_j = 1e5 * phi(x_j), x_j = -5 + 10 j / (M - 1).
* ``random_network``  -- a random mass-action network (order 1 and 2 reactions,
                         net stoichiometry in {-2,-1,+1,+2}), with initial counts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Reaction types of the network format (shared vocabulary, no arithmetic).
RT_SOURCE = 0   # 0 -> products            h = 1
RT_UNI = 1      # A -> products            h = x_A
RT_BI = 2       # A + B -> products        h = x_A * x_B   (A != B)
RT_DIMER = 3    # 2A -> products           h = x_A (x_A - 1) / 2


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def plain_uniform(M: int = 1024, seed: int = 101) -> np.ndarray:
    """alpha_j = 1 - U[0,1) in (0, 1], FP64."""
    return (1.0 - _rng(seed).random(M)).astype(np.float64)


def skewed(M: int = 1029, seed: int = 200, zero_frac: float = 0.3,
           sigma: float = 2.0) -> np.ndarray:
    """FP32 lognormal(0, sigma) with exactly round(zero_frac * M) zeros."""
    g = _rng(seed)
    a = g.lognormal(0.0, sigma, M).astype(np.float32)
    nz = int(round(zero_frac * M))
    a[g.permutation(M)[:nz]] = 0.0
    return a


@dataclass
class Batch:
    alpha: np.ndarray        # concatenated propensities, FP32
    offsets: np.ndarray      # int64 [B+1], alpha_b = alpha[offsets[b]:offsets[b+1]]
    out_offsets: np.ndarray  # int64 [B+1], K_b = out_offsets[b+1] - out_offsets[b]

    @property
    def B(self) -> int:
        return len(self.offsets) - 1

    @property
    def sizes(self) -> np.ndarray:
        return np.diff(self.offsets)

    @property
    def ks(self) -> np.ndarray:
        return np.diff(self.out_offsets)


def batched_uneven(B: int = 4096, seed: int = 300, m_lo: int = 64,
                   m_hi: int = 16384, K: int | np.ndarray = 256,
                   dtype=np.float32) -> Batch:
    """B realizations, M_b = floor(exp(U(ln m_lo, ln m_hi))), alpha ~ Exp(1)."""
    g = _rng(seed)
    sizes = np.floor(np.exp(g.uniform(math.log(m_lo), math.log(m_hi), B))).astype(np.int64)
    sizes = np.clip(sizes, m_lo, m_hi)
    offsets = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    alpha = g.standard_exponential(int(offsets[-1])).astype(dtype)
    ks = np.broadcast_to(np.asarray(K, dtype=np.int64), (B,))
    out_offsets = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(ks, out=out_offsets[1:])
    return Batch(alpha, offsets, out_offsets)


def batch_from_vectors(vectors, ks) -> Batch:
    """Concatenate explicit per-realization vectors (used for edge cases)."""
    sizes = np.array([len(v) for v in vectors], dtype=np.int64)
    offsets = np.zeros(len(vectors) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    dt = vectors[0].dtype if len(vectors) else np.float32
    alpha = (np.concatenate(vectors).astype(dt) if len(vectors)
             else np.zeros(0, dtype=np.float32))
    ks = np.asarray(ks, dtype=np.int64)
    out_offsets = np.zeros(len(vectors) + 1, dtype=np.int64)
    np.cumsum(ks, out=out_offsets[1:])
    return Batch(alpha, offsets, out_offsets)


def wide_range(M: int = 1 << 20, seed: int = 400, lo_dec: float = -6.0,
               hi_dec: float = 6.0) -> np.ndarray:
    """FP32 alpha = 10^U(lo_dec, hi_dec)."""
    e = _rng(seed).uniform(lo_dec, hi_dec, M)
    return np.power(10.0, e).astype(np.float32)


def gaussian_paper(M: int) -> np.ndarray:
    """The paper's discrete Gaussian test propensities, FP64 (1e5 * N(0,1) density)."""
    x = -5.0 + np.arange(M, dtype=np.float64) * (10.0 / (M - 1))
    return 1e5 * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


@dataclass
class Network:
    """Mass-action network.  Propensity of reaction r: a_r = c_r * h_r(X)."""
    n_species: int
    rtype: np.ndarray      # int32 [M]
    reactants: np.ndarray  # int32 [M, 2]; -1 where unused
    rate: np.ndarray       # float64 [M]
    nu_ptr: np.ndarray     # int32 [M+1]  CSR of the net state change of each reaction
    nu_species: np.ndarray  # int32 [nnz]
    nu_delta: np.ndarray   # int32 [nnz]

    @property
    def M(self) -> int:
        return len(self.rtype)


def network_from_lists(n_species, reactions) -> Network:
    """reactions: list of (rtype, (A, B), rate, [(species, delta), ...])."""
    M = len(reactions)
    rtype = np.zeros(M, dtype=np.int32)
    reac = -np.ones((M, 2), dtype=np.int32)
    rate = np.zeros(M, dtype=np.float64)
    ptr = [0]
    sp, dl = [], []
    for r, (t, ab, c, nu) in enumerate(reactions):
        rtype[r] = t
        reac[r, 0], reac[r, 1] = ab
        rate[r] = c
        for s, d in nu:
            sp.append(s)
            dl.append(d)
        ptr.append(len(sp))
    return Network(n_species, rtype, reac, rate, np.array(ptr, dtype=np.int32),
                   np.array(sp, dtype=np.int32), np.array(dl, dtype=np.int32))


def random_network(N: int = 641, M: int = 1029, seed: int = 500,
                   p_types=(0.45, 0.40, 0.15), c_lo: float = 1e-3,
                   c_hi: float = 1e1) -> Network:
    """Random network: uni / bi / dimer reactions, products disjoint from reactants.

    Reactant species are consumed (-1 each, -2 for a dimer); one or two product
    species gain +1 or +2.  Rate constants are log-uniform on [c_lo, c_hi].
    """
    g = _rng(seed)
    reactions = []
    for _ in range(M):
        t = int(g.choice([RT_UNI, RT_BI, RT_DIMER], p=p_types))
        if t == RT_BI:
            a, b = (int(v) for v in g.choice(N, 2, replace=False))
            nu = [(a, -1), (b, -1)]
            used = {a, b}
            ab = (a, b)
        else:
            a = int(g.integers(N))
            nu = [(a, -2 if t == RT_DIMER else -1)]
            used = {a}
            ab = (a, -1)
        n_prod = int(g.integers(1, 3))
        for _p in range(n_prod):
            while True:
                s = int(g.integers(N))
                if s not in used:
                    break
            used.add(s)
            nu.append((s, int(g.choice([1, 2]))))
        c = float(10.0 ** g.uniform(math.log10(c_lo), math.log10(c_hi)))
        reactions.append((t, ab, c, nu))
    return network_from_lists(N, reactions)


def initial_counts(N: int, B: int, seed: int = 501, lo: int = 0,
                   hi: int = 100) -> np.ndarray:
    """int32 [B, N] counts drawn uniform on {lo..hi}."""
    return _rng(seed).integers(lo, hi + 1, size=(B, N)).astype(np.int32)
