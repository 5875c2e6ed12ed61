"""Seeded synthetic inputs for the NMC sweep: random CNF / QAP instances and beta profiles.

This module is shared by the oracle, the CUDA path, the tests and the bench. It builds
*inputs only* (instances and inverse-temperature profiles) and holds none of the method's
arithmetic: no energy, no move, no random number the sweep itself draws, no acceptance rule.

Every random draw comes from SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used in counter form: draw j of stream `seed` is
mix(seed + (j + 1) * GAMMA). That makes the inputs identical on every machine and numpy
version, unlike numpy's distribution methods.

Workload shapes follow the paper's problem classes: uniform random k-SAT with M = round(alpha*N)
clauses of k distinct variables and Bernoulli(1/2) signs (Sec. "4-SAT Problems Near
Computational Phase Transitions": N=5000, alpha=9.884 gives 49,420 clauses), and Koopmans-Beckmann
QAP with symmetric flow and distance matrices (Sec. "Quadratic Assignment Problems").
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK32 = np.uint64(0xFFFFFFFF)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset..offset+n-1 of the SplitMix64 stream for `seed` (uint64 array)."""
    with np.errstate(over="ignore"):
        j = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + j * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, n, self.pos)
        self.pos += n
        return out

    def below(self, bound, n: int) -> np.ndarray:
        """n integers in [0, bound) by multiply-shift of the high 32 bits (bound <= 2^32)."""
        hi = self.u64(n) >> np.uint64(32)
        b = np.asarray(bound, dtype=np.uint64)
        return ((hi * b) >> np.uint64(32)).astype(np.int64)

    def unit(self, n: int) -> np.ndarray:
        """n doubles uniform in [0, 1) from the top 53 bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def n_clauses(n_vars: int, alpha: float) -> int:
    """M = round(alpha * N), the convention that makes N=5000, alpha=9.884 give 49,420."""
    return int(np.floor(alpha * n_vars + 0.5))


def random_ksat(n_vars: int, alpha: float, k: int, seed: int) -> np.ndarray:
    """Uniform random k-SAT: int32 [M, k], DIMACS literals +-(var+1).

    Each clause takes k distinct variables uniformly (rows with a repeated variable are
    redrawn from fresh draws of the same stream) and each literal is negated with
    probability 1/2.
    """
    if k < 1 or k > n_vars:
        raise ValueError("need 1 <= k <= n_vars")
    m = n_clauses(n_vars, alpha)
    s = Stream(seed)
    var = s.below(n_vars, m * k).reshape(m, k)
    while True:
        srt = np.sort(var, axis=1)
        bad = np.nonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1))[0]
        if bad.size == 0:
            break
        var[bad] = s.below(n_vars, bad.size * k).reshape(bad.size, k)
    neg = (s.u64(m * k) >> np.uint64(63)).astype(np.int64).reshape(m, k)
    lits = (var + 1) * (1 - 2 * neg)
    return lits.astype(np.int32)


def linear_profile(b0: float, b1: float, n_steps: int) -> np.ndarray:
    """beta(t) = b0 + (b1 - b0) t / (T - 1), float64 [T]."""
    if n_steps == 1:
        return np.array([b0], dtype=np.float64)
    t = np.arange(n_steps, dtype=np.float64)
    return b0 + (b1 - b0) * t / (n_steps - 1)


def geometric_profile(b0: float, b1: float, n_steps: int) -> np.ndarray:
    """beta(t) = b0 (b1/b0)^(t/(T-1)), float64 [T]."""
    if n_steps == 1:
        return np.array([b0], dtype=np.float64)
    t = np.arange(n_steps, dtype=np.float64)
    return b0 * np.power(b1 / b0, t / (n_steps - 1))


def seeded_subset(n_units: int, frac: float, seed: int) -> np.ndarray:
    """Boolean mask of round(frac * n) units chosen by a seeded shuffle (sort by draw)."""
    keys = splitmix64(seed, n_units)
    order = np.argsort(keys, kind="stable")
    mask = np.zeros(n_units, dtype=bool)
    mask[order[: int(np.floor(frac * n_units + 0.5))]] = True
    return mask


def beta_inhomogeneous_linear(n_units, n_steps, b0, b1, frac, scale, seed) -> np.ndarray:
    """float32 [n_units, n_steps]: linear b0->b1; a seeded `frac` subset scaled by `scale`
    for the whole run (the backbone-heated profile of the sampling stage)."""
    base = linear_profile(b0, b1, n_steps)
    mask = seeded_subset(n_units, frac, seed)
    fac = np.where(mask, scale, 1.0)
    return (fac[:, None] * base[None, :]).astype(np.float32)


def beta_frozen_ramp(n_units, n_steps, b0, b1, frac, scale, seed) -> np.ndarray:
    """float32 [n_units, n_steps]: geometric b0->b1; a seeded `frac` subset runs at `scale`x
    for the first half, then its factor ramps linearly from `scale` at t=T/2 to 1 at t=T-1."""
    base = geometric_profile(b0, b1, n_steps)
    mask = seeded_subset(n_units, frac, seed)
    t = np.arange(n_steps, dtype=np.float64)
    half = n_steps // 2
    ramp = np.full(n_steps, scale, dtype=np.float64)
    if n_steps - 1 > half:
        ramp[half:] = scale + (1.0 - scale) * (t[half:] - half) / (n_steps - 1 - half)
    else:
        ramp[half:] = 1.0
    fac = np.where(mask[:, None], ramp[None, :], 1.0)
    return (fac * base[None, :]).astype(np.float32)


def beta_scaled_linear(n_units, n_steps, b0, b1, lo, hi, seed) -> np.ndarray:
    """float32 [n_units, n_steps]: linear b0->b1 times a per-unit factor uniform in [lo, hi]."""
    base = linear_profile(b0, b1, n_steps)
    fac = lo + (hi - lo) * Stream(seed).unit(n_units)
    return (fac[:, None] * base[None, :]).astype(np.float32)


def beta_constant(n_units, n_steps, beta) -> np.ndarray:
    return np.full((n_units, n_steps), beta, dtype=np.float32)


def random_qap(n: int, seed: int, max_entry: int = 99, flow_zero_frac: float = 0.5):
    """Symmetric F (flows) and D (distances), int32 [n, n], zero diagonals.

    Off-diagonal entries are uniform in [0, max_entry]; each off-diagonal flow pair is
    additionally set to zero with probability `flow_zero_frac`.
    """
    s = Stream(seed)
    iu = np.triu_indices(n, 1)
    npair = iu[0].size
    f = s.below(max_entry + 1, npair)
    d = s.below(max_entry + 1, npair)
    zero = s.unit(npair) < flow_zero_frac
    f = np.where(zero, 0, f)
    F = np.zeros((n, n), dtype=np.int32)
    D = np.zeros((n, n), dtype=np.int32)
    F[iu] = f
    D[iu] = d
    F = F + F.T
    D = D + D.T
    return F, D


# ----------------------------------------------------------------------------------------
# Named workloads (seeds: instance 1000+i, schedule 2000+i)
# ----------------------------------------------------------------------------------------

def workload_ksat_small(n_steps: int = 1000):
    """Random 4-SAT N=200, M=1920 (alpha 9.6), 64 replicas, beta linear 0.5->4.0 with a
    seeded 30% subset at 0.5x; Philox seed 1."""
    n = 200
    lits = random_ksat(n, 9.6, 4, 1001)
    beta = beta_inhomogeneous_linear(n, n_steps, 0.5, 4.0, 0.30, 0.5, 2001)
    return dict(name="4sat_n200_m1920_r64", lits=lits, n_vars=n, beta=beta, replicas=64,
                n_steps=n_steps, seed=1)


def workload_ksat_large(n_steps: int = 5000, n_vars: int = 50_000):
    """Random 4-SAT N=50,000, M=480,000 (alpha 9.6), 1024 replicas, beta geometric 0.3->6.0
    with a seeded 20% subset held at 0.4x for the first half, then ramped to 1x."""
    lits = random_ksat(n_vars, 9.6, 4, 1002)
    beta = beta_frozen_ramp(n_vars, n_steps, 0.3, 6.0, 0.20, 0.4, 2002)
    return dict(name=f"4sat_n{n_vars}_m{lits.shape[0]}_r1024", lits=lits, n_vars=n_vars,
                beta=beta, replicas=1024, n_steps=n_steps, seed=2)


def workload_ksat_batch(n_instances: int = 256, n_steps: int = 2000, n_min=1000, n_max=20000,
                        r_min=32, r_max=256, seed=1003):
    """Uneven batch: each instance 3-SAT (alpha 4.2) or 4-SAT (alpha 9.6) with p=1/2,
    N uniform in [n_min, n_max], replicas uniform in [r_min, r_max], beta as the small
    workload (linear 0.5->4.0, 30% at 0.5x)."""
    s = Stream(seed)
    kind = s.below(2, n_instances)
    ns = n_min + s.below(n_max - n_min + 1, n_instances)
    rs = r_min + s.below(r_max - r_min + 1, n_instances)
    out = []
    for i in range(n_instances):
        k, alpha = (3, 4.2) if kind[i] == 0 else (4, 9.6)
        n = int(ns[i])
        lits = random_ksat(n, alpha, k, seed * 1000 + i)
        beta = beta_inhomogeneous_linear(n, n_steps, 0.5, 4.0, 0.30, 0.5, seed * 2000 + i)
        out.append(dict(lits=lits, n_vars=n, beta=beta, replicas=int(rs[i]), n_steps=n_steps,
                        seed=10_000 + i, k=k))
    return out


def workload_ksat_mix(n_instances: int = 256, n_steps: int = 2000, mix=((3, 4.2), (4, 9.6)),
                      seed: int = 1003):
    """The uneven batch of the batched benchmark: instance i is kind mix[j] (k, alpha) with j
    drawn uniformly, N uniform in [1000, 20000], replicas uniform in [32, 256], Philox seed
    10,000 + i; a factored schedule: base[t] linear 0.5 -> 4.0 over n_steps, factor[u] 0.5 on a
    seeded 30% of the variables and 1 elsewhere (beta[u][t] = float32(factor[u] * base[t]))."""
    s = Stream(seed)
    kind = s.below(len(mix), n_instances)
    ns = 1000 + s.below(19001, n_instances)
    rs_n = 32 + s.below(225, n_instances)
    base = linear_profile(0.5, 4.0, n_steps).astype(np.float32)
    out = []
    for i in range(n_instances):
        k, alpha = mix[int(kind[i])]
        n = int(ns[i])
        lits = random_ksat(n, alpha, k, seed * 1000 + i)
        factor = np.where(seeded_subset(n, 0.3, seed * 2000 + i), 0.5, 1.0).astype(np.float32)
        out.append(dict(lits=lits, n=n, k=k, factor=factor, base=base, R=int(rs_n[i]),
                        seed=10_000 + i))
    return out


def workload_qap_batch(n_instances: int = 64, n_steps: int = 10_000, n_min=32, n_max=256,
                       replicas=4096, seed=1004):
    """QAP batch: n uniform in [n_min, n_max], F,D symmetric uniform [0,99] (F half zeros),
    beta linear 0.01->1.0 times a per-facility factor uniform in [0.5, 1.5]."""
    s = Stream(seed)
    ns = n_min + s.below(n_max - n_min + 1, n_instances)
    out = []
    for i in range(n_instances):
        n = int(ns[i])
        F, D = random_qap(n, seed * 1000 + i)
        beta = beta_scaled_linear(n, n_steps, 0.01, 1.0, 0.5, 1.5, seed * 2000 + i)
        out.append(dict(F=F, D=D, n=n, beta=beta, replicas=replicas, n_steps=n_steps,
                        seed=20_000 + i))
    return out
