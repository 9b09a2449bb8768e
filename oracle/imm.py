"""IMM seed selection, written plainly from Tang, Shi and Xiao, "Influence
Maximization in Near-Linear Time: A Martingale Approach" (SIGMOD 2015), over
the oracle's RR sets and greedy (test infrastructure only).

The paper's Section 2 names IMM as the state-of-the-art RIS algorithm whose
sample complexity theta fixes the number of RR sets; the sampler is its inner
step.  Readings (also stated in include/fbpt.h, fbpt_imm):
  - natural logarithms; ln C(n, k) as a sum of logs of exact quotients;
  - ell is first raised to ell * (1 + ln 2 / ln n) (IMM's adjustment for the
    two phases);
  - the estimation rounds are i = 1 .. ceil(log2 n) - 1;
  - each round extends the sample to ceil(lambda' / x) RR sets (sample ids
    0, 1, ... under one seed; earlier sets are kept, never redrawn);
  - theta = ceil(lambda* / LB); the final selection runs over theta RR sets
    drawn afresh (sample ids after those of the estimation rounds): Chen
    (2018) showed that reusing the estimation sets, as the original IMM does,
    breaks the martingale argument behind the guarantee.
"""
from __future__ import annotations

import math

import numpy as np

from . import RRSets, greedy, rr_sets

E = 2.718281828459045  # the double nearest e (math.e)


def log_binom(n: float, k: float) -> float:
    """ln C(n, k) as the sum over i < min(k, n - k) of ln((n - i) / (i + 1))."""
    kk = min(k, n - k)
    s, i = 0.0, 0.0
    while i < kk:
        s += math.log((n - i) / (i + 1.0))
        i += 1.0
    return s


def imm_params(n: int, k: int, epsilon: float, ell: float):
    """(eps', lambda', lambda*) of IMM for n vertices and k seeds."""
    n = float(n)
    ln_n = math.log(n)
    ellp = ell * (1.0 + math.log(2.0) / ln_n)
    epsp = math.sqrt(2.0) * epsilon
    L = log_binom(n, float(k))
    lam_p = (2.0 + 2.0 * epsp / 3.0) * (L + ellp * ln_n + math.log(math.log2(n))) * n / (epsp * epsp)
    alpha = math.sqrt(ellp * ln_n + math.log(2.0))
    beta = math.sqrt((1.0 - 1.0 / E) * (L + ellp * ln_n + math.log(2.0)))
    ab = (1.0 - 1.0 / E) * alpha + beta
    lam_s = 2.0 * n * ab * ab / (epsilon * epsilon)
    return epsp, lam_p, lam_s


class _Sample:
    """The growing sample R: RR sets of sample ids 0 .. size-1."""

    def __init__(self, g, seed):
        self.g, self.seed = g, seed
        self.offsets = np.zeros(1, np.uint64)
        self.verts = np.zeros(0, np.uint32)

    @property
    def size(self):
        return self.offsets.size - 1

    def extend(self, target):
        if target <= self.size:
            return
        add = rr_sets(self.g, self.seed, self.size, target - self.size)
        self.offsets = np.concatenate([self.offsets[:-1], add.offsets + self.offsets[-1]])
        self.verts = np.concatenate([self.verts, add.verts])

    def rr(self):
        return RRSets(self.offsets, self.verts)


def imm(g, k: int, epsilon: float, ell: float, seed: int):
    """(seeds[k], gains[k], info) following IMM's sampling phase, then greedy."""
    n = g.n
    epsp, lam_p, lam_s = imm_params(n, k, epsilon, ell)
    R = _Sample(g, seed)
    LB, rounds = 1.0, 0
    for i in range(1, math.ceil(math.log2(n))):
        x = n / 2.0 ** i
        R.extend(math.ceil(lam_p / x))
        seeds, gains = greedy(n, R.rr(), k)
        rounds = i
        F = int(gains.sum()) / R.size
        if n * F >= (1.0 + epsp) * x:
            LB = n * F / (1.0 + epsp)
            break
    theta = math.ceil(lam_s / LB)
    final = rr_sets(g, seed, R.size, theta)
    seeds, gains = greedy(n, final, k)
    info = {"theta": theta, "samples": theta, "lower_bound": LB, "coverage": int(gains.sum()) / theta,
            "lambda_prime": lam_p, "lambda_star": lam_s, "rounds": rounds, "first_final_id": R.size}
    return seeds, gains, info
