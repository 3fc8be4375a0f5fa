"""Seeded synthetic workloads: the inputs of the benchmarks and tests.

Only input generation lives here (set sizes, kinds, seeds, arrival times);
none of the method's arithmetic.  The thesis's own workloads are synthetic
sprinklings too (Section "Simulations and Scaling Evaluations"), so nothing
here stands in for a dataset.  A sprinkled set's size is Poisson distributed
with mean nu * V (Appendix "Causal Set Sprinklings", general method).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0xC5E70000
KIND_2D_ORDER, KIND_2D_DIAMOND, KIND_4D_DIAMOND, KIND_3D_DIAMOND, KIND_2D_DS_SLAB = 0, 1, 2, 3, 4
KIND_2D_SQUARE, KIND_2D_CYLINDER = 5, 6

# name: (kind, n, seed, description)
SINGLE = {
    "2d_order_1024": (KIND_2D_ORDER, 1024, SEED_BASE + 1, "random 2D order, N=1024"),
    "4d_diamond_16384": (KIND_4D_DIAMOND, 16384, SEED_BASE + 2, "4D Minkowski diamond, N=16384, int32 grid 2^20"),
    "2d_order_131072": (KIND_2D_ORDER, 131072, SEED_BASE + 3, "random 2D order, N=131072 (2.1 GB bitset)"),
}


def ensemble(n2d=512, mean2d=4096, n4d=256, mean4d=2048, seed=SEED_BASE + 4):
    """Batched ensemble: n2d 2D diamonds with N ~ Poisson(mean2d) and n4d 4D
    diamonds with N ~ Poisson(mean4d); set s gets seed + 1 + s.
    Returns a list of (kind, n, seed)."""
    rng = np.random.default_rng(seed)
    sizes = list(rng.poisson(mean2d, n2d)) + list(rng.poisson(mean4d, n4d))
    kinds = [KIND_2D_DIAMOND] * n2d + [KIND_4D_DIAMOND] * n4d
    return [(k, max(int(n), 1), seed + 1 + s) for s, (k, n) in enumerate(zip(kinds, sizes))]


def serving_requests(rate=200.0, duration_s=5.0, log2_min=10, log2_max=16, seed=SEED_BASE + 5):
    """Poisson arrivals at `rate` per second for `duration_s`; N = floor(2^U),
    U uniform on [log2_min, log2_max]; kinds 50/50 random 2D order / 4D diamond;
    request r gets seed + 1 + r.  Returns a list of (t_arrival_s, kind, n, seed)."""
    rng = np.random.default_rng(seed)
    out, t, r = [], 0.0, 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s:
            return out
        n = int(np.floor(2.0 ** rng.uniform(log2_min, log2_max)))
        kind = KIND_2D_ORDER if rng.random() < 0.5 else KIND_4D_DIAMOND
        out.append((t, kind, n, seed + 1 + r))
        r += 1
