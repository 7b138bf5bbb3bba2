"""Seed vertices drawn uniformly without replacement.

Partial Fisher-Yates shuffle of 0..n_v-1 driven by SplitMix64: at position t
the element is swapped with position t + (x_t mod (n_v - t)), x_t being output
t of the stream ``seed``.  Layer id of a seed = its position in the result.
"""
import numpy as np

from .rng import splitmix64


def sample_seeds(n_v, k, seed):
    if not (1 <= k <= n_v):
        raise ValueError(f"need 1 <= k <= n_v, got k={k}, n_v={n_v}")
    x = splitmix64(seed, np.arange(k, dtype=np.uint64))
    perm = np.arange(n_v, dtype=np.int64)
    for t in range(k):
        j = t + int(x[t] % np.uint64(n_v - t))
        perm[t], perm[j] = perm[j], perm[t]
    return perm[:k].astype(np.int32)
