"""Job mixes for the batching and serving forms.

Each job is a mesh (kind and size), a seed count, a storage type and a step
count, all drawn from one SplitMix64 stream; the meshes themselves come from
synth.meshes.  Nothing here computes layered fields.

batch_mix: 64 jobs, icosphere or noisy torus with probability 1/2 each,
n_v log-uniform in [10k, 600k] (an icosphere snaps to the nearest level 4..8,
a torus takes side round(sqrt(n_v))), k log-uniform in [32, 2048], FP32 or
BF16 with probability 1/2, 1000 steps each.

serve_trace: Poisson arrivals at `rate` jobs/s until `n_jobs` jobs or
`duration` seconds; n_v log-normal with median sqrt(5k * 2M) whose +-2.326
sigma range is [5k, 2M], clipped to it; kind uniform over icosphere, torus
and grid; k log-uniform in [16, 8192] (at most n_v / 4); steps uniform in
{500, ..., 3000}; with probability 1/2 (a stream of its own, seed + 1) the job
also asks for 5 Lloyd-like rounds and the dual mesh.
"""
import math
from dataclasses import dataclass

import numpy as np

from .rng import uniform01
from .meshes import icosphere, noisy_torus, planar_grid

ICO_LEVELS = (4, 5, 6, 7, 8, 9)


@dataclass(frozen=True)
class JobSpec:
    kind: str            # "ico", "torus" or "grid"
    size: int            # icosphere level, or grid side
    k: int               # seeds
    dtype: str           # "f32", "bf16" or "f16"
    steps: int
    seed_stream: int     # stream of the seed vertices
    arrival: float = 0.0 # seconds from the start of the trace
    lloyd_rounds: int = 0
    dual: bool = False

    @property
    def n_v(self):
        return 10 * 4 ** self.size + 2 if self.kind == "ico" else self.size * self.size


def _log_uniform(u, lo, hi):
    return math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))


def _snap_ico(n_v, levels):
    return min(levels, key=lambda L: abs(math.log(10 * 4 ** L + 2) - math.log(n_v)))


def batch_mix(n_jobs=64, seed=6, steps=1000, nv_range=(10_000, 600_000), k_range=(32, 2048)):
    u = uniform01(seed, np.arange(4 * n_jobs, dtype=np.uint64)).reshape(n_jobs, 4)
    jobs = []
    for i in range(n_jobs):
        n_v = _log_uniform(u[i, 1], *nv_range)
        if u[i, 0] < 0.5:
            kind, size = "ico", _snap_ico(n_v, ICO_LEVELS[:5])
        else:
            kind, size = "torus", int(round(math.sqrt(n_v)))
        k = int(round(_log_uniform(u[i, 2], *k_range)))
        dtype = "f32" if u[i, 3] < 0.5 else "bf16"
        jobs.append(JobSpec(kind, size, k, dtype, steps, 1000 + i))
    return jobs


def serve_trace(n_jobs=2000, seed=7, rate=200.0, duration=60.0, nv_range=(5_000, 2_000_000),
                k_range=(16, 8192), steps_range=(500, 3000)):
    u = uniform01(seed, np.arange(6 * n_jobs, dtype=np.uint64)).reshape(n_jobs, 6)
    extra = uniform01(seed + 1, np.arange(n_jobs, dtype=np.uint64))
    median = math.sqrt(nv_range[0] * nv_range[1])
    sigma = math.log(nv_range[1] / nv_range[0]) / (2 * 2.326)
    jobs, t = [], 0.0
    for i in range(n_jobs):
        t += -math.log(1.0 - u[i, 0]) / rate
        if t > duration:
            break
        # Box-Muller normal from two uniforms
        z = math.sqrt(-2.0 * math.log(1.0 - u[i, 1])) * math.cos(2.0 * math.pi * u[i, 2])
        n_v = min(max(median * math.exp(sigma * z), nv_range[0]), nv_range[1])
        kind = ("ico", "torus", "grid")[min(2, int(u[i, 3] * 3))]
        size = _snap_ico(n_v, ICO_LEVELS) if kind == "ico" else int(round(math.sqrt(n_v)))
        spec_nv = 10 * 4 ** size + 2 if kind == "ico" else size * size
        k = min(int(round(_log_uniform(u[i, 4], *k_range))), spec_nv // 4)
        steps = steps_range[0] + min(steps_range[1] - steps_range[0], int(u[i, 5] * (steps_range[1] - steps_range[0] + 1)))
        full = extra[i] < 0.5
        jobs.append(JobSpec(kind, size, k, "f32", steps, 2000 + i, t, 5 if full else 0, full))
    return jobs


def make_mesh(spec):
    """The synthetic mesh of a job (grid jitter stream 2, torus noise stream 4)."""
    if spec.kind == "ico":
        return icosphere(spec.size)
    if spec.kind == "torus":
        return noisy_torus(spec.size)
    return planar_grid(spec.size, jitter=0.2, seed=2)
