"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This package holds none of the layered-field arithmetic: it only builds
triangle meshes (icosphere, jittered planar grid, noisy torus, a shuffled
numbering of any of them) and draws seed
vertices.  Every draw goes through one counter-based generator (SplitMix64,
Steele, Lea and Flood, OOPSLA 2014), so the same (seed, counter) pair gives the
same number on every machine.
"""
from .rng import splitmix64, uniform01, uniform
from .meshes import icosphere, planar_grid, noisy_torus, shuffled, Mesh
from .seeds import sample_seeds
from .jobs import JobSpec, batch_mix, serve_trace, make_mesh

__all__ = [
    "splitmix64", "uniform01", "uniform",
    "icosphere", "planar_grid", "noisy_torus", "shuffled", "Mesh",
    "sample_seeds",
    "JobSpec", "batch_mix", "serve_trace", "make_mesh",
]
