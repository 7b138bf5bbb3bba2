"""GB300-native layered fields (Zayer et al., arXiv 1804.09152).

The time-iteration runs in the CUDA library ``_build/liblf.so`` behind the C
ABI of ``include/lf.h``; ``paper_1804_09152_gb300.lf`` is its ctypes binding.
``build()`` compiles the library for sm_103a.

A tessellation with Lloyd-like rounds and its dual mesh::

    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import lf
    with lf.Mesh(V, F) as mesh:              # V: (n_v, 3) float64, F: (n_f, 3) int32
        mesh.seed(seed_vertices)             # k distinct vertex ids
        mesh.step(2000)                      # time-iterations of Algorithm 1
        seeds = mesh.lloyd(10, 2000)         # seed updates, each followed by 2000 steps
        labels = mesh.labels()               # cell of every vertex (-1: base layer)
        triangles = mesh.extract_dual()      # dual mesh over the seed vertices

Many meshes at once: ``lf.lf_step_batch([m0, m1, ...], counts)``; a stream of
jobs under a memory budget: ``lf.Server``.  ``mesh.tune(32)`` times the step
kernel's five schedules on the job itself and keeps the fastest (they give the
same bits); ``mesh.set_schedule("hot")`` fixes one.
"""
from .native import build, LIB

__all__ = ["build", "LIB", "lf"]


def __getattr__(name):
    if name == "lf":
        from . import _lib
        return _lib
    raise AttributeError(name)
