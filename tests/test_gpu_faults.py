"""Failures injected on the host: an allocator that refuses memory.

The mesh's lf_device hooks go through torch's caching allocator but refuse
any request once a byte budget would be exceeded.  Nothing here faults the
GPU: the library sees a NULL from its allocator and must return LF_ERR_OOM
with every byte it took given back (creation), or keep its state and resume
exactly where it stopped once memory is there again (growth of the field
buffers during lf_step, seeding).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib
    return _lib


class BudgetDevice:
    """lf_device on torch's allocator that refuses requests beyond `budget` bytes."""

    def __init__(self, lf, budget=None):
        import torch
        self.stream = torch.cuda.current_stream()
        self.budget, self.used, self.refused, self.live = budget, 0, 0, {}

        def _alloc(nbytes, cuda_stream, user):
            if self.budget is not None and self.used + nbytes > self.budget:
                self.refused += 1
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), self.stream.device.index or 0, self.stream)
            self.live[p] = nbytes
            self.used += nbytes
            return p

        def _free(ptr, user):
            self.used -= self.live.pop(ptr)
            torch.cuda.caching_allocator_delete(ptr)

        d = lf.lf_device()
        d.cuda_stream = self.stream.cuda_stream
        d.alloc = lf._ALLOC_FN(_alloc)
        d.free = lf._FREE_FN(_free)
        d.user = None
        d._keep = (d.alloc, d.free)
        self.dev = d


def test_creation_refused_at_every_point_gives_everything_back(lf):
    m = synth.planar_grid(61, seed=2)
    probe = BudgetDevice(lf)
    with lf.Mesh(m.V, m.F, device=probe.dev) as mesh:
        full = probe.used                      # what a created mesh holds
        peak = max(full, mesh.stats()["device_bytes"])
    assert probe.used == 0
    # budgets that cut creation at its successive allocations
    for frac in (0.0, 0.05, 0.2, 0.4, 0.6, 0.8, 0.95):
        bd = BudgetDevice(lf, int(frac * peak))
        with pytest.raises(lf.LFError) as ei:
            lf.Mesh(m.V, m.F, device=bd.dev)
        assert ei.value.status == lf.LF_ERR_OOM, frac
        assert bd.refused >= 1 and bd.used == 0 and not bd.live, frac


def test_growth_refused_then_resumed_is_bit_exact(lf):
    t = synth.noisy_torus(40)
    seeds = synth.sample_seeds(t.n_v, 32, 5)
    with lf.Mesh(t.V, t.F, initial_capacity=t.n_v) as ref:         # the run without failures
        ref.seed(seeds)
        ref.step(200)
        want = ref.get_field()
        want_stats = ref.stats()
    bd = BudgetDevice(lf)
    mesh = lf.Mesh(t.V, t.F, initial_capacity=t.n_v, device=bd.dev)
    try:
        mesh.seed(seeds)
        mesh.step(1)
        bd.budget = bd.used                    # no byte more: the first growth is refused
        with pytest.raises(lf.LFError) as ei:
            mesh.step(199)
        assert ei.value.status == lf.LF_ERR_OOM and bd.refused >= 1
        st = mesh.stats()
        assert 1 <= st["steps"] < 200 and bd.used == bd.budget
        bd.budget = None                       # memory is back
        mesh.step(200 - st["steps"])
        got = mesh.get_field()
        for x, y in zip(want, got):
            assert np.array_equal(x, y)
        assert mesh.stats()["skeleton_total"] == want_stats["skeleton_total"]
    finally:
        mesh.close()
    assert bd.used == 0


def test_seeding_refused_keeps_the_mesh_usable(lf):
    m = synth.icosphere(3)
    seeds = synth.sample_seeds(m.n_v, 16, 1)
    bd = BudgetDevice(lf)
    with lf.Mesh(m.V, m.F, device=bd.dev) as mesh:
        mesh.seed(seeds)
        mesh.step(50)
        before = mesh.get_field()
        bd.budget = bd.used                    # seeding needs a small upload buffer
        with pytest.raises(lf.LFError) as ei:
            mesh.seed(seeds)
        assert ei.value.status == lf.LF_ERR_OOM
        for x, y in zip(before, mesh.get_field()):
            assert np.array_equal(x, y)        # the field is untouched
        bd.budget = None
        mesh.seed(seeds)
        mesh.step(50)
        for x, y in zip(before, mesh.get_field()):
            assert np.array_equal(x, y)
