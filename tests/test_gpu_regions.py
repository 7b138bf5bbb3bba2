"""GPU parity of region seeds (Sec. 3.2) through lf_seed_regions: the initial
field is exact (integer decisions), the first steps from it match the oracle
under the tolerances of the other parity tests."""
import numpy as np
import pytest

import synth
from parity_util import ambiguous_rows, check_compare, compare, field_from_lib, to_f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lf():
    import paper_1804_09152_gb300 as pkg
    pkg.build()
    from paper_1804_09152_gb300 import _lib
    return _lib


@pytest.mark.parametrize("name,fac,k,sid", [
    ("grid61", lambda: synth.planar_grid(61, seed=2), 64, 3),
    ("torus50", lambda: synth.noisy_torus(50), 48, 5),
    ("ico3_crowded", lambda: synth.icosphere(3), 120, 4),     # many overlapping rings
])
def test_region_seeds_and_steps_match_the_oracle(lf, oracle_mod, name, fac, k, sid):
    m = fac()
    L = oracle_mod.cotan_laplacian(m.V, m.F)
    seeds = synth.sample_seeds(m.n_v, k, sid)
    F = oracle_mod.seed_regions(L, seeds, 1)
    with lf.Mesh(m.V, m.F) as mesh:
        mesh.seed_regions(seeds, 1)
        rp, lay, val = mesh.get_field()
        assert np.array_equal(rp, F.rowptr) and np.array_equal(lay, F.ids) and np.array_equal(val, F.vals)
        for t in range(3):
            F32 = to_f32(F, oracle_mod)
            Fo, sko, mg = oracle_mod.step(L, F32, {}, margins=True)
            mesh.set_field(F32.rowptr, F32.ids, F32.vals, F32.n_layers)
            sk0 = mesh.stats()["skeleton_total"]
            mesh.step(1)
            skg = mesh.stats()["skeleton_total"] - sk0
            r = compare(Fo, field_from_lib(*mesh.get_field(), F.n_layers, oracle_mod), ambiguous_rows(mg), oracle_mod)
            check_compare(r)
            assert abs(int(skg) - int(sko)) <= 16 * r["disagreeing_rows"], (t, skg, sko)
            F, _ = oracle_mod.step(L, F, {})


def test_region_seed_arguments(lf):
    m = synth.icosphere(2)
    with lf.Mesh(m.V, m.F) as mesh:
        for rings in (-1, 2):
            with pytest.raises(lf.LFError) as ei:
                mesh.seed_regions(synth.sample_seeds(m.n_v, 4, 1), rings)
            assert ei.value.status == lf.LF_ERR_INVALID
        mesh.seed_regions(synth.sample_seeds(m.n_v, 4, 1), 0)
        assert mesh.stats()["nnz"] == m.n_v
        seeds = mesh.lloyd(0, 0)                  # the seeds are remembered
        assert np.array_equal(seeds, synth.sample_seeds(m.n_v, 4, 1))
