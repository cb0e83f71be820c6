"""The seeded input generators (synth/): the same seed gives the same fields
bit for bit, another seed gives other fields, and every generator returns
contiguous float64 arrays of the finest grid with non-negative depths
(no GPU)."""
import numpy as np
import pytest

import synth

SEEDED = {
    "bumpy": lambda s: synth.bumpy_dam_break(L=6, seed=s),
    "columns": lambda s: synth.columns_dam_break(L=6, seed=s),
    "terrain": lambda s: synth.terrain_flood(L=7, seed=s),
    "dry_bed_rough": lambda s: synth.dry_bed_dam_break(L=6, relief=0.05, seed=s),
    "lake": lambda s: synth.lake_at_rest(L=5, seed=s),
    "mound": lambda s: synth.wet_mound(L=5, seed=s),
    "inflow": lambda s: synth.inflow_basin(L=5, seed=s),
}

FIXED = {
    "circle": lambda: synth.circular_dam_break(L=5),
    "pseudo2d": lambda: synth.pseudo_2d_dam_break(L=5),
    "ritter": lambda: synth.ritter_dam_break(L=5),
    "uniform": lambda: synth.uniform_flow(L=4),
}


def _check_shapes(p, f):
    n = 1 << p["L"]
    for k in ("h", "qx", "qy", "z"):
        a = f[k]
        assert a.shape == (n, n) and a.dtype == np.float64 and a.flags.c_contiguous, k
        assert np.all(np.isfinite(a)), k
    assert f["h"].min() >= 0.0


@pytest.mark.parametrize("name", sorted(SEEDED))
def test_seeded_generators_are_reproducible(name):
    make = SEEDED[name]
    (p1, f1), (p2, f2), (_, f3) = make(11), make(11), make(12)
    _check_shapes(p1, f1)
    assert p1 == p2
    for k in ("h", "qx", "qy", "z"):
        assert np.array_equal(f1[k].view(np.uint64), f2[k].view(np.uint64)), k
    assert any(not np.array_equal(f1[k], f3[k]) for k in ("h", "qx", "qy", "z"))


@pytest.mark.parametrize("name", sorted(FIXED))
def test_fixed_generators_are_well_formed(name):
    p, f = FIXED[name]()
    _check_shapes(p, f)


def test_ensemble_is_reproducible_and_mixes_levels():
    a, b = synth.ensemble(count=12, seed=4), synth.ensemble(count=12, seed=4)
    assert [p["L"] for p, _ in a] == [p["L"] for p, _ in b]
    assert len({p["L"] for p, _ in a}) > 1
    for (pa, fa), (pb, fb) in zip(a, b):
        assert np.array_equal(fa["h"], fb["h"]) and np.array_equal(fa["z"], fb["z"])
