"""The exact leaf-value store (hwfv1_set_leaf_store): flat-bed subtrees are
stored at their deepest leaf level, encoded from there and decoded only down
to there.  Its results must be the plain method's bit for bit, so it is
compared with the plain oracle step by step: leaves, fields, time and step,
on flat beds at zero and above zero, wet/dry, with inflow and friction, next
to uneven beds, and across switching the store on and off."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _flat_shift(case, c):
    """The same case over a bed raised to the constant c everywhere."""
    p, f = case
    return p, dict(f, z=f["z"] + c)


def _run(p, f, steps, exact=True, toggle=None, expect_coarse=True):
    from paper_2206_05761_gb300.sim import Simulation
    sim = Simulation(p, f)
    ref = oracle.State(p, f)
    sim.set_leaf_store(True)
    coarse = False
    for s in range(steps):
        if toggle and s in toggle:
            sim.set_leaf_store(toggle[s])
        sim.advance(max_steps=1)
        res = ref.step(want=("leaves",))
        lv = sim.leaves()
        assert len(lv) == res["num_leaves"] and np.array_equal(lv, res["leaves"]), "step %d leaves" % s
        g = sim.fields()
        for q in ("h", "qx", "qy"):
            o = getattr(ref, q)
            if exact:
                assert np.array_equal(g[q], o), "step %d %s: %g" % (s, q, np.abs(g[q] - o).max())
            else:
                assert np.abs(g[q] - o).max() <= 1e-12 * max(np.abs(o).max(), 1e-300), (s, q)
        t, dt, n = sim.time()
        assert n == ref.steps and t == ref.t, s
        if exact:
            assert dt == ref.dt
        coarse = coarse or bool((sim.skip_levels(1) < p["L"]).any())
    if expect_coarse:
        assert coarse                       # some subtree was stored above the finest level
    sim.close()


@pytest.mark.parametrize("case", ["columns", "circular", "columns_raised"])
def test_flat_beds_match_the_plain_oracle(case):
    make = {"columns": lambda: synth.columns_dam_break(L=8, eps=1e-3, seed=3),
            "circular": lambda: synth.circular_dam_break(L=7, eps=1e-3),
            "columns_raised": lambda: _flat_shift(synth.columns_dam_break(L=7, eps=1e-3, seed=5), 0.3)}[case]
    p, f = make()
    _run(p, f, 25)


def test_pseudo2d_dam_break_smooth_and_vigorous_phases():
    p, f = synth.pseudo_2d_dam_break(L=8, eps=1e-3)
    _run(p, f, 40)


def test_dry_bed_wet_dry_front():
    p, f = synth.dry_bed_dam_break(L=8, eps=1e-3)
    _run(p, f, 30)


def test_uneven_beds_and_inflow_are_stored_at_the_finest_level():
    # humps: no subtree is flat, so everything stays at L (the plain step);
    # inflow over humps likewise
    p, f = synth.bumpy_dam_break(L=7, eps=1e-3, seed=2)
    _run(p, f, 12, expect_coarse=False)
    p, f = synth.inflow_basin(L=6, eps=1e-3)
    _run(p, f, 12, expect_coarse=False)


def test_friction_on_a_flat_bed():
    p, f = synth.columns_dam_break(L=7, eps=1e-3, seed=7)
    _run(dict(p, manning_n=0.03), f, 15, exact=False)


def test_switching_the_store_on_and_off():
    p, f = synth.columns_dam_break(L=7, eps=1e-3, seed=9)
    _run(p, f, 20, toggle={5: False, 9: True, 15: False, 17: True})


def test_rejects_zero_eps():
    from paper_2206_05761_gb300 import hwfv1 as H
    from paper_2206_05761_gb300.sim import Simulation
    p, f = synth.columns_dam_break(L=6, eps=0.0)
    sim = Simulation(p, f)
    with pytest.raises(H.Hwfv1Error):
        sim.set_leaf_store(True)
    sim.close()
