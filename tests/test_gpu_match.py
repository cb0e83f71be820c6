"""GPU parity of the conservative variant (matched fluxes at resolution
changes, HWFV1_FLUX_MATCH) against the oracle's R-match reading: bit-exact
in float64 without friction, 1e-12 relative with Manning friction; mass
conservation on the GPU; quiescent-tile skipping stays exact."""
import numpy as np
import pytest

import oracle
import synth

from test_gpu_parity import RTOL_FRICTION, _compare_fields, _sim, one_step_parity

pytestmark = pytest.mark.gpu


def _fm(p):
    return dict(p, flux_match=True)


def _closed_circle(L):
    p, f = synth.circular_dam_break(L=L, eps=1e-3)
    p["bc"] = ("closed",) * 4
    return _fm(p), f


def _wet_bumps(L):
    p, f = synth.wet_mound(L=L, eps=1e-3)
    return _fm(p), f


@pytest.mark.parametrize("L", [3, 5, 6])
def test_matched_circular_dam_break(L):
    p, f = _closed_circle(L)
    one_step_parity(p, f, pre_steps=10)


@pytest.mark.parametrize("seed", [2, 11])
def test_matched_bumpy_dam_break_wet_dry(seed):
    p, f = synth.bumpy_dam_break(L=7, eps=1e-3, seed=seed)
    one_step_parity(_fm(p), f, pre_steps=5)


def test_matched_terrain_flood_with_friction_and_inflow():
    p, f = synth.terrain_flood(L=7)
    one_step_parity(_fm(p), f, exact=False, pre_steps=30)


def test_matched_non_square_open_domain():
    p, f = synth.pseudo_2d_dam_break(L=7, eps=1e-3)
    one_step_parity(_fm(p), f, pre_steps=3)


def test_matched_trajectory_conserves_mass():
    # graph replay (hwfv1_advance) against the oracle's loop, and the
    # volume of a closed, fully wet adaptive basin held to rounding
    p, f = _wet_bumps(7)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    cell = (p["lx"] / (1 << 7)) * (p["ly"] / (1 << 7))
    v0 = float(f["h"].sum()) * cell
    for chunk in range(6):
        sim.advance(max_steps=10)
        for _ in range(9):
            ref.step()
        res = ref.step(want=("leaves",))
        assert np.array_equal(sim.leaves(), res["leaves"]), "chunk %d" % chunk
        assert len(set((res["leaves"] >> 28).tolist())) >= 2
        _compare_fields(sim, ref)
        assert sim.time()[:2] == (ref.t, ref.dt)
    v = float(sim.fields()["h"].sum()) * cell
    assert abs(v - v0) <= 1e-13 * v0
    sim.close()


def test_matched_with_quiescent_tiles_equals_full_sweep():
    p, f = synth.dry_bed_dam_break(L=8, eps=1e-3, relief=0.05)
    p = _fm(p)
    sim = _sim(p, f)
    full = _sim(dict(p, full_sweep=True), f)
    ref = oracle.State(p, f)
    for chunk in range(4):
        sim.advance(max_steps=10)
        full.advance(max_steps=10)
        for _ in range(9):
            ref.step()
        res = ref.step(want=("leaves",))
        assert np.array_equal(sim.leaves(), res["leaves"]), "chunk %d" % chunk
        _compare_fields(sim, ref)
        _compare_fields(full, ref)
    _, lu, au, _, _ = sim.counters()
    assert au < lu
    sim.close()
    full.close()


def test_matched_profiled_step_is_an_ordinary_step():
    # the shared-face kernels with the walk over finer halves, and the flag
    # words they read, in a step launched kernel by kernel
    from paper_2206_05761_gb300 import hwfv1 as Hh
    p, f = _closed_circle(6)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    names = [n for n, _ in Hh.hwfv1_profile_step(sim.hd)]
    assert "k_flag" in names and "k_fv1_faces" in names and "k_fv1_update" in names
    ref.step()
    _compare_fields(sim, ref)
    sim.close()


def test_matched_full_size_terrain_flood_L12():
    # the 4096 x 4096 terrain flood with its channel flowing, two steps
    p, f = synth.terrain_flood(L=12, fill=2.0, fill_q=1.0)
    p = _fm(p)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    sim.advance(max_steps=2)
    ref.step()
    res = ref.step(want=("leaves",))
    lv = sim.leaves()
    assert len(lv) == res["num_leaves"] and np.array_equal(lv, res["leaves"])
    _compare_fields(sim, ref, exact=False)
    t, dt, steps = sim.time()
    assert steps == 2 and abs(dt - ref.dt) <= RTOL_FRICTION * ref.dt
    sim.close()


def test_matched_rejected_with_batches_and_learned_lookahead():
    from paper_2206_05761_gb300 import hwfv1 as H
    from paper_2206_05761_gb300.sim import Ensemble
    p, f = _closed_circle(6)
    with pytest.raises(Exception):
        Ensemble([(p, f)])
    sim = _sim(p, f)
    net = H.hwfv1_skipnet_create(3)
    with pytest.raises(Exception):
        sim.set_skipnet(net)
    H.hwfv1_skipnet_destroy(net)
    sim.close()


def test_matched_full_size_wet_domain_one_step():
    # 4096 x 4096 bumpy dam-break: more queued leaves than the shared-face
    # buffer holds, so the matched update takes its one-pass form
    p, f = synth.bumpy_dam_break(L=12, eps=1e-3)
    one_step_parity(_fm(p), f)
