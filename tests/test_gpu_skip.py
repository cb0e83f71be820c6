"""GPU parity of the learned subtree skip (each level-(L-4) subtree encoded,
flagged and stored only down to a predicted level) against the oracle's
statement of it.  The predicted levels are seeded inputs given to both sides
(hwfv1_set_skip_levels on the GPU, SkipState.skip_step on the CPU), so the
comparison is exact in float64: leaves, storage levels, stored and finest
fields, time and step, over runs that mix skip steps and exact audits."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _levels(rng, L, lo=None):
    Ls = L - 4
    n = 1 << Ls
    return rng.integers(Ls if lo is None else lo, L + 1, size=(n, n)).astype(np.uint8)


def _compare(sim, ref, k, exact=True):
    g = sim.fields()
    o = ref.fields()
    for q in ("h", "qx", "qy"):
        if exact:
            assert np.array_equal(g[q], o[q]), "step %d field %s: max diff %g" % (k, q, np.abs(g[q] - o[q]).max())
        else:
            scale = max(np.abs(o[q]).max(), 1e-300)
            assert np.abs(g[q] - o[q]).max() <= 1e-12 * scale, (k, q)
    assert np.array_equal(sim.skip_levels(1), ref.m.reshape(sim.skip_levels(1).shape)), "step %d levels" % k
    t, dt, n = sim.time()
    assert t == ref.t and n == ref.steps, k
    if exact:
        assert dt == ref.dt, k


def _run(p, f, level_seq, audit_K, exact=True):
    """Both sides through the same schedule: step s is an audit when
    s % audit_K == 0, else a skip step with level_seq[s]."""
    from paper_2206_05761_gb300.sim import Simulation
    sim = Simulation(p, f)
    ref = oracle.SkipState(p, f)
    assert sim.time()[1] == ref.dt
    for s, lev in enumerate(level_seq):
        sim.set_skip_levels(lev, audit_K=audit_K)        # the same interval: only the levels change
        sim.advance(max_steps=1)
        res = ref.plain_step(want=("leaves",)) if s % audit_K == 0 else ref.skip_step(lev, want=("leaves",))
        lv = sim.leaves()
        assert len(lv) == res["num_leaves"] and np.array_equal(lv, res["leaves"]), "step %d leaves" % s
        _compare(sim, ref, s, exact)
    sim.close()


@pytest.mark.parametrize("seed", [1, 2])
def test_random_levels_bumpy_dam_break(seed):
    rng = np.random.default_rng(seed)
    L = 7
    p, f = synth.bumpy_dam_break(L=L, eps=1e-3, seed=seed, eta_up=1.4)
    _run(p, f, [_levels(rng, L) for _ in range(12)], audit_K=5)


def test_random_levels_columns_flat_bed():
    rng = np.random.default_rng(3)
    L = 8
    p, f = synth.columns_dam_break(L=L, eps=1e-3, seed=4)
    _run(p, f, [_levels(rng, L) for _ in range(10)], audit_K=4)


def test_levels_held_and_changed_across_intervals():
    # the same levels kept over several skip steps (the stored subtrees then
    # stay at their level: no prolongation), then deeper, then shallower
    rng = np.random.default_rng(5)
    L = 7
    p, f = synth.bumpy_dam_break(L=L, eps=1e-3, seed=7, eta_up=1.6)
    a, b = _levels(rng, L), _levels(rng, L, lo=L - 1)
    _run(p, f, [a] * 4 + [b] * 3 + [a] * 3 + [np.full_like(a, L - 4)] * 3, audit_K=100)


def test_full_depth_levels_are_the_plain_step():
    from paper_2206_05761_gb300.sim import Simulation
    L = 7
    p, f = synth.bumpy_dam_break(L=L, eps=1e-3, seed=3)
    a, b = Simulation(p, f), Simulation(p, f)
    b.set_skip_levels(np.full((8, 8), L), audit_K=3)
    a.advance(max_steps=10)
    b.advance(max_steps=10)
    ga, gb = a.fields(), b.fields()
    for q in ga:
        assert np.array_equal(ga[q], gb[q])
    assert np.array_equal(a.leaves(), b.leaves())
    a.close()
    b.close()


def test_eps_zero_and_single_subtree_level():
    # eps = 0: every formed detail is significant; L = 5 has level-1 subtrees
    rng = np.random.default_rng(6)
    for p, f in (synth.circular_dam_break(L=6, eps=0.0), synth.circular_dam_break(L=5, eps=1e-3)):
        _run(p, f, [_levels(rng, p["L"]) for _ in range(6)], audit_K=3)


def test_wet_dry_inflow_and_friction():
    # the terrain flood's channel (inflow, Manning friction, dry banks) at
    # L = 8: fields within 1e-12 (friction), leaves and levels exact
    rng = np.random.default_rng(8)
    L = 8
    p, f = synth.terrain_flood(L=L, fill=2.0, fill_q=1.0)
    _run(p, f, [_levels(rng, L) for _ in range(6)], audit_K=3, exact=False)


def test_larger_grid_L10():
    rng = np.random.default_rng(9)
    L = 10
    p, f = synth.bumpy_dam_break(L=L, eps=1e-3, seed=11, eta_up=1.5)
    _run(p, f, [_levels(rng, L, lo=L - 2) for _ in range(4)], audit_K=3)


def test_rejects_levels_out_of_range_and_unsupported_problems():
    from paper_2206_05761_gb300 import hwfv1 as H
    from paper_2206_05761_gb300.sim import Simulation
    p, f = synth.bumpy_dam_break(L=6, eps=1e-3)
    sim = Simulation(p, f)
    for bad in (np.full((4, 4), 1), np.full((4, 4), 7)):
        with pytest.raises(H.Hwfv1Error):
            sim.set_skip_levels(bad, audit_K=3)
    sim.close()
    sim = Simulation(dict(p, flux_match=True), f)
    with pytest.raises(H.Hwfv1Error):
        sim.set_skip_levels(np.full((4, 4), 6), audit_K=3)
    sim.close()


def test_reading_the_fields_leaves_the_run_unchanged():
    # the finest fields of a state stored above level L are formed in the
    # other buffer: reading them after every step changes nothing
    from paper_2206_05761_gb300.sim import Simulation
    rng = np.random.default_rng(12)
    L = 7
    p, f = synth.bumpy_dam_break(L=L, eps=1e-3, seed=13, eta_up=1.3)
    seq = [_levels(rng, L) for _ in range(9)]
    a, b = Simulation(p, f), Simulation(p, f)
    for lev in seq:
        for s in (a, b):
            s.set_skip_levels(lev, audit_K=4)
            s.advance(max_steps=1)
        b.fields()
    ga, gb = a.fields(), b.fields()
    for q in ga:
        assert np.array_equal(ga[q], gb[q])
    assert np.array_equal(a.skip_levels(1), b.skip_levels(1))
    a.close()
    b.close()


def test_phases_refused_and_profiled_skip_step():
    from paper_2206_05761_gb300 import hwfv1 as H
    from paper_2206_05761_gb300.sim import Simulation
    L = 7
    p, f = synth.bumpy_dam_break(L=L, eps=1e-3, seed=3)
    sim = Simulation(p, f)
    sim.set_skip_levels(np.full((8, 8), L - 2), audit_K=3)
    with pytest.raises(H.Hwfv1Error) as e:
        sim.encode()
    assert e.value.status == 7                       # HWFV1_ERR_STATE
    names = [n for n, _ in H.hwfv1_profile_step(sim.hd)]     # the audit step
    assert names[0] == "k_skip_finest" and names[1] == "k_clear_words" and names[-1] == "k_decode_finish"
    names = [n for n, _ in H.hwfv1_profile_step(sim.hd)]     # a skip step
    assert names[:2] == ["k_clear_words", "k_skip_encode"] and names[-1] == "k_skip_decode"
    ref = oracle.SkipState(p, f)
    ref.plain_step()
    ref.skip_step(np.full((8, 8), L - 2))
    g, o = sim.fields(), ref.fields()
    for q in g:
        assert np.array_equal(g[q], o[q])
    sim.close()
