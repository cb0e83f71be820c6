"""Batched ensembles: every member advanced by the batched launches must
match the oracle bit for bit, whatever launch configuration the autotuner
picks."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _cases():
    # mixed depths, including L < 5 (one tile) and different problems
    return [synth.bumpy_dam_break(L=6, eps=1e-3, seed=21),
            synth.circular_dam_break(L=2, eps=1e-3),
            synth.circular_dam_break(L=5, eps=1e-3),
            synth.bumpy_dam_break(L=7, eps=1e-4, seed=22, eta_up=1.6),
            synth.inflow_basin(L=4, eps=1e-3, q=0.01),
            synth.lake_at_rest(L=3, eps=1e-3, wet=False)]


def _check_members(ens, cases, steps):
    for d, (p, f) in enumerate(cases):
        ref = oracle.State(p, f)
        for _ in range(steps - 1):
            ref.step()
        res = ref.step(want=("leaves",))
        g = ens.member_fields(d)
        for k in ("h", "qx", "qy"):
            assert np.array_equal(g[k], getattr(ref, k)), "member %d field %s" % (d, k)
        assert np.array_equal(ens.member_leaves(d), res["leaves"]), "member %d leaves" % d
        t, dt, n = ens.member_time(d)
        assert n == steps and t == ref.t and dt == ref.dt


def test_batch_matches_oracle_per_member():
    from paper_2206_05761_gb300.sim import Ensemble
    cases = _cases()
    ens = Ensemble(cases)
    ens.advance(max_steps=12)
    _check_members(ens, cases, 12)
    assert ens.launches_per_step() <= 16
    ens.close()


def test_batch_members_at_the_benched_depths():
    # the benched ensemble's deeper members (L = 9 and 10: 256 and 1024
    # tiles, other tile paths than the small members) next to a small one,
    # with the autotuner's choice, against the oracle
    from paper_2206_05761_gb300.sim import Ensemble
    cases = [synth.bumpy_dam_break(L=10, eps=1e-3, seed=4, eta_up=1.7),
             synth.bumpy_dam_break(L=9, eps=1e-3, seed=5, eta_up=0.8),
             synth.bumpy_dam_break(L=7, eps=1e-3, seed=6, eta_up=1.2)]
    ens = Ensemble(cases)
    ens.advance(max_steps=4)
    _check_members(ens, cases, 4)
    ens.autotune(trial_steps=1)               # 12 candidates x 2 steps
    _check_members(ens, cases, 28)
    ens.close()


def test_autotune_keeps_results_bit_identical():
    from paper_2206_05761_gb300.sim import Ensemble
    cases = _cases()
    a = Ensemble(cases)
    choice = a.autotune(trial_steps=1)        # 12 candidates x 2 steps = 24 steps
    assert choice[0] in (3, 4, 5) and choice[1] in (8, 32, 128, 512)
    _check_members(a, cases, 24)
    a.advance(max_steps=3)
    _check_members(a, cases, 27)
    a.close()


def test_batch_t_end_per_member():
    from paper_2206_05761_gb300.sim import Ensemble
    cases = [synth.circular_dam_break(L=5, eps=1e-3), synth.bumpy_dam_break(L=6, eps=1e-3, seed=3)]
    ens = Ensemble(cases)
    ens.advance(t_end=0.01, max_steps=100)
    for d, (p, f) in enumerate(cases):
        ref = oracle.State(p, f)
        n = ref.run(t_end=0.01)
        t, dt, steps = ens.member_time(d)
        assert t == 0.01 and steps == n
        g = ens.member_fields(d)
        assert np.array_equal(g["h"], ref.h)
    ens.close()


def test_batch_float32_matches_single_domain_path():
    # float32 members have no shared-face buffer: the batched update takes
    # the one-pass kernel body; every member must equal the single-domain
    # float32 run bit for bit (fields, leaves, time)
    from paper_2206_05761_gb300.sim import Ensemble, Simulation
    cases = _cases()[:4]
    ens = Ensemble(cases, 32)
    ens.advance(max_steps=15)
    for d, (p, f) in enumerate(cases):
        sim = Simulation(p, f, 32)
        sim.advance(max_steps=15)
        g, s = ens.member_fields(d), sim.fields()
        for k in ("h", "qx", "qy"):
            assert g[k].dtype == s[k].dtype
            assert np.array_equal(g[k], s[k]), "member %d field %s" % (d, k)
        assert np.array_equal(ens.member_leaves(d), sim.leaves()), "member %d leaves" % d
        assert tuple(ens.member_time(d)) == tuple(sim.time())
        sim.close()
    ens.close()


def test_batch_member_refuses_the_skip_modes():
    # the batched kernels read a member's finest leaves; a member stored
    # above level L (learned skip, exact leaf-value store) would break them
    import paper_2206_05761_gb300.hwfv1 as H
    from paper_2206_05761_gb300.sim import Ensemble
    ens = Ensemble([synth.bumpy_dam_break(L=7, eps=1e-3, seed=3)])
    hd = H.hwfv1_batch_member(ens.bt, 0)
    with pytest.raises(H.Hwfv1Error):
        H.hwfv1_set_leaf_store(hd, 1)
    with pytest.raises(H.Hwfv1Error):
        H.hwfv1_set_skip_levels(hd, np.full((8, 8), 7, np.uint8), 10)
    ens.advance(t_end=0.002, max_steps=100)
    ref = oracle.State(*synth.bumpy_dam_break(L=7, eps=1e-3, seed=3))
    ref.run(t_end=0.002)
    assert np.array_equal(ens.member_fields(0)["h"], ref.h)
    ens.close()
