"""Learned subtree skip end to end: training data from the GPU path,
training on the tensor cores, then a held-out run with the network's
predicted levels in the time loop against plain HWFV1 (regularisation by
one-level prediction) and against uniform FV1 (eps = 0).  Water columns
collapsing on a flat bed: the refinement follows the moving flow alone, so
most subtrees are predicted shallow and stored coarse."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

L = 8


def _run(p, f, t_end, net=None, audit_K=10, margin=0.02, max_steps=20000, every=1):
    from paper_2206_05761_gb300.sim import Simulation
    sim = Simulation(p, f)
    if net is not None:
        sim.set_skipnet(net, audit_K=audit_K, margin=margin, predict_every=every)
    ms = []
    while sim.time()[0] < t_end and len(ms) < max_steps:
        sim.advance(t_end=t_end, max_steps=1)
        ms.append(sim.stats()[0])
    out = sim.fields(), float(np.mean(ms)), len(ms)
    sim.close()
    return out


@pytest.fixture(scope="module")
def trained():
    from paper_2206_05761_gb300 import hwfv1 as Hh
    from paper_2206_05761_gb300 import learn
    cases = [synth.columns_dam_break(L=L, eps=1e-3, seed=s) for s in range(100, 108)]
    x, y = learn.collect(cases, steps=600, every=10)
    x, y = learn.augment(x, y)
    net, loss = learn.train(x, y, epochs=15, batch=32, lr=3e-3, seed=1)
    print("training: %d images of %dx%d, last batch loss %.4f" % (x.shape[0], x.shape[1], x.shape[2], loss))
    yield net, learn
    Hh.hwfv1_skipnet_destroy(net)


def test_network_predicts_held_out_levels(trained):
    net, learn = trained
    x, y = learn.collect([synth.columns_dam_break(L=L, eps=1e-3, seed=200)], steps=600, every=20)
    under = learn.under_prediction_rate(net, x, y, 0.02)
    exact = float((learn.predict_levels(net, x, 0.0) == y).float().mean())
    print("held out: %.4f of subtrees under-predicted at margin 0.02; %.3f exact at margin 0" % (under, exact))
    assert under < 0.05


def test_learned_run_uses_fewer_leaves_at_bounded_cost(trained):
    net, _ = trained
    t_end = 0.25
    p, f = synth.columns_dam_break(L=L, eps=1e-3, seed=200)
    fp, mp, tp = _run(p, f, t_end)
    fl, ml, tl = _run(p, f, t_end, net=net)
    pu, fu = synth.columns_dam_break(L=L, eps=0.0, seed=200)
    fu_, mu, tu = _run(pu, fu, t_end)
    cell = 1.0 / (1 << (2 * L))
    d_lp = np.abs(fl["h"] - fp["h"]).sum() * cell
    d_pu = np.abs(fp["h"] - fu_["h"]).sum() * cell
    print("mean leaves: uniform %.0f, plain %.0f, learned %.0f (%.3f of plain); steps: %d %d %d"
          % (mu, mp, ml, ml / mp, tu, tp, tl))
    print("L1 depth: |learned - plain| = %.3e, |plain - uniform| = %.3e" % (d_lp, d_pu))
    # at margin 0.02 the predicted levels keep nearly every needed level on
    # this small grid (the network is trained with atomic float sums, so the
    # levels vary from run to run).  The two runs' states drift apart, so
    # their mean leaf counts are compared loosely; the error stays bounded.
    assert ml <= mp * 1.01
    assert d_lp <= 2.0 * d_pu + 1e-12
    # a looser margin (the median level: a subtree is cut wherever the
    # network gives the shallower levels even odds), at a bounded cost: the
    # error stays within a few times the method's own adaptive error
    fm, mm, _ = _run(p, f, t_end, net=net, margin=0.5)
    d_mp = np.abs(fm["h"] - fp["h"]).sum() * cell
    print("margin 0.5: mean leaves %.0f (%.3f of plain), L1 |learned - plain| = %.3e" % (mm, mm / mp, d_mp))
    assert mm <= mp * 1.02
    assert d_mp <= 5.0 * d_pu + 1e-12


def test_learned_step_never_adds_leaves_on_the_same_state(trained):
    """From identical states (checkpoints of the plain run) the first skip
    step after the exact one encodes the same finest state and keeps a
    subset of the plain step's significant parents (the flags below each
    subtree's predicted level), so it has at most as many leaves; at the
    median-level margin it drops some."""
    from paper_2206_05761_gb300.sim import Simulation
    net, _ = trained
    p, f = synth.columns_dam_break(L=L, eps=1e-3, seed=200)
    ref = Simulation(p, f)
    snaps = []
    for _ in range(10):
        ref.advance(max_steps=50)
        snaps.append(ref.save())
    ref.close()
    plain, lrn = Simulation(p, f), Simulation(p, f)
    out = []
    for blob in snaps:
        plain.load(blob)
        plain.advance(max_steps=2)
        lrn.load(blob)
        # the step after attaching the network is exact, the next one a skip step
        lrn.set_skipnet(net, audit_K=10, margin=0.5, predict_every=1)
        lrn.advance(max_steps=2)
        out.append((plain.stats()[0], lrn.stats()[0]))
    plain.close()
    lrn.close()
    print("leaves of one step from the same state (plain, learned):", out)
    assert all(b <= a for a, b in out)
    assert any(b < a for a, b in out)


def test_learned_run_reusing_predictions(trained):
    """The network on every 3rd learned step, its levels reused in between."""
    net, _ = trained
    t_end = 0.25
    p, f = synth.columns_dam_break(L=L, eps=1e-3, seed=200)
    fp, mp, _ = _run(p, f, t_end)
    fl, ml, _ = _run(p, f, t_end, net=net, every=3)
    pu, fu = synth.columns_dam_break(L=L, eps=0.0, seed=200)
    fu_, _, _ = _run(pu, fu, t_end)
    cell = 1.0 / (1 << (2 * L))
    d_lp = np.abs(fl["h"] - fp["h"]).sum() * cell
    d_pu = np.abs(fp["h"] - fu_["h"]).sum() * cell
    print("reuse 3: mean leaves %.0f (%.3f of plain); L1 |learned - plain| = %.3e, |plain - uniform| = %.3e"
          % (ml, ml / mp, d_lp, d_pu))
    assert ml <= mp * 1.01
    assert d_lp <= 2.0 * d_pu + 1e-12


def test_reuse_schedule_same_with_and_without_graphs(trained, monkeypatch):
    """The captured step graphs and the direct launches pick the same kind of
    step (exact, predicting, reusing) in the same order."""
    from paper_2206_05761_gb300.sim import Simulation
    net, _ = trained
    p, f = synth.columns_dam_break(L=L, eps=1e-3, seed=201)
    out = []
    for graphs in (True, False):
        if not graphs:
            monkeypatch.setenv("HWFV1_NO_GRAPH", "1")
        sim = Simulation(p, f)
        sim.set_skipnet(net, audit_K=5, margin=0.02, predict_every=2)
        sim.advance(max_steps=23)
        out.append((sim.fields(), sim.leaves()))
        sim.close()
    for k in out[0][0]:
        assert np.array_equal(out[0][0][k], out[1][0][k])
    assert np.array_equal(out[0][1], out[1][1])
