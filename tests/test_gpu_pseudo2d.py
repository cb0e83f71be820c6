"""Pseudo-2D dam-break of Sec. 3.2 on the GPU (50 m x 25 m, 6 m / 2 m, dam at
x = 10 m, open sides): HWFV1 and uniform FV1 against the exact (Stoker)
solution of the 1D Riemann problem, and a trajectory against the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

G = 9.80665


def _stoker(x, t, hl, hr, x0):
    """Exact depth of the 1D dam-break over a wet bed: left rarefaction,
    constant state (hm, um), right-moving shock (the classical construction:
    um from the rarefaction's Riemann invariant equals um from the shock's
    Rankine-Hugoniot conditions)."""
    from scipy.optimize import brentq
    cl = np.sqrt(G * hl)

    def f(hm):
        um = 2.0 * (cl - np.sqrt(G * hm))
        return um - (hm - hr) * np.sqrt(0.5 * G * (hm + hr) / (hm * hr))

    hm = brentq(f, hr, hl, xtol=1e-14)
    um = 2.0 * (cl - np.sqrt(G * hm))
    cm = np.sqrt(G * hm)
    s = hm * um / (hm - hr)
    xi = (x - x0) / t
    h = np.where(xi <= -cl, hl, 0.0)
    fan = (xi > -cl) & (xi <= um - cm)
    h = np.where(fan, (2.0 * cl - xi) ** 2 / (9.0 * G), h)
    h = np.where((xi > um - cm) & (xi < s), hm, h)
    h = np.where(xi >= s, hr, h)
    return h


def _run(L, eps, uniform):
    from paper_2206_05761_gb300.sim import Simulation
    p, f = synth.pseudo_2d_dam_break(L=L, eps=eps)
    sim = Simulation(p, f)
    for _ in range(100000):
        t = sim.time()[0]
        if t >= 1.0:
            break
        if uniform:
            sim.advance_uniform(t_end=1.0, max_steps=500)
        else:
            sim.advance(t_end=1.0, max_steps=500)
    assert sim.time()[0] == 1.0
    x, _ = synth.centres(p)
    h = sim.fields()["h"]
    n, lu, _, _, _ = sim.counters()
    sim.close()
    return float(np.mean(np.abs(h - _stoker(x, 1.0, 6.0, 2.0, 10.0)))), h, lu / n


def test_gpu_dam_break_converges_to_exact_solution():
    errs_u, errs_a = [], []
    for L in (8, 9, 10):
        eu, hu, _ = _run(L, 0.0, True)
        ea, ha, m = _run(L, 1e-3, False)
        errs_u.append(eu)
        errs_a.append(ea)
        # 1D flow: every row the same
        assert np.abs(hu - hu[0:1, :]).max() <= 1e-12
        # the adaptive run stays close to the uniform one and uses fewer cells
        assert float(np.mean(np.abs(ha - hu))) < 2e-2
        assert m < (1 << (2 * L))
    print("L1 error vs exact, L = 8, 9, 10: uniform %s, HWFV1 %s" % (errs_u, errs_a))
    assert errs_u[0] > errs_u[1] > errs_u[2] and errs_u[2] < 0.04
    assert errs_a[0] > errs_a[1] > errs_a[2] and errs_a[2] < 0.04


def test_gpu_dam_break_trajectory_matches_oracle():
    from paper_2206_05761_gb300.sim import Simulation
    p, f = synth.pseudo_2d_dam_break(L=7, eps=1e-3)
    sim = Simulation(p, f)
    ref = oracle.State(p, f)
    for chunk in range(3):
        sim.advance(max_steps=20)
        for _ in range(19):
            ref.step()
        res = ref.step(want=("leaves",))
        assert np.array_equal(sim.leaves(), res["leaves"])
        g = sim.fields()
        for k in ("h", "qx", "qy"):
            assert np.array_equal(g[k], getattr(ref, k)), k
        assert sim.time()[:2] == (ref.t, ref.dt)
    sim.close()
