"""Pins of the oracle's FV1 operator and HWFV1 time loop against closed
forms, exact solutions and invariants the paper relies on (no GPU)."""
import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
import synth

G = 9.80665


# --------------------------------------------------------------------------
# HLL flux (Eq. 1 fluxes; L_c reading)
# --------------------------------------------------------------------------

def _phys_flux(h, qx, qy):
    u, v = qx / h, qy / h
    return np.array([qx, qx * u + 0.5 * G * h * h, qx * v])


@pytest.mark.parametrize("state", [(1.0, 0.3, -0.2), (2.5, -1.0, 0.4), (0.2, 0.0, 0.0)])
def test_hll_consistency(state):
    h, qx, qy = state
    F = oracle.hll_x(G, 1e-3, [h, qx, qy, 0.0], [h, qx, qy, 0.0])
    np.testing.assert_allclose(F, _phys_flux(h, qx, qy), rtol=1e-14, atol=1e-15)


def test_hll_supersonic_upwinding():
    # u > sqrt(gh) on both sides: the flux is the left physical flux exactly
    L_ = [1.0, 5.0, 0.5, 0.0]
    R_ = [0.8, 4.5, 0.1, 0.0]
    F = oracle.hll_x(G, 1e-3, L_, R_)
    assert np.array_equal(F, _phys_flux(*L_[:3]))
    # mirrored: right state wins
    L2 = [0.8, -4.5, 0.1, 0.0]
    R2 = [1.0, -5.0, 0.5, 0.0]
    F = oracle.hll_x(G, 1e-3, L2, R2)
    assert np.array_equal(F, _phys_flux(*R2[:3]))


def test_hll_dry_faces():
    assert np.all(oracle.hll_x(G, 1e-3, [0, 0, 0, 0], [0, 0, 0, 0]) == 0)
    # water below a higher bed step: the reconstructed depths are zero
    assert np.all(oracle.hll_x(G, 1e-3, [0.5, 0.1, 0, 0.0], [0.0, 0, 0, 2.0]) == 0)


def test_hll_lake_at_rest_face_is_pressure_only():
    # same free surface on both sides: no mass flux, momentum flux 0.5*g*h*^2
    F = oracle.hll_x(G, 1e-3, [1.0, 0, 0, 0.25], [0.75, 0, 0, 0.5])
    hs = 0.75
    assert F[0] == 0.0 and F[2] == 0.0
    assert F[1] == pytest.approx(0.5 * G * hs * hs, rel=1e-15)


# --------------------------------------------------------------------------
# Whole-step properties
# --------------------------------------------------------------------------

def _volume(st):
    L = st.p["L"]
    return float(np.sum(st.h)) * (st.p["lx"] / (1 << L)) * (st.p["ly"] / (1 << L))


@pytest.mark.parametrize("eps", [1e-3, 0.0])
def test_lake_at_rest_fully_wet(eps):
    # Sec. 3.1: discharges stay zero to round-off over an uneven, wet bed
    p, f = synth.lake_at_rest(L=6, eps=eps)
    st = oracle.State(p, f)
    st.run(max_steps=300)
    assert max(np.abs(st.qx).max(), np.abs(st.qy).max()) <= 1e-10
    assert np.abs(st.h + st.z - 1.0).max() <= 1e-10


def test_lake_at_rest_with_dry_humps_stays_bounded():
    # Table 3 setting (humps emerge): the paper reports bounded discharge
    # errors rather than round-off; here they must stay small
    p, f = synth.lake_at_rest(L=6, eps=1e-3, wet=False)
    assert (f["h"] == 0).any()
    st = oracle.State(p, f)
    st.run(max_steps=200)
    assert max(np.abs(st.qx).max(), np.abs(st.qy).max()) <= 1e-6


def test_eps_zero_hwfv1_equals_uniform_fv1_bitwise():
    p, f = synth.circular_dam_break(L=5, eps=0.0)
    a = oracle.State(p, f)
    b = oracle.State(p, f)
    for _ in range(25):
        res = a.step(want=("leaves",))
        assert res["num_leaves"] == 1 << 10
        b.fv1_step()
        assert a.dt == b.dt
    assert np.array_equal(a.h, b.h) and np.array_equal(a.qx, b.qx) and np.array_equal(a.qy, b.qy)


@pytest.mark.parametrize("eps", [0.0, 1e-3])
def test_mass_conserved_with_closed_walls_uniform_grid(eps):
    # conservative only when every leaf is on one level; eps=1e-3 on a flat
    # still start stays uniform only at eps=0, so the adaptive case reports
    p, f = synth.circular_dam_break(L=5, eps=eps)
    p["bc"] = ("closed",) * 4
    st = oracle.State(p, f)
    v0 = _volume(st)
    st.run(max_steps=100)
    drift = abs(_volume(st) - v0) / v0
    if eps == 0.0:
        assert drift <= 1e-13
    else:
        assert drift <= 1e-2        # reported, not round-off (same-level rule)


def _stoker(x, t, hl, hr, x0):
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


def test_dam_break_converges_to_exact_solution():
    # Sec. 3.2 pseudo-2D dam-break (6 m / 2 m, dam at x = 10 m) against the
    # exact (Stoker) solution of the 1D Riemann problem at t = 1 s
    errs = []
    for L in (5, 6, 7):
        p, f = synth.pseudo_2d_dam_break(L=L, eps=0.0)
        st = oracle.State(p, f)
        st.run(t_end=1.0, uniform=True)
        assert st.t == 1.0
        x, _ = synth.centres(p)
        ex = _stoker(x, 1.0, 6.0, 2.0, 10.0)
        errs.append(float(np.mean(np.abs(st.h - ex))))
        # 1D flow: every row identical
        assert np.abs(st.h - st.h[0:1, :]).max() <= 1e-12
        assert np.abs(st.qy).max() <= 1e-12
    # first order with a shock: L1 error falls by ~dx^0.6-0.8 per level
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[2] > 2.0
    assert errs[2] < 0.07


def test_hwfv1_dam_break_close_to_uniform():
    p, f = synth.pseudo_2d_dam_break(L=6, eps=1e-3)
    a = oracle.State(p, f)
    a.run(t_end=1.0)
    p0, f0 = synth.pseudo_2d_dam_break(L=6, eps=0.0)
    b = oracle.State(p0, f0)
    b.run(t_end=1.0, uniform=True)
    assert a.leaf_updates < b.leaf_updates
    assert float(np.mean(np.abs(a.h - b.h))) < 2e-2


@pytest.mark.parametrize("h", [1.0, 2.5, 0.4])
def test_friction_decay_matches_closed_form(h):
    # uniform flow on a flat bed: fluxes cancel and the semi-implicit Manning
    # step solves du/dt = -k u^2 exactly: 1/u(t) = 1/u0 + k t, k = g n^2 / h^(4/3)
    # (depths other than 1 tell the Manning exponent apart)
    u0, n = 2.0, 0.03
    p, f = synth.uniform_flow(L=4, h=h, u=u0, manning_n=n)
    st = oracle.State(p, f)
    st.run(max_steps=200)
    k = G * n * n / h ** (4.0 / 3.0)
    u_exact = u0 / (1.0 + k * u0 * st.t)
    np.testing.assert_allclose(st.qx / st.h, u_exact, rtol=1e-11)
    assert np.all(st.h == h) and np.all(st.qy == 0.0)


def test_no_friction_keeps_uniform_flow():
    p, f = synth.uniform_flow(L=4, manning_n=0.0)
    st = oracle.State(p, f)
    st.run(max_steps=50)
    assert np.array_equal(st.qx, f["qx"])


def test_inflow_adds_exact_volume():
    p, f = synth.inflow_basin(L=5, eps=0.0, q=0.01)
    st = oracle.State(p, f)
    v0 = _volume(st)
    st.run(max_steps=100)
    added = 0.01 * st.t
    assert abs(_volume(st) - v0 - added) <= 1e-12 * _volume(st)


def test_inflow_follows_the_piecewise_linear_hydrograph():
    # R-inflow: each step adds Q(t) dt at its start time t, Q interpolated
    # linearly between the hydrograph's points (np.interp), and the closed
    # basin loses nothing; the steps cross a breakpoint of the hydrograph
    tq, Q = [0.0, 0.2, 1.0], [0.0, 0.03, 0.005]
    p, f = synth.inflow_basin(L=5, eps=0.0, q=0.01)
    p = dict(p, inflow=dict(p["inflow"], t=tq, Q=Q))
    st = oracle.State(p, f)
    v = _volume(st)
    while st.t < 0.4:
        t0 = st.t
        st.step()
        v_new = _volume(st)
        assert abs((v_new - v) - np.interp(t0, tq, Q) * (st.t - t0)) <= 1e-12 * v_new
        v = v_new


def test_depths_stay_non_negative_when_a_cell_drains_through_two_faces():
    # a shallow cell moving diagonally into dry ground at CFL 1 (u = v = 10
    # m/s > sqrt(g h): every face upwinds) sends q dt / dx out through each
    # of its east and north faces, more than it holds; its depth is clamped
    # at zero and its discharges dropped
    p = synth.problem(3, lx=8.0, ly=8.0, eps=0.0, cfl=1.0, bc=("transmissive",) * 4)
    x, _ = synth.centres(p)
    h = np.zeros_like(x)
    h[3, 3] = 0.01
    f = dict(h=h, qx=10.0 * h, qy=10.0 * h, z=np.zeros_like(x))
    st = oracle.State(p, f)
    dt, dx = st.dt, p["lx"] / 8
    assert 0.01 - 2 * 0.1 * dt / dx < 0.0
    st.step()
    assert st.h.min() >= 0.0
    assert st.h[3, 3] == 0.0 and st.qx[3, 3] == 0.0 and st.qy[3, 3] == 0.0


def _ritter(x, t, h0, x0):
    a0 = np.sqrt(G * h0)
    xi = (x - x0) / t
    return np.where(xi <= -a0, h0, np.where(xi >= 2 * a0, 0.0, (2 * a0 - xi) ** 2 / (9 * G)))


def test_dry_bed_dam_break_mirror_and_ritter():
    # Ritter's dam break onto a dry bed, with the water on the west and on
    # the east: the two runs are mirror images (the HLL dry-bed speeds of a
    # dry left side and of a dry right side agree), every row is the same
    # (1D flow), and the depth converges to Ritter's solution
    errs = []
    for L in (6, 7):
        out = {}
        for water in ("west", "east"):
            p, f = synth.ritter_dam_break(L=L, water=water)
            st = oracle.State(p, f)
            st.run(t_end=5.0, uniform=True)
            assert st.t == 5.0
            assert np.abs(st.h - st.h[0:1, :]).max() <= 1e-12
            out[water] = st
        w, e = out["west"], out["east"]
        assert np.abs(w.h - e.h[:, ::-1]).max() <= 1e-12
        assert np.abs(w.qx + e.qx[:, ::-1]).max() <= 1e-12
        x, _ = synth.centres(w.p)
        errs.append(float(np.mean(np.abs(w.h - _ritter(x, 5.0, 1.0, 50.0)))))
    assert errs[1] < errs[0] / 1.3


@pytest.mark.parametrize("us, as_, aL, aR", [(0.3, 2.0, 2.5, 3.0), (-1.2, 1.5, 1.7, 4.0), (2.0, 0.5, 3.0, 0.6)])
def test_star_estimate_exact_for_two_rarefactions(us, as_, aL, aR):
    # states joined to the star state (us, as) by a left and a right
    # rarefaction (aL, aR >= as): u + 2a is carried across the left wave and
    # u - 2a across the right one, so the exact star state is known; the
    # two-rarefaction estimate must return it
    uL = us + 2 * as_ - 2 * aL
    uR = us - 2 * as_ + 2 * aR
    e_us, e_as = oracle.star_estimate(uL, aL, uR, aR)
    assert abs(e_us - us) <= 1e-14 * 8 and abs(e_as - as_) <= 1e-14 * 8


def test_circular_dam_break_symmetry():
    # Sec. 3.2: the circular dam-break is symmetric under transpose (x<->y,
    # qx<->qy) and mirror in x; round-off breaks bit equality only
    p, f = synth.circular_dam_break(L=6, eps=1e-3)
    st = oracle.State(p, f)
    for _ in range(40):
        res = st.step(want=("leaves",))
    h = st.h
    assert np.abs(h - h.T).max() <= 1e-12
    assert np.abs(h - h[:, ::-1]).max() <= 1e-12
    assert np.abs(st.qx - st.qy.T).max() <= 1e-12
    assert np.abs(st.qx + st.qx[:, ::-1]).max() <= 1e-12
    # leaf set symmetric under transpose
    L = p["L"]
    cells = set()
    for pk in res["leaves"]:
        n, code = int(pk) >> 28, int(pk) & 0x0FFFFFFF
        cells.add((n, *oracle.demorton(code)))
    assert {(n, j, i) for (n, i, j) in cells} == cells


def test_dt_from_cfl_and_dry_default():
    p, f = synth.circular_dam_break(L=4)
    st = oracle.State(p, f)
    dx = 1.0 / 16
    a = np.sqrt(G * f["h"])
    assert st.dt == pytest.approx(0.5 * np.min(dx / a), rel=1e-15)
    p, f = synth.terrain_flood(L=5)
    st = oracle.State(p, f)
    assert st.dt == p["dt_max"]


@pytest.mark.parametrize("dt_max", [1e-3, 2.5e-4])
def test_wet_cfl_step_is_capped_at_dt_max(dt_max):
    # R-cfl: a wet step is min(CFL * bound, dt_max).  The dam-break's CFL
    # step at L=4 is 0.5 * (1/16) / sqrt(2 g) = 7.06e-3 s, above both caps,
    # so the initial step and every step after it equal the cap exactly;
    # the time then advances by the cap per step
    p, f = synth.circular_dam_break(L=4)
    cfl_dt = 0.5 * (1.0 / 16) / np.sqrt(2.0 * G)
    assert cfl_dt > 5 * dt_max
    p = dict(p, dt_max=dt_max)
    st = oracle.State(p, f)
    assert st.dt == dt_max
    t = 0.0
    for _ in range(3):
        st.step()
        t += dt_max
        assert st.dt == dt_max
        assert st.t == t
    # above the CFL step the cap plays no part: the uncapped value returns
    st2 = oracle.State(dict(p, dt_max=1.0), f)
    assert st2.dt == pytest.approx(cfl_dt, rel=1e-15)


def test_dry_bumpy_domain_stays_dry():
    # a dry coarse leaf hands its depth (0) down unchanged: no water appears
    # in the hollows of the bed
    p, f = synth.bumpy_dam_break(L=6)
    f["h"][:] = 0.0
    st = oracle.State(p, f)
    for _ in range(10):
        res = st.step(want=("leaves",))
        levels = res["leaves"] >> 28
        assert levels.min() < p["L"]          # coarse dry leaves exist
    assert np.all(st.h == 0.0) and np.all(st.qx == 0.0) and np.all(st.qy == 0.0)


@pytest.mark.parametrize("eta", [0.875, 1.78, 1.95])
def test_lake_at_rest_at_table3_free_surface_levels(eta):
    # Sec. 3.1, Table 3: still water at the three printed free-surface
    # levels over humps up to 1.4 m (some emerge at the lowest level): the
    # discharges stay at round-off where the domain is fully wet and small
    # where humps emerge, and the free surface does not move
    p, f = synth.lake_at_rest(L=6, eps=1e-3, eta=eta, wet=False)
    st = oracle.State(p, f)
    st.run(max_steps=150)
    qmax = max(np.abs(st.qx).max(), np.abs(st.qy).max())
    wet = f["h"] > 0
    if wet.all():
        assert qmax <= 1e-10
    else:
        assert qmax <= 1e-6
    assert np.abs((st.h + st.z)[st.h > 1e-3] - eta).max() <= 1e-6
