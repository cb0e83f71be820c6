"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle on
the same seeded inputs.  In float64 the significance flags, leaf lists,
encoded coefficients, fields and timesteps must be bit-identical when there
is no friction; with Manning friction (cbrt is not correctly rounded on
either side) fields are held to 1e-12 relative."""
import numpy as np
import pytest

import oracle
import synth

from _util import level_slice, rm_to_morton

pytestmark = pytest.mark.gpu

RTOL_FRICTION = 1e-12


def _sim(p, f, precision=64):
    from paper_2206_05761_gb300.sim import Simulation
    return Simulation(p, f, precision)


def _unpack(words, L):
    from paper_2206_05761_gb300.sim import unpack_bits
    return unpack_bits(words, L)


def _compare_fields(sim, ref, exact=True):
    g = sim.fields()
    for k in ("h", "qx", "qy"):
        o = getattr(ref, k)
        if exact:
            assert np.array_equal(g[k], o), "field %s: max diff %g" % (k, np.abs(g[k] - o).max())
        else:
            scale = max(np.abs(o).max(), 1e-300)
            assert np.abs(g[k] - o).max() <= RTOL_FRICTION * scale, k


def one_step_parity(p, f, exact=True, pre_steps=0):
    """Run pre_steps on both sides (state compared after them), then one
    step phase by phase, comparing every intermediate."""
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    L = p["L"]
    t, dt, _ = sim.time()
    assert dt == ref.dt and t == ref.t
    for _ in range(pre_steps):
        sim.step()
        ref.step()
    if pre_steps:
        _compare_fields(sim, ref, exact)
        if not exact:      # continue from an identical state
            sim.set_fields({"h": ref.h, "qx": ref.qx, "qy": ref.qy})
        t, dt, _ = sim.time()
        if not exact:
            sim.set_time(ref.t, ref.dt)
        else:
            assert t == ref.t and dt == ref.dt
    res = ref.step(want=("T", "S", "leaves", "hier"))
    sim.encode()
    N = 1 << (2 * L)
    P = (N - 1) // 3
    for q in range(3):
        hier = res["hier"][q]
        for n in range(L):
            got = sim.level(q, n)
            exp = rm_to_morton(hier[level_slice(n)], n)
            assert np.array_equal(got, exp), "field %d level %d" % (q, n)
    sim.flag()
    T = _unpack(sim.flags(0), L)
    S = _unpack(sim.flags(1), L)
    for n in range(L):
        assert np.array_equal(T[n], rm_to_morton(res["T"][level_slice(n)], n)), "T level %d" % n
        assert np.array_equal(S[n], rm_to_morton(res["S"][level_slice(n)], n)), "S level %d" % n
    assert P == len(res["T"])
    M = sim.traverse(want_count=True)
    assert M == res["num_leaves"]
    assert np.array_equal(sim.leaves(), res["leaves"])
    sim.fv1()
    sim.decode()
    _compare_fields(sim, ref, exact)
    t, dt, steps = sim.time()
    assert t == ref.t
    if exact:
        assert dt == ref.dt
    else:
        assert abs(dt - ref.dt) <= RTOL_FRICTION * ref.dt
    sim.close()
    return res


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 6])
def test_circular_dam_break_small_levels(L):
    p, f = synth.circular_dam_break(L=L, eps=1e-3)
    one_step_parity(p, f)


def test_circular_dam_break_L6_after_steps():
    p, f = synth.circular_dam_break(L=6, eps=1e-3)
    one_step_parity(p, f, pre_steps=20)


@pytest.mark.parametrize("seed", [2, 11])
def test_bumpy_dam_break_wet_dry(seed):
    p, f = synth.bumpy_dam_break(L=7, eps=1e-3, seed=seed)
    one_step_parity(p, f, pre_steps=5)


def test_lake_at_rest_dry_humps():
    p, f = synth.lake_at_rest(L=7, eps=1e-3, wet=False)
    one_step_parity(p, f, pre_steps=3)


@pytest.mark.parametrize("eta", [0.875, 1.78, 1.95])
def test_lake_at_rest_table3_levels(eta):
    # Table 3's free-surface levels over humps that partly emerge: 20 steps
    # of the graph path against the oracle, bit for bit
    p, f = synth.lake_at_rest(L=7, eps=1e-3, eta=eta, wet=False)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    sim.advance(max_steps=20)
    for _ in range(19):
        ref.step()
    res = ref.step(want=("leaves",))
    assert np.array_equal(sim.leaves(), res["leaves"])
    _compare_fields(sim, ref)
    assert max(np.abs(ref.qx).max(), np.abs(ref.qy).max()) <= 1e-6
    sim.close()


def test_inflow_basin():
    p, f = synth.inflow_basin(L=6, eps=1e-3, q=0.01)
    one_step_parity(p, f, pre_steps=4)


def test_non_square_domain_open_boundaries():
    p, f = synth.pseudo_2d_dam_break(L=7, eps=1e-3)
    one_step_parity(p, f, pre_steps=3)


def test_eps_zero_every_leaf_finest():
    p, f = synth.circular_dam_break(L=5, eps=0.0)
    res = one_step_parity(p, f)
    assert res["num_leaves"] == 1 << 10


def test_huge_eps_single_root_leaf():
    p, f = synth.lake_at_rest(L=5, eps=1e300)
    f["z"][:] = 0.0
    f["h"][:] = 1.0
    res = one_step_parity(p, f)
    assert res["num_leaves"] == 1


@pytest.mark.parametrize("predict,close", [(True, False), (False, True), (False, False)])
def test_regularisation_variants(predict, close):
    p, f = synth.bumpy_dam_break(L=6, eps=1e-3)
    p["reg_predict"], p["reg_close"] = predict, close
    one_step_parity(p, f, pre_steps=2)


def test_threshold_edges_decided_like_the_oracle():
    # 2 x 2 blocks whose largest detail sits within a relative r of the
    # level-(L-1) threshold (r from 1e-15 to 1e-3, both signs, both detail
    # directions, several magnitudes): the float pre-check of the encode may
    # decide only where its error bound allows, so every flag must equal the
    # oracle's double decision
    L = 6
    p, f = synth.circular_dam_break(L=L, eps=1e-3)
    p["bc"] = ("closed",) * 4
    thr = p["eps"] * 0.5                                  # s_max = 1 (all h <= 1)
    rs = [s * m for m in (1e-15, 1e-13, 1e-11, 1e-9, 1e-8, 1e-7, 3e-7, 1e-6, 1e-5, 1e-3) for s in (1, -1)]
    xs = [1e-3, 0.01, 0.05, 0.3, 0.9]
    h = np.zeros((1 << L, 1 << L))
    k = 0
    for pj in range(1 << (L - 1)):
        for pi in range(1 << (L - 1)):
            r = rs[k % len(rs)]
            x = xs[(k // len(rs)) % len(xs)]
            d = 2.0 * thr * (1.0 + r)
            if (k // (len(rs) * len(xs))) % 2 == 0:       # detail beta: columns differ
                blk = [[x, x + d], [x, x + d]]
            else:                                         # detail alpha: rows differ
                blk = [[x, x], [x + d, x + d]]
            h[2 * pj: 2 * pj + 2, 2 * pi: 2 * pi + 2] = blk
            k += 1
    assert h.max() <= 1.0
    f = dict(f, h=np.ascontiguousarray(h), qx=np.zeros_like(h), qy=np.zeros_like(h),
             z=np.zeros_like(h))
    res = one_step_parity(p, f)
    T = res["T"][level_slice(L - 1)]
    assert 0 < T.sum() < T.size                           # both decisions occur


def test_all_dry_terrain():
    p, f = synth.terrain_flood(L=7)
    p["bc"] = ("closed",) * 4
    p["inflow"] = None
    one_step_parity(p, f, pre_steps=2)


def test_terrain_flood_with_friction_and_inflow():
    p, f = synth.terrain_flood(L=7)
    one_step_parity(p, f, exact=False, pre_steps=30)


def test_uniform_friction_flow():
    p, f = synth.uniform_flow(L=4, manning_n=0.03)
    one_step_parity(p, f, exact=False, pre_steps=5)


def test_trajectory_circular_dam_break_100_steps():
    # configs: circular dam-break, 64 x 64, eps 1e-3, 100 steps; the graph
    # replay path (hwfv1_advance) against the oracle's time loop
    p, f = synth.circular_dam_break(L=6, eps=1e-3)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    for chunk in range(10):
        sim.advance(max_steps=10)
        for _ in range(9):
            ref.step()
        res = ref.step(want=("leaves",))
        assert np.array_equal(sim.leaves(), res["leaves"]), "chunk %d" % chunk
        _compare_fields(sim, ref)
        t, dt, steps = sim.time()
        assert t == ref.t and dt == ref.dt and steps == ref.steps
    sim.close()


@pytest.mark.parametrize("water", ["west", "east"])
def test_dry_bed_dam_break_trajectory(water):
    # Ritter's dam break onto a dry flat bed, with the water on either side:
    # the dry-bed HLL speeds of both orientations, 40 steps of the graph path
    p, f = synth.ritter_dam_break(L=6, eps=1e-3, water=water)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    sim.advance(max_steps=40)
    for _ in range(39):
        ref.step()
    res = ref.step(want=("leaves",))
    assert np.array_equal(sim.leaves(), res["leaves"])
    _compare_fields(sim, ref)
    t, dt, steps = sim.time()
    assert t == ref.t and dt == ref.dt and steps == 40
    sim.close()


def test_cell_draining_through_two_faces_is_clamped_like_the_oracle():
    # CFL 1: a shallow cell moving diagonally into dry ground loses more than
    # it holds in one step; both sides clamp its depth at zero
    p = synth.problem(3, lx=8.0, ly=8.0, eps=0.0, cfl=1.0, bc=("transmissive",) * 4)
    x, _ = synth.centres(p)
    h = np.zeros_like(x)
    h[3, 3] = 0.01
    f = dict(h=h, qx=10.0 * h, qy=10.0 * h, z=np.zeros_like(x))
    res = one_step_parity(p, f)
    assert res["num_leaves"] == 64


def test_trajectory_in_multi_step_graphs():
    # advances of 37 steps: two 16-step graph launches and five single-step
    # ones each, against the oracle's loop
    p, f = synth.circular_dam_break(L=6, eps=1e-3)
    p["bc"] = ("closed",) * 4
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    for chunk in range(3):
        sim.advance(max_steps=37)
        for _ in range(36):
            ref.step()
        res = ref.step(want=("leaves",))
        assert np.array_equal(sim.leaves(), res["leaves"]), "chunk %d" % chunk
        _compare_fields(sim, ref)
        t, dt, steps = sim.time()
        assert t == ref.t and dt == ref.dt and steps == ref.steps
    sim.close()


def test_counters_sum_the_leaf_updates():
    # the running leaf-update count equals the oracle's sum of M over the
    # same steps; the captured step graph launches a positive, fixed number
    # of kernels
    p, f = synth.circular_dam_break(L=6, eps=1e-3)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    sim.advance(max_steps=25)
    for _ in range(25):
        ref.step()
    steps, lu, au, wu, kps = sim.counters()
    assert steps == 25 and lu == ref.leaf_updates
    assert 0 < wu <= au <= lu and 0 < kps < 64
    sim.close()


def test_profiled_step_is_an_ordinary_step():
    # hwfv1_profile_step launches the plain step kernel by kernel with events
    # in between: same state as one oracle step, every kernel listed
    from paper_2206_05761_gb300 import hwfv1 as Hh
    p, f = synth.circular_dam_break(L=6, eps=1e-3)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    prof = Hh.hwfv1_profile_step(sim.hd)
    names = [n for n, _ in prof]
    assert names[0] == "k_clear_words" and names[-1] == "k_decode_finish"
    for k in ("k_encode_tail", "k_trav_classify", "k_trav_list", "k_fv1_dry", "k_fv1_faces", "k_fv1_update"):
        assert k in names
    # the plain step forms the regularised flags inside the traversal
    assert "k_flag" not in names
    assert all(t >= 0.0 for _, t in prof)
    res = ref.step(want=("leaves", "S"))
    assert np.array_equal(sim.leaves(), res["leaves"])
    # the flag words, formed on demand after such a step, are the oracle's S
    S = _unpack(sim.flags(1), p["L"])
    for n in range(p["L"]):
        assert np.array_equal(S[n], rm_to_morton(res["S"][level_slice(n)], n)), "S level %d" % n
    _compare_fields(sim, ref)
    assert sim.time()[:3] == (ref.t, ref.dt, 1)
    sim.close()


def test_profiled_update_is_an_ordinary_step():
    # hwfv1_profile_update replays the update of the queued leaves inside
    # one step: the state after it is one oracle step, bit for bit
    from paper_2206_05761_gb300 import hwfv1 as Hh
    p, f = synth.bumpy_dam_break(L=7, eps=1e-3, seed=2)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    sim.advance(max_steps=3)
    for _ in range(3):
        ref.step()
    ms = Hh.hwfv1_profile_update(sim.hd, reps=7)
    assert ms > 0.0
    res = ref.step(want=("leaves",))
    assert np.array_equal(sim.leaves(), res["leaves"])
    _compare_fields(sim, ref)
    assert sim.time()[:3] == (ref.t, ref.dt, 4)
    sim.close()


def test_advance_stops_at_t_end():
    p, f = synth.circular_dam_break(L=5, eps=1e-3)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    t_end = 0.02
    sim.advance(t_end=t_end, max_steps=200)
    n = ref.run(t_end=t_end)
    t, dt, steps = sim.time()
    assert steps == n and t == ref.t == t_end
    _compare_fields(sim, ref)
    sim.close()


def test_bumpy_dam_break_L10_one_step():
    # configs: bumpy dam-break 1024 x 1024 (L = 10), eps 1e-3 and 1e-4
    for eps in (1e-3, 1e-4):
        p, f = synth.bumpy_dam_break(L=10, eps=eps)
        one_step_parity(p, f, pre_steps=2)


def test_checkpoint_resume_is_bit_identical():
    p, f = synth.bumpy_dam_break(L=6, eps=1e-3)
    a = _sim(p, f)
    a.advance(max_steps=5)
    blob = a.save()
    a.advance(max_steps=7)
    ga = a.fields()
    ta = a.time()
    b = _sim(p, f)
    b.load(blob)
    assert b.time()[2] == 5
    b.advance(max_steps=7)
    gb = b.fields()
    assert b.time() == ta
    for k in ga:
        assert np.array_equal(ga[k], gb[k])
    a.close()
    b.close()


@pytest.mark.parametrize("field", ["h", "qx", "z"])
def test_nonfinite_input_is_reported(field):
    # a NaN planted in the initial fields (on the host) is latched on the
    # device and reported by the next synchronising call
    from paper_2206_05761_gb300.hwfv1 import Hwfv1Error
    p, f = synth.circular_dam_break(L=4, eps=1e-3)
    f[field][3, 3] = np.nan
    sim = _sim(p, f)
    with pytest.raises(Hwfv1Error) as e:
        sim.time()
    assert e.value.status == 4
    sim.close()


def test_nonfinite_discharge_during_run_is_reported():
    # a state that turns non-finite during a step (huge discharge overflows
    # the momentum flux) is caught by the step's own check
    from paper_2206_05761_gb300.hwfv1 import Hwfv1Error
    p, f = synth.circular_dam_break(L=4, eps=1e-3)
    sim = _sim(p, f)
    g = {k: f[k].copy() for k in ("h", "qx", "qy")}
    g["qx"][3, 3] = 1e300
    sim.set_fields(g)
    sim.step()
    with pytest.raises(Hwfv1Error) as e:
        sim.time()
    assert e.value.status == 4
    sim.close()


def test_float32_path_errors_stated():
    # 32-bit arithmetic against the float64 oracle: errors per field after
    # 20 steps of the circular dam-break are reported and stay small
    p, f = synth.circular_dam_break(L=6, eps=1e-3)
    sim = _sim(p, f, precision=32)
    ref = oracle.State(p, f)
    t_end = 0.02
    sim.advance(t_end=t_end, max_steps=200)
    ref.run(t_end=t_end)
    g = sim.fields()
    errs = {k: float(np.abs(g[k] - getattr(ref, k)).max()) for k in ("h", "qx", "qy")}
    print("float32 vs float64 oracle at t=%g: max abs error %s" % (t_end, errs))
    assert errs["h"] < 1e-4 and errs["qx"] < 1e-4 and errs["qy"] < 1e-4
    sim.close()


@pytest.mark.parametrize("steps", [3, 5])
def test_full_size_terrain_flood_L12_bench_window(steps):
    # the bench's timed window at full size (4096 x 4096, 10 km, eps 1e-3,
    # Manning 0.03): its generator-built start state at the hydrograph peak
    # (t = 1800 s, inflow at 500 m^3/s, the channel running full, the rest
    # dry), advanced through the same graph-replay path bench.py times (dry
    # tiles skipped from the second step on), against the oracle's steps;
    # leaves exactly, fields within 1e-12 (friction)
    p, f, t0 = synth.terrain_flood_peak(L=12)
    sim = _sim(p, f)
    ref = oracle.State(p, f, t=t0)
    t, dt, _ = sim.time()
    assert dt == ref.dt
    sim.set_time(t0, dt)
    sim.advance(max_steps=steps)
    for _ in range(steps - 1):
        ref.step()
    res = ref.step(want=("leaves",))
    lv = sim.leaves()
    assert len(lv) == res["num_leaves"] and np.array_equal(lv, res["leaves"])
    _compare_fields(sim, ref, exact=False)
    t, dt, n = sim.time()
    assert n == steps and abs(t - ref.t) <= RTOL_FRICTION * ref.t
    assert abs(dt - ref.dt) <= RTOL_FRICTION * ref.dt
    n, lu, au, wu, kps = sim.counters()
    assert lu == ref.leaf_updates and au < lu and wu > 0
    sim.close()


def test_full_sweep_L12_encode_levels():
    # every tile encoded (HWFV1_FULL_SWEEP) at 4096 x 4096: the first pass
    # stops after three levels of each 1024-cell block and the next pass
    # takes the block's top levels; every level, flag and leaf against the
    # oracle
    p, f = synth.terrain_flood(L=12, fill=2.0, fill_q=1.0)
    one_step_parity(dict(p, full_sweep=True), f, exact=False)


def test_full_size_wet_domain_one_step():
    # 4096 x 4096 bumpy dam-break: about 16 M wet leaves, more than the
    # shared-face buffer holds, so the update takes its one-pass form
    p, f = synth.bumpy_dam_break(L=12, eps=1e-3)
    one_step_parity(p, f)


@pytest.mark.parametrize("relief", [0.0, 0.05])
def test_quiescent_tile_skipping_is_exact(relief):
    # water released onto dry ground: most 32 x 32 tiles hold +0 in both
    # state buffers; leaves, fields and time must equal the oracle's and the
    # full sweep's bit for bit.  On the flat bed the dry ground is covered by
    # leaves coarser than a tile (its encode and decode writes are skipped);
    # on rough ground the dry tiles hold their own fine leaves (skipped)
    p, f = synth.dry_bed_dam_break(L=8, eps=1e-3, relief=relief)
    sim = _sim(p, f)
    full = _sim(dict(p, full_sweep=True), f)
    ref = oracle.State(p, f)
    for chunk in range(6):
        sim.advance(max_steps=10)
        full.advance(max_steps=10)
        for _ in range(9):
            ref.step()
        res = ref.step(want=("leaves",))
        assert np.array_equal(sim.leaves(), res["leaves"]), "chunk %d" % chunk
        assert np.array_equal(full.leaves(), res["leaves"]), "chunk %d" % chunk
        _compare_fields(sim, ref)
        _compare_fields(full, ref)
        assert sim.time()[:2] == (ref.t, ref.dt)
    _, lu, au, _, _ = sim.counters()
    _, lu_f, au_f, _, _ = full.counters()
    assert lu == lu_f == ref.leaf_updates and au_f == lu_f
    if relief > 0:
        assert au < 0.5 * lu
    sim.close()
    full.close()


def test_listed_encode_tiles_L11():
    # 2048 x 2048, water released on rough dry ground: more tiles (4096)
    # than the first encode pass has CTAs, so it works from the list of
    # non-quiescent tiles; 16-step graphs; against the oracle and the full
    # sweep
    p, f = synth.dry_bed_dam_break(L=11, eps=1e-3, relief=0.05)
    sim = _sim(p, f)
    full = _sim(dict(p, full_sweep=True), f)
    ref = oracle.State(p, f)
    sim.advance(max_steps=17)
    full.advance(max_steps=17)
    for _ in range(16):
        ref.step()
    res = ref.step(want=("leaves",))
    assert np.array_equal(sim.leaves(), res["leaves"])
    assert np.array_equal(full.leaves(), res["leaves"])
    _compare_fields(sim, ref)
    _compare_fields(full, ref)
    assert sim.time()[:2] == (ref.t, ref.dt)
    _, lu, au, _, _ = sim.counters()
    assert au < 0.5 * lu
    sim.close()
    full.close()


def test_uniform_fv1_matches_oracle():
    # hwfv1_advance_uniform: uniform FV1 on the finest grid (the comparison
    # solver), against the oracle's uniform step, bit for bit
    p, f = synth.circular_dam_break(L=6, eps=1e-3)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    for chunk in range(4):
        sim.advance_uniform(max_steps=5)
        for _ in range(5):
            ref.fv1_step()
        _compare_fields(sim, ref)
        t, dt, steps = sim.time()
        assert (t, dt, steps) == (ref.t, ref.dt, ref.steps)
    sim.close()


def test_uniform_fv1_with_friction_and_inflow():
    p, f = synth.terrain_flood(L=8, fill=2.0, fill_q=1.0)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    sim.advance_uniform(max_steps=6)
    for _ in range(6):
        ref.fv1_step()
    _compare_fields(sim, ref, exact=False)
    sim.close()


def test_uniform_and_adaptive_steps_mix():
    # adaptive steps (with quiescent tiles skipped), then uniform steps, then
    # adaptive again on dry rough ground: the same as the oracle's sequence
    p, f = synth.dry_bed_dam_break(L=8, eps=1e-3, relief=0.05)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    sim.advance(max_steps=8)
    for _ in range(8):
        ref.step()
    sim.advance_uniform(max_steps=8)
    for _ in range(8):
        ref.fv1_step()
    sim.advance(max_steps=8)
    for _ in range(7):
        ref.step()
    res = ref.step(want=("leaves",))
    assert np.array_equal(sim.leaves(), res["leaves"])
    _compare_fields(sim, ref)
    assert sim.time()[:2] == (ref.t, ref.dt)
    sim.close()


def test_top_of_range_L13_one_step_matches_oracle():
    # 8192 x 8192 (67 M finest cells), the circular dam-break: one step of
    # the graph-replay path against one oracle step, leaves and fields bit
    # for bit (the level offsets, 28-bit Morton codes and tile counts of the
    # top of the accepted range, L <= 14, in use)
    p, f = synth.circular_dam_break(L=13, eps=1e-3)
    sim = _sim(p, f)
    ref = oracle.State(p, f)
    assert sim.time()[1] == ref.dt
    sim.advance(max_steps=1)
    res = ref.step(want=("leaves",))
    lv = sim.leaves()
    assert len(lv) == res["num_leaves"] and np.array_equal(lv, res["leaves"])
    _compare_fields(sim, ref)
    sim.close()


def test_top_of_range_L14_keeps_the_symmetries():
    # 16384 x 16384 (268 M finest cells): too large for the oracle in a
    # test, so the properties the oracle pins for this case hold instead --
    # the circular dam-break stays symmetric under the transpose (hu and hv
    # swap) and under both mirrors (the normal discharge flips) up to the
    # rounding of the x- and y-sums' different order (1e-12, as the oracle's
    # pin), and the leaves tile the domain
    p, f = synth.circular_dam_break(L=14, eps=1e-3)
    sim = _sim(p, f)
    del f
    sim.advance(max_steps=3)
    g = sim.fields()
    h, qx, qy = g["h"], g["qx"], g["qy"]
    assert np.isfinite(h).all() and h.max() > 1.0 and np.abs(qx).max() > 0.0
    tol = 1e-12
    assert np.abs(h - h.T).max() <= tol and np.abs(qx - qy.T).max() <= tol
    assert np.abs(h - h[::-1, :]).max() <= tol and np.abs(qy + qy[::-1, :]).max() <= tol
    assert np.abs(h - h[:, ::-1]).max() <= tol and np.abs(qx + qx[:, ::-1]).max() <= tol
    lv = (sim.leaves() >> 28).astype(np.int64)
    assert np.sum(np.ldexp(1.0, -2 * lv)) == 1.0
    sim.close()


def test_fp64_throughput_probe():
    # the measured DADD rate behind the roofline's context figure: positive
    # and below the FP64 pipe's nominal rate (2 per cycle per SM)
    import torch
    from paper_2206_05761_gb300 import hwfv1 as Hh
    v = Hh.hwfv1_fp64_throughput()
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 2 * 2.2e9 / 1e12
    assert 0.0 < v <= nominal
