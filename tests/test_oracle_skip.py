"""Pins of the oracle's learned subtree skip (reading R-skip: each level-(L-4)
subtree encoded, flagged and stored only down to its predicted level) against
what fixes it independently of its own code (no GPU):
- every predicted level at L is the plain step, bit for bit;
- every predicted level at L-4 is the plain step of the problem coarsened to
  level L-4 (the same arithmetic on the level-(L-4) coefficients, with the
  threshold's level scaling eps 2^(n-L) written for that problem);
- a skip step reads only stored values (everything else poisoned with NaN);
- no leaf of a subtree is finer than its predicted level;
- a lake at rest stays at rest whatever the predicted levels.
"""
import numpy as np
import pytest

import oracle
import synth


def _levels(rng, Ls, L):
    n = 1 << Ls
    return rng.integers(Ls, L + 1, size=(n, n)).astype(np.uint8)


def test_skip_at_full_depth_is_the_plain_step():
    p, f = synth.bumpy_dam_break(L=6, eps=1e-3, seed=5)
    a, b = oracle.State(p, f), oracle.SkipState(p, f)
    assert a.dt == b.dt
    for k in range(8):
        ra = a.step(want=("leaves", "S"))
        # every third step the exact audit (from a state stored at level L)
        rb = b.plain_step(want=("S",)) if k % 3 == 2 else b.skip_step(np.full((4, 4), 6), want=("S",))
        assert np.array_equal(ra["leaves"], rb["leaves"]) and np.array_equal(ra["S"], rb["S"]), k
        g = b.fields()
        for q in ("h", "qx", "qy"):
            assert np.array_equal(getattr(a, q), g[q]), (k, q)
        assert a.t == b.t and a.dt == b.dt
    assert np.all(b.m == 6)


@pytest.mark.parametrize("L,eps", [(7, 1e-3), (8, 1e-2)])
def test_skip_at_subtree_level_is_the_coarsened_plain_step(L, eps):
    # every subtree cut at level Ls = L-4: its leaves are no finer than Ls and
    # it is stored at Ls, so the step is the plain step of the problem whose
    # finest grid is level Ls (the level-Ls coefficients of the state and the
    # bed), with the threshold eps 2^(n-L) = (eps/16) 2^(n-Ls).  The values
    # stay within 1, so s_max is 1 on both sides; the steps are given.
    Ls = L - 4
    p, f = synth.bumpy_dam_break(L=L, eps=eps, seed=5, eta_up=1.0, eta_down=0.5)
    b = oracle.SkipState(p, f)
    pc = dict(p, L=Ls, eps=eps / 16)
    fc = {k: oracle.level(oracle.encode(L, f[k])[0], Ls).copy() for k in ("h", "qx", "qy", "z")}
    a = oracle.State(pc, fc)
    cut = np.full((1 << Ls, 1 << Ls), Ls)
    adaptive = False
    for k, dt in enumerate([1e-3, 2e-3, 1.5e-3, 1e-3, 2e-3, 2e-3]):
        rb = b.skip_step(cut, dt=dt)
        ra = a.step(dt=dt, want=("leaves",))
        assert np.array_equal(ra["leaves"], rb["leaves"]), k
        adaptive = adaptive or ra["num_leaves"] < (1 << (2 * Ls))
        assert np.all(b.m == Ls)
        blocks = b.stored()
        n = 1 << Ls
        for iq, q in enumerate(("h", "qx", "qy")):
            got = np.array([blk[1 + iq][0, 0] for blk in blocks]).reshape(n, n)
            assert np.array_equal(got, getattr(a, q)), (k, q)
        for q in ("h", "qx", "qy"):
            assert np.abs(getattr(a, q)).max() <= 1.0
        assert a.t == b.t
    assert adaptive or L == 7


POISON = 1e6


def _poison(st):
    """Poison everywhere in the hierarchies except each subtree's stored
    cells: a wet, finite value far outside the flow (non-finite values would
    be laundered by the wet/dry tests), which any read of it carries into
    the coefficients, fluxes and stored values."""
    L, Ls = st.L, st.Ls
    keep = [(ms, *[v.copy() for v in vals]) for ms, *vals in st.stored()]
    st.hier[:] = POISON
    n = 1 << Ls
    for s, (ms, *vals) in enumerate(keep):
        sj, si = divmod(s, n)
        w = 1 << (ms - Ls)
        for q in range(3):
            lev = st.hier[q, oracle.level_start(ms): oracle.level_start(ms) + (1 << (2 * ms))].reshape(1 << ms, 1 << ms)
            lev[sj * w:(sj + 1) * w, si * w:(si + 1) * w] = vals[q]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_skip_step_reads_only_the_stored_state(seed):
    # a neighbour cell, a coarser coefficient or a cell below a subtree's
    # storage level that the step used without forming it would carry the
    # poison into the result
    rng = np.random.default_rng(seed)
    p, f = synth.bumpy_dam_break(L=7, eps=1e-3, seed=seed, eta_up=1.4)
    st = oracle.SkipState(p, f)
    for k in range(6):
        _poison(st)
        res = st.skip_step(_levels(rng, 3, 7))
        for ms, *vals in st.stored():
            for v in vals:
                assert np.abs(v).max() < 1e3, k
        assert np.isfinite(st.dt) and res["num_leaves"] > 0
    _poison(st)
    st.plain_step()
    for v in st.fields().values():
        assert np.abs(v).max() < 1e3


def test_no_leaf_finer_than_its_subtree_level():
    rng = np.random.default_rng(4)
    L, Ls = 7, 3
    p, f = synth.columns_dam_break(L=L, eps=1e-3, seed=2)
    st = oracle.SkipState(p, f)
    for k in range(5):
        lev = _levels(rng, Ls, L)
        res = st.skip_step(lev)
        for pk in res["leaves"]:
            n, code = int(pk >> 28), int(pk & 0x0FFFFFFF)
            if n <= Ls:
                continue
            i, j = oracle.demorton(code)
            assert n <= lev[j >> (n - Ls), i >> (n - Ls)], (k, n)
        # leaves tile the domain
        assert sum(4.0 ** -int(pk >> 28) for pk in res["leaves"]) == 1.0


def test_lake_at_rest_whatever_the_levels():
    # still water over a fully wet, uneven bed: restricting, prolonging and
    # storing at any level keeps the free surface flat, so nothing moves
    rng = np.random.default_rng(5)
    p, f = synth.lake_at_rest(L=7, eps=1e-3, eta=1.0, wet=True)
    st = oracle.SkipState(p, f)
    for k in range(40):
        st.skip_step(_levels(rng, 3, 7)) if k % 10 else st.plain_step()
    g = st.fields()
    assert np.abs(g["qx"]).max() <= 1e-10 and np.abs(g["qy"]).max() <= 1e-10
    assert np.abs(g["h"] + f["z"] - 1.0).max() <= 1e-12


def test_eps_zero_gives_each_subtree_a_uniform_grid_at_its_level():
    # with eps = 0 every detail the step forms is significant, so the leaves
    # of each subtree are exactly its cells at the predicted level; stripes of
    # full-depth and cut subtrees put fine leaves against cut subtrees on
    # every side, whose cells at those fine levels must have been formed
    # (everything not stored is poisoned)
    L, Ls = 6, 2
    p, f = synth.circular_dam_break(L=L, eps=0.0)
    n = 1 << Ls
    col, row = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    for k, lev in enumerate([np.where(col % 2 == 0, L, Ls),          # stripes along y
                             np.where(row % 2 == 1, L, Ls),          # stripes along x
                             np.where((col + row) % 2 == 0, L - 1, Ls + 1)]):   # checkerboard
        lev = lev.astype(np.uint8)
        st = oracle.SkipState(p, f)
        for _ in range(3):
            _poison(st)
            res = st.skip_step(lev)
            got = {}
            for pk in res["leaves"]:
                lv, code = int(pk >> 28), int(pk & 0x0FFFFFFF)
                i, j = oracle.demorton(code)
                s = (j >> (lv - Ls), i >> (lv - Ls))
                got.setdefault(s, set()).add(lv)
            for sj in range(n):
                for si in range(n):
                    assert got[(sj, si)] == {int(lev[sj, si])}, (k, sj, si)
            for ms, *vals in st.stored():
                for v in vals:
                    assert np.abs(v).max() < 1e3, k


def test_subtree_details_below_the_prediction_are_not_tested():
    # still water over a bed that is flat at the level of the subtrees
    # (L-4) but not one level finer: a +a/-a pattern over each subtree's
    # four level-(L-3) cells.  Cut at L-4, nothing is significant and the
    # whole domain is one leaf; at full depth the bed's details refine it
    L, Ls = 6, 2
    p, f = synth.lake_at_rest(L=L, eps=1e-3, eta=1.0, wet=True)
    n = 1 << L
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    w = 1 << (L - Ls - 1)
    z = 0.3 + 0.1 * np.where(((i // w) + (j // w)) % 2 == 0, 1.0, -1.0)
    f = dict(f, z=z, h=1.0 - z, qx=np.zeros_like(z), qy=np.zeros_like(z))
    cut = oracle.SkipState(p, f).skip_step(np.full((1 << Ls, 1 << Ls), Ls))
    assert cut["num_leaves"] == 1 and int(cut["leaves"][0]) == 0
    full = oracle.SkipState(p, f).skip_step(np.full((1 << Ls, 1 << Ls), L))
    assert full["num_leaves"] > 1 << (2 * Ls)
