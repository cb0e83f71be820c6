"""Pins of the oracle's regularisation and leaf identification: the worked
example of Sec. 2.2.2-2.2.3, brute force over tiny trees, and the tiling
invariant (no GPU)."""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _ls(n):
    return oracle.level_start(n)


def _morton_order_to_rowmajor(L, bits_morton):
    """Significance given per level in Morton order -> oracle layout
    (row-major per level)."""
    out = np.zeros(_ls(L), np.uint8)
    for n in range(L):
        s = 1 << n
        for code in range(s * s):
            i, j = oracle.demorton(code)
            out[_ls(n) + j * s + i] = bits_morton[_ls(n) + code]
    return out


def _brute_leaves(L, S):
    """Leaves by definition: cells whose strict ancestors are all
    significant and which are either finest or not significant; returned as
    Z-order indices sorted by the Morton code of their first finest cell."""
    out = []
    for n in range(L + 1):
        s = 1 << n
        for code in range(s * s):
            ok = True
            for k in range(n):
                c = code >> (2 * (n - k))
                i, j = oracle.demorton(c)
                if not S[_ls(k) + j * (1 << k) + i]:
                    ok = False
                    break
            if not ok:
                continue
            i, j = oracle.demorton(code)
            if n == L or not S[_ls(n) + j * s + i]:
                out.append((code << (2 * (L - n)), oracle.zindex(n, code)))
    return [z for _, z in sorted(out)]


def _unpack(L, packed):
    return [oracle.zindex(int(p) >> 28, int(p) & 0x0FFFFFFF) for p in packed]


def test_worked_example_of_sec_2_2():
    with open(os.path.join(GOLD, "ptt_worked_example.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    sig = np.array([int(v) for v in rows[0] + rows[1]], np.uint8)
    ptt_expect = [int(v) for v in rows[2]]
    leaves_expect = [int(v) for v in rows[3]]
    L = 2
    S = _morton_order_to_rowmajor(L, sig)
    ptt = oracle.leaves_ptt(L, S)
    assert list(ptt) == ptt_expect
    assert _unpack(L, oracle.leaves_dft(L, S)) == leaves_expect
    # duplicates removed in order = DFT order
    dedup = [v for k, v in enumerate(ptt) if k == 0 or v != ptt[k - 1]]
    assert dedup == leaves_expect


def test_dft_ptt_bruteforce_exhaustive_L2():
    L = 2
    P = _ls(L)
    for mask in range(1 << P):
        S = np.array([(mask >> b) & 1 for b in range(P)], np.uint8)
        dft = _unpack(L, oracle.leaves_dft(L, S))
        ptt = oracle.leaves_ptt(L, S)
        dedup = [v for k, v in enumerate(ptt) if k == 0 or v != ptt[k - 1]]
        assert dft == dedup == _brute_leaves(L, S)


@pytest.mark.parametrize("L", [3, 4, 5, 6])
def test_dft_ptt_bruteforce_random(L):
    rng = np.random.default_rng(L)
    for trial in range(6 if L < 6 else 2):
        T = (rng.random(_ls(L)) < rng.uniform(0.2, 0.8)).astype(np.uint8)
        for predict, close in itertools.product([0, 1], [0, 1]):
            S = oracle.regularise(L, T, predict, close)
            dft = _unpack(L, oracle.leaves_dft(L, S))
            ptt = oracle.leaves_ptt(L, S)
            dedup = [v for k, v in enumerate(ptt) if k == 0 or v != ptt[k - 1]]
            assert dft == dedup
            if L <= 4:
                assert dft == _brute_leaves(L, S)


@pytest.mark.parametrize("L", [2, 3, 5, 7])
def test_leaves_tile_the_domain(L):
    rng = np.random.default_rng(100 + L)
    T = (rng.random(_ls(L)) < 0.4).astype(np.uint8)
    S = oracle.regularise(L, T)
    leaves = oracle.leaves_dft(L, S)
    # areas 4^-n sum to one and the finest-cell ranges are disjoint and in order
    area = sum(4.0 ** -(int(p) >> 28) for p in leaves)
    assert area == 1.0
    pos = 0
    for p in leaves:
        n, code = int(p) >> 28, int(p) & 0x0FFFFFFF
        first = code << (2 * (L - n))
        assert first == pos
        pos += 1 << (2 * (L - n))
    assert pos == 1 << (2 * L)


def _subtree_any(L, T, n, i, j):
    for m in range(n, L):
        w = 1 << (m - n)
        blk = T[_ls(m): _ls(m) + (1 << (2 * m))].reshape(1 << m, 1 << m)
        if blk[j * w:(j + 1) * w, i * w:(i + 1) * w].any():
            return True
    return False


@pytest.mark.parametrize("predict,close", [(1, 1), (1, 0), (0, 1), (0, 0)])
def test_regularisation_characterisation(predict, close):
    # Brute-force statement of the regularised significance at (n, i, j):
    #  closure part: some threshold flag in the subtree rooted at (n, i, j)
    #                (or the cell's own flag without closure);
    #  prediction part: the parent's threshold flag.
    L = 4
    rng = np.random.default_rng(7)
    for _ in range(5):
        T = (rng.random(_ls(L)) < 0.15).astype(np.uint8)
        S = oracle.regularise(L, T, predict, close)
        for n in range(L):
            s = 1 << n
            for j in range(s):
                for i in range(s):
                    own = _subtree_any(L, T, n, i, j) if close else bool(T[_ls(n) + j * s + i])
                    par = bool(predict and n >= 1 and
                               T[_ls(n - 1) + (j // 2) * (s // 2) + i // 2])
                    assert S[_ls(n) + j * s + i] == int(own or par)


def test_closed_tree_has_significant_ancestors():
    L = 5
    rng = np.random.default_rng(8)
    T = (rng.random(_ls(L)) < 0.05).astype(np.uint8)
    S = oracle.regularise(L, T, 1, 1)
    for n in range(1, L):
        s = 1 << n
        for j in range(s):
            for i in range(s):
                if S[_ls(n) + j * s + i]:
                    assert S[_ls(n - 1) + (j // 2) * (s // 2) + i // 2]


def test_prediction_refines_one_level_below_threshold_tree():
    # one significant detail at level 1 of an L = 3 tree: R1 makes its four
    # children (level 2) significant, R2 makes the root significant; leaves
    # are the 16 finest cells under that level-1 cell and the 3 other
    # level-1 cells
    L = 3
    T = np.zeros(_ls(L), np.uint8)
    T[_ls(1) + 0] = 1              # level-1 cell (0, 0)
    S = oracle.regularise(L, T)
    leaves = _unpack(L, oracle.leaves_dft(L, S))
    expect = [oracle.zindex(3, c) for c in range(16)] + [oracle.zindex(1, c) for c in (1, 2, 3)]
    assert leaves == expect


def test_subtrees_under_leaves_on_a_flat_bed_encode_to_the_leaf_value():
    # After a step, R-decode hands every leaf's new (h, hu, hv) to all the
    # finest cells under it; on a flat bed the depth too is constant there.
    # Re-encoding then gives the leaf's value at every level of its subtree
    # (the average of four equal values is that value, bit for bit) and +0
    # for every detail: the exactness an encode restricted to the tree
    # relies on.
    p, f = synth.pseudo_2d_dam_break(L=6, eps=1e-3)
    st = oracle.State(p, f)
    for _ in range(30):
        st.step()
    res = st.step(want=("leaves",))
    L = p["L"]
    checked = 0
    for q in (st.h, st.qx, st.qy):
        hier, det = oracle.encode(L, q)
        for pk in res["leaves"]:
            n, code = int(pk) >> 28, int(pk) & 0x0FFFFFFF
            if n == L:
                continue
            i, j = oracle.demorton(code)
            v = q[j << (L - n), i << (L - n)]
            for m in range(n, L + 1):
                w = 1 << (m - n)
                blk = oracle.level(hier, m)[j * w:(j + 1) * w, i * w:(i + 1) * w]
                assert np.all(blk.view(np.uint64) == np.float64(v).view(np.uint64))
                if m < L:
                    s = 1 << m
                    rows = [oracle.level_start(m) + jj * s + ii
                            for jj in range(j * w, (j + 1) * w) for ii in range(i * w, (i + 1) * w)]
                    assert np.all(det[rows] == 0.0)
            checked += 1
    assert checked > 30
