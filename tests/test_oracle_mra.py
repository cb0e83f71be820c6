"""Pins of the oracle's indexing, Haar encode/decode and significance flags
against what the paper and the mathematics fix (no GPU)."""
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# Indexing (Sec. 2.2.1, Fig. 5, footnote 2)
# --------------------------------------------------------------------------

def test_morton_matches_fig5b_table():
    rows = _rows("fig5b_morton.txt")
    for j, row in enumerate(rows):
        for i, v in enumerate(row):
            assert oracle.morton(i, j) == int(v)


def test_morton_matches_fig5a_binary_table():
    rows = _rows("fig5a_morton_binary.txt")
    for j, row in enumerate(rows):
        for i, v in enumerate(row):
            assert oracle.morton(i, j) == int(v, 2)


def test_zindex_footnote2():
    # finest cell with Morton code 3 at L = 2 has Z-order index 8
    assert oracle.zindex(2, 3) == 8
    # levels are contiguous: level n starts where level n-1 ends
    for n in range(1, 12):
        assert oracle.zindex(n, 0) == oracle.zindex(n - 1, (1 << (2 * (n - 1))) - 1) + 1


def test_demorton_inverts_morton():
    rng = np.random.default_rng(0)
    for i, j in rng.integers(0, 1 << 16, size=(200, 2)):
        assert oracle.demorton(oracle.morton(int(i), int(j))) == (int(i), int(j))


def test_children_are_contiguous_in_zorder():
    # Sec. 2.2.1: the four children of a parent are consecutive Morton codes
    for i in range(8):
        for j in range(8):
            c = oracle.morton(i, j)
            kids = [oracle.morton(2 * i + (k & 1), 2 * j + (k >> 1)) for k in range(4)]
            assert kids == [4 * c + k for k in range(4)]


# --------------------------------------------------------------------------
# Haar encoding / decoding (Eq. 3, Eq. 4)
# --------------------------------------------------------------------------

def test_parent_is_block_average():
    L = 6
    x = synth.random_state(L, seed=1)
    hier, _ = oracle.encode(L, x)
    for n in range(L + 1):
        w = 1 << (L - n)
        avg = x.reshape(1 << n, w, 1 << n, w).mean(axis=(1, 3))
        np.testing.assert_allclose(oracle.level(hier, n), avg, rtol=0, atol=1e-13)


@pytest.mark.parametrize("A,B", [(3.0, -5.0), (0.0, 1.0), (2.0, 0.0), (-0.75, 0.25)])
def test_linear_field_details_closed_form(A, B):
    # f(i, j) = A*i + B*j: at level n the details are
    # d_alpha = -B*2^(L-n-2), d_beta = -A*2^(L-n-2), d_gamma = 0 (exact)
    L = 5
    j, i = np.mgrid[0:1 << L, 0:1 << L].astype(np.float64)
    f = A * i + B * j
    _, det = oracle.encode(L, f)
    for n in range(L):
        s = 1 << n
        d = det[oracle.level_start(n): oracle.level_start(n) + s * s]
        w = 2.0 ** (L - n - 2)
        assert np.all(d[:, 0] == -B * w)
        assert np.all(d[:, 1] == -A * w)
        assert np.all(d[:, 2] == 0.0)


@pytest.mark.parametrize("pattern,which", [("stripes_i", 1), ("stripes_j", 0), ("checker", 2)])
def test_alternating_patterns_select_one_detail(pattern, which):
    # (-1)^i varies along x only -> d_beta; (-1)^j -> d_alpha; (-1)^(i+j) -> d_gamma
    L = 3
    j, i = np.mgrid[0:1 << L, 0:1 << L]
    f = {"stripes_i": (-1.0) ** i, "stripes_j": (-1.0) ** j, "checker": (-1.0) ** (i + j)}[pattern]
    hier, det = oracle.encode(L, f)
    n = L - 1
    s = 1 << n
    d = det[oracle.level_start(n): oracle.level_start(n) + s * s]
    expect = np.zeros(3)
    expect[which] = 1.0
    assert np.all(d == expect)
    assert np.all(oracle.level(hier, n) == 0.0)


def test_constant_children_give_zero_details():
    for v in [0.0, 1.0, -3.5, 1e-300, 7.123456789e5]:
        o = oracle.encode_parent([v, v, v, v])
        assert o[0] == v and o[1] == 0.0 and o[2] == 0.0 and o[3] == 0.0


def test_roundtrip_exact_for_dyadic_values():
    L = 6
    x = synth.random_state(L, seed=2, dyadic=True)
    hier, det = oracle.encode(L, x)
    y = oracle.decode_all(L, hier, det)
    assert np.array_equal(x, y)


def test_roundtrip_close_for_random_values():
    L = 6
    x = synth.random_state(L, seed=3)
    hier, det = oracle.encode(L, x)
    y = oracle.decode_all(L, hier, det)
    # each level of the round trip adds at most a few ulp of max|x|
    assert np.max(np.abs(y - x)) <= 4 * L * np.finfo(float).eps * np.max(np.abs(x))


def test_decode_parent_inverts_encode_parent():
    rng = np.random.default_rng(4)
    for _ in range(100):
        c = rng.integers(-1000, 1000, size=4).astype(float) / 8.0
        assert np.array_equal(oracle.decode_parent(oracle.encode_parent(c)), c)


# --------------------------------------------------------------------------
# Significance flags (Sec. 2.1.2, Algorithm 1)
# --------------------------------------------------------------------------

def _flags(p, f):
    L = p["L"]
    dets, sm = [], []
    for q in ("h", "qx", "qy", "z"):
        _, d = oracle.encode(L, f[q])
        dets.append(d)
        sm.append(oracle.smax(L, f[q]))
    return oracle.threshold_flags(L, p["eps"], dets, sm)


def test_eps_zero_flags_everything():
    p, f = synth.bumpy_dam_break(L=5, eps=0.0)
    T = _flags(p, f)
    assert T.size == oracle.level_start(5) and np.all(T == 1)
    # and the flat, still case too: every detail (0) >= 0
    p, f = synth.lake_at_rest(L=4, eps=0.0)
    f["z"][:] = 0.0
    assert np.all(_flags(p, f) == 1)


def test_huge_eps_on_flat_still_water_gives_single_root_leaf():
    p, f = synth.lake_at_rest(L=5, eps=1e300)
    f["z"][:] = 0.0
    T = _flags(p, f)
    assert np.all(T == 0)
    S = oracle.regularise(5, T)
    leaves = oracle.leaves_dft(5, S)
    assert list(leaves) == [0]


def test_threshold_uses_greater_or_equal():
    # L = 1: h children [2, 0, 2, 0] -> d_beta = 1, s_max,h = 2; the level-0
    # threshold is eps*2^-1*2 = eps, so eps = 1 sits exactly on the boundary
    p = synth.problem(1)
    h = np.array([[2.0, 0.0], [2.0, 0.0]])
    zero = np.zeros((2, 2))
    f = dict(h=h, qx=zero, qy=zero, z=zero)
    for eps, expect in [(1.0, 1), (np.nextafter(1.0, 2.0), 0), (np.nextafter(1.0, 0.0), 1)]:
        p["eps"] = eps
        assert _flags(p, f)[0] == expect


def test_smax_has_floor_one():
    assert oracle.smax(2, np.zeros((4, 4))) == 1.0
    assert oracle.smax(2, np.full((4, 4), -3.0)) == 3.0


def test_bed_alone_can_flag():
    p, f = synth.lake_at_rest(L=5, eps=1e-3)
    f["h"][:] = 1.0
    T = _flags(p, f)
    assert T.any()
    f["z"][:] = 0.0
    assert not _flags(p, f).any()


def test_flags_symmetric_under_transpose():
    # transposing swaps d_alpha and d_beta, the max is unchanged
    p, f = synth.bumpy_dam_break(L=5, eps=1e-3, seed=9)
    g = {k: np.ascontiguousarray(v.T) for k, v in f.items()}
    g["qx"], g["qy"] = np.ascontiguousarray(f["qy"].T), np.ascontiguousarray(f["qx"].T)
    T1, T2 = _flags(p, f), _flags(p, g)
    for n in range(p["L"]):
        s = 1 << n
        a = T1[oracle.level_start(n): oracle.level_start(n) + s * s].reshape(s, s)
        b = T2[oracle.level_start(n): oracle.level_start(n) + s * s].reshape(s, s)
        assert np.array_equal(a, b.T)
