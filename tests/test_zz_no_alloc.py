"""hwfv1_traverse_noalloc, the traversal entry point for callers that cannot
allocate device memory (its scratch is a fixed array inside the library),
must give exactly the leaf list of the regular hwfv1_traverse, and at the
scratch's full size (L=12, 16,384 tiles) the oracle's depth-first leaves.
Kept in a file that pytest collects last."""
import numpy as np
import pytest

import oracle
import synth
from _util import pack_bits

pytestmark = pytest.mark.gpu


def _regular(sim):
    """Leaves and regularised bits of the simulation's current state, from the
    regular entry points (encode, flag, traverse)."""
    import torch
    from paper_2206_05761_gb300 import hwfv1 as H
    sim.encode()
    sim.flag()
    n = sim.traverse(want_count=True)
    words = torch.zeros(max(H.bits_words(sim.L), 1), dtype=torch.int32, device="cuda")
    H.hwfv1_get_flags(sim.hd, 1, words)
    return sim.leaves(), words, n


def _noalloc(words, L, cap):
    import torch
    from paper_2206_05761_gb300 import hwfv1 as H
    leaves = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    H.hwfv1_traverse_noalloc(words, L, leaves, count)
    torch.cuda.synchronize()
    n = int(count.item())
    return leaves.cpu().numpy().view(np.uint32)[:min(n, cap)], n


def test_noalloc_traverse_matches_regular_on_two_calls():
    import torch
    from paper_2206_05761_gb300.sim import Simulation
    # calls in a row on different trees (different sizes, so a call must not
    # see the previous call's scratch); below L=5 one tile is the whole grid
    cases = [synth.bumpy_dam_break(L=9, eps=1e-3), synth.circular_dam_break(L=6, eps=1e-3),
             synth.circular_dam_break(L=4, eps=1e-3), synth.circular_dam_break(L=2, eps=1e-3),
             synth.circular_dam_break(L=1, eps=1e-3)]
    for p, f in cases:
        sim = Simulation(p, f)
        sim.advance(max_steps=3)
        expect, words, n = _regular(sim)
        got, m = _noalloc(words, p["L"], cap=1 << (2 * p["L"]))
        assert m == n == len(expect)
        assert np.array_equal(got, expect)
        sim.close()
    torch.cuda.synchronize()


def test_noalloc_traverse_cut_list_and_limits():
    import torch
    from paper_2206_05761_gb300 import hwfv1 as H
    from paper_2206_05761_gb300.sim import Simulation
    p, f = synth.circular_dam_break(L=5, eps=1e-3)
    sim = Simulation(p, f)
    expect, words, n = _regular(sim)
    got, m = _noalloc(words, 5, cap=7)          # cut: the count is still the full one
    assert m == n and np.array_equal(got, expect[:7])
    with pytest.raises(H.Hwfv1Error) as e:      # beyond the scratch's L <= 12
        H.hwfv1_traverse_noalloc(words, 13, torch.zeros(4, dtype=torch.int32, device="cuda"),
                                 torch.zeros(1, dtype=torch.int32, device="cuda"))
    assert e.value.status == 1
    sim.close()


def test_noalloc_traverse_full_scratch_L12_matches_oracle_dft():
    import torch
    # the terrain flood's first step at L=12: the oracle's regularised flags
    # (bed details flag most of the domain) give 4^7 = 16,384 tiles, the
    # scratch's full size; the leaves must be the oracle's depth-first list
    p, f = synth.terrain_flood(L=12)
    res = oracle.State(p, f).step(want=("S", "leaves"))
    words = torch.from_numpy(pack_bits(res["S"], 12).view(np.int32)).cuda()
    n_exp = res["num_leaves"]
    for _ in range(2):
        got, m = _noalloc(words, 12, cap=1 << 24)
        assert m == n_exp
        assert np.array_equal(got, res["leaves"])
    torch.cuda.synchronize()
