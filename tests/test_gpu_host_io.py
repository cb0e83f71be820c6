"""Host buffers at the C ABI: hwfv1_init reads its four fields from device,
pinned host or pageable host memory (copied in by the library, the bed
first) and hwfv1_get_fields writes into any of them.  Every combination must
give the run the device buffers give, bit for bit, and the host path must
match the CPU oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

KEYS = ("z", "h", "qx", "qy")


def _tensors(f, kind):
    import torch
    out = {}
    for i, k in enumerate(KEYS):
        a = torch.from_numpy(np.ascontiguousarray(f[k], dtype=np.float64).reshape(-1).copy())
        kk = kind if isinstance(kind, str) else kind[i]
        if kk == "device":
            a = a.cuda()
        elif kk == "pinned":
            a = a.pin_memory()
        out[k] = a                      # "pageable": ordinary host memory
    return out


def _run(p, f, kind, steps):
    """Init from buffers of the given kind(s), advance, return the fields
    read into device buffers (numpy)."""
    import torch
    from paper_2206_05761_gb300 import hwfv1 as H
    t = _tensors(f, kind)
    hd = H.hwfv1_init(H.make_problem(p, 64), t["z"], t["h"], t["qx"], t["qy"])
    try:
        H.hwfv1_advance(hd, float("inf"), steps)
        N = 1 << (2 * p["L"])
        out = {k: torch.empty(N, dtype=torch.float64, device="cuda") for k in ("h", "qx", "qy")}
        H.hwfv1_get_fields(hd, out["h"], out["qx"], out["qy"])
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}, H.hwfv1_get_time(hd)
    finally:
        H.hwfv1_destroy(hd)


def _same(a, b):
    for k in ("h", "qx", "qy"):
        assert np.array_equal(a[k].view(np.uint64), b[k].view(np.uint64)), k


@pytest.mark.parametrize("kind", ["pinned", "pageable", ("pageable", "device", "pinned", "device"),
                                  ("device", "pinned", "device", "pageable")])
def test_init_from_host_buffers_gives_the_device_run(kind):
    p, f = synth.terrain_flood(L=8)
    ref, tref = _run(p, f, "device", 24)
    got, tgot = _run(p, f, kind, 24)
    _same(ref, got)
    assert tref == tgot


@pytest.mark.parametrize("L", [1, 2, 5])
def test_host_init_small_grids(L):
    p, f = synth.circular_dam_break(L=L, eps=1e-3)
    ref, _ = _run(p, f, "device", 3)
    got, _ = _run(p, f, "pinned", 3)
    _same(ref, got)


def test_host_init_matches_the_oracle():
    p, f = synth.circular_dam_break(L=7, eps=1e-3)
    got, (t, dt, steps) = _run(p, f, "pageable", 5)
    ref = oracle.State(p, f)
    for _ in range(5):
        ref.step()
    for k in ("h", "qx", "qy"):
        assert np.array_equal(got[k], np.asarray(getattr(ref, k)).reshape(-1)), k
    assert t == ref.t and dt == ref.dt


@pytest.mark.parametrize("store", [False, True])
def test_get_fields_into_host_buffers(store):
    """Outputs on the device, pinned and pageable, some NULL; with the leaf
    store on, the fields are formed from the stored levels first."""
    import torch
    from paper_2206_05761_gb300 import hwfv1 as H
    p, f = synth.bumpy_dam_break(L=8, eps=1e-3)
    t = _tensors(f, "device")
    hd = H.hwfv1_init(H.make_problem(p, 64), t["z"], t["h"], t["qx"], t["qy"])
    try:
        if store:
            H.hwfv1_set_leaf_store(hd, True)
        H.hwfv1_advance(hd, float("inf"), 12)
        N = 1 << 16
        dev = {k: torch.empty(N, dtype=torch.float64, device="cuda") for k in ("h", "qx", "qy")}
        H.hwfv1_get_fields(hd, dev["h"], dev["qx"], dev["qy"])
        torch.cuda.synchronize()
        ref = {k: v.cpu().numpy() for k, v in dev.items()}
        pin = {k: torch.full((N,), np.nan, dtype=torch.float64).pin_memory() for k in ("h", "qx", "qy")}
        H.hwfv1_get_fields(hd, pin["h"], pin["qx"], pin["qy"])     # written when the call returns
        _same(ref, {k: v.numpy() for k, v in pin.items()})
        pag = {k: torch.full((N,), np.nan, dtype=torch.float64) for k in ("h", "qx", "qy")}
        H.hwfv1_get_fields(hd, pag["h"], None, pag["qy"])
        assert np.array_equal(pag["h"].numpy().view(np.uint64), ref["h"].view(np.uint64))
        assert np.array_equal(pag["qy"].numpy().view(np.uint64), ref["qy"].view(np.uint64))
        assert np.isnan(pag["qx"].numpy()).all()
        # a mix: h to the device, qx pinned, qy pageable
        d2 = torch.empty(N, dtype=torch.float64, device="cuda")
        p2 = torch.empty(N, dtype=torch.float64).pin_memory()
        g2 = torch.empty(N, dtype=torch.float64)
        H.hwfv1_get_fields(hd, d2, p2, g2)
        torch.cuda.synchronize()
        _same(ref, {"h": d2.cpu().numpy(), "qx": p2.numpy(), "qy": g2.numpy()})
        # the run goes on as if the fields had not been read
        H.hwfv1_advance(hd, float("inf"), 4)
        H.hwfv1_get_fields(hd, pin["h"], pin["qx"], pin["qy"])
    finally:
        H.hwfv1_destroy(hd)
    again, _ = _run_store(p, f, store, 16)
    _same(again, {k: v.numpy() for k, v in pin.items()})


def _run_store(p, f, store, steps):
    import torch
    from paper_2206_05761_gb300 import hwfv1 as H
    t = _tensors(f, "device")
    hd = H.hwfv1_init(H.make_problem(p, 64), t["z"], t["h"], t["qx"], t["qy"])
    try:
        if store:
            H.hwfv1_set_leaf_store(hd, True)
        H.hwfv1_advance(hd, float("inf"), 12)
        H.hwfv1_advance(hd, float("inf"), steps - 12)
        N = 1 << (2 * p["L"])
        out = {k: torch.empty(N, dtype=torch.float64, device="cuda") for k in ("h", "qx", "qy")}
        H.hwfv1_get_fields(hd, out["h"], out["qx"], out["qy"])
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}, None
    finally:
        H.hwfv1_destroy(hd)
