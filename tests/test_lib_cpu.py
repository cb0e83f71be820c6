"""The C-ABI library loads and exports every symbol of include/hwfv1.h, and
rejects bad problem descriptions before touching a GPU (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

import synth
from paper_2206_05761_gb300 import hwfv1 as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "hwfv1.h")).read()
    return sorted(set(re.findall(r"\b(hwfv1_[a-z0-9_]+)\s*\(", txt)))


def test_header_and_binding_agree():
    assert _declared() == sorted(H.exported_symbols())


def test_library_exports_every_declared_symbol():
    lib = H.lib()
    for name in _declared():
        assert hasattr(lib, name), name
    assert lib.hwfv1_version() == 1


def test_problem_struct_layout():
    # 10 doubles, 4 + 4*4 + 4*4 bytes of ints, 2 pointers
    assert C.sizeof(H.Problem) == 80 + 8 + 16 + 16 + 16


@pytest.mark.parametrize("field,value", [
    ("L", 0), ("L", 15), ("lx", 0.0), ("ly", -1.0), ("eps", -1e-3), ("eps", 1e-250),
    ("cfl", 0.0), ("cfl", 1.5), ("g", 0.0), ("manning_n", -0.1), ("tol_h", 0.0),
    ("dt_max", 0.0), ("precision", 16), ("flags", 16),
    ("flags", 8)])                 # flux matching without the upward closure
def test_invalid_spec_rejected_without_gpu(field, value):
    p, _ = synth.circular_dam_break(L=3)
    s = H.make_problem(p)
    setattr(s, field, value)
    hd = C.c_void_p()
    # NULL field pointers are never dereferenced: validation fails first
    st = H.lib().hwfv1_init(C.byref(s), None, None, None, None, None, C.byref(hd))
    assert st == 1 and not hd.value


def test_bad_inflow_rejected():
    p, _ = synth.inflow_basin(L=4)
    s = H.make_problem(p)
    s.inflow_a1 = 1 << 5          # past the side
    hd = C.c_void_p()
    assert H.lib().hwfv1_init(C.byref(s), None, None, None, None, None, C.byref(hd)) == 1
    s = H.make_problem(p)
    s.bc[1] = 2                   # two inflow sides
    assert H.lib().hwfv1_init(C.byref(s), None, None, None, None, None, C.byref(hd)) == 1


def test_null_handle_is_state_error():
    assert H.lib().hwfv1_encode(None) == 7
    assert H.lib().hwfv1_last_error(None) == b"NULL handle"
    # the learned skip and the exact leaf-value store check the handle first
    levels = (C.c_uint8 * 16)()
    assert H.lib().hwfv1_set_skip_levels(None, C.cast(levels, C.c_void_p), 10) == 7
    assert H.lib().hwfv1_get_skip_levels(None, 1, C.cast(levels, C.c_void_p), 16) == 7
    assert H.lib().hwfv1_set_leaf_store(None, 1) == 7
    assert H.lib().hwfv1_set_skipnet(None, None, 10, 0.0, 1) == 7


def _batch_init(specs, n, ptrs):
    """hwfv1_batch_init on host-side descriptions; ptrs[d] is the field
    pointer of member d (every field), or None.  Returns (status, handle)."""
    arr = (H.Problem * max(len(specs), 1))(*specs)
    fields = [(C.c_void_p * max(len(ptrs), 1))(*ptrs) for _ in range(4)]
    out = C.c_void_p()
    st = H.lib().hwfv1_batch_init(arr, n, *[C.cast(f, C.POINTER(C.c_void_p)) for f in fields], None, C.byref(out))
    return st, out.value


def _two(p=None):
    p = p or synth.circular_dam_break(L=3)[0]
    return [H.make_problem(p), H.make_problem(p)]


# A real host buffer stands for a device field: validation fails before any
# pointer is read.
_BUF = (C.c_double * 64)()


@pytest.mark.parametrize("case", ["empty", "mixed_precision", "flux_match", "null_field", "bad_member"])
def test_batch_init_rejects_bad_descriptions_without_gpu(case):
    specs, n, ptrs = _two(), 2, [C.addressof(_BUF)] * 2
    if case == "empty":
        n = 0
    elif case == "mixed_precision":
        specs[1].precision = 32
    elif case == "flux_match":
        specs[0].flags |= 8                  # HWFV1_FLUX_MATCH: single domains only
    elif case == "null_field":
        ptrs = [C.addressof(_BUF), None]
    elif case == "bad_member":
        specs[1].L = 0
    st, hd = _batch_init(specs, n, ptrs)
    assert st == 1 and not hd


def test_batch_init_needs_an_output_pointer():
    specs = _two()
    arr = (H.Problem * 2)(*specs)
    f = (C.c_void_p * 2)(C.addressof(_BUF), C.addressof(_BUF))
    pp = C.cast(f, C.POINTER(C.c_void_p))
    assert H.lib().hwfv1_batch_init(arr, 2, pp, pp, pp, pp, None, None) == 1


def test_null_batch_is_state_error():
    assert H.lib().hwfv1_batch_advance(None, 1.0, 1) == 7
    assert H.lib().hwfv1_batch_launches_per_step(None) == 0
    assert H.lib().hwfv1_batch_last_error(None) == b"NULL batch"


def test_network_parameter_count_matches_the_oracle_cnn():
    # w1[16][4][3][3], b1[16], w2[16][16][3][3], b2[16], w3[5][16][3][3], b3[5]
    import numpy as np
    from oracle import cnn
    params = cnn.init_params(np.random.default_rng(0))
    assert H.hwfv1_skipnet_num_params() == sum(a.size for a in params) == 3637


def test_null_network_arguments_are_rejected_without_gpu():
    L = H.lib()
    assert L.hwfv1_skipnet_create(1, None) == 1
    assert L.hwfv1_skipnet_set_params(None, None, 0) == 1
    assert L.hwfv1_skipnet_get_params(None, None, 0) == 1
    assert L.hwfv1_skipnet_forward(None, None, 1, 8, 8, None) == 1
    L.hwfv1_skipnet_destroy(None)              # a no-op


def test_field_pointers_take_contiguous_float64_only():
    """hwfv1_init and hwfv1_get_fields take device or host float64 buffers;
    the binding refuses other dtypes and strided views before any call."""
    import torch
    from paper_2206_05761_gb300 import hwfv1 as H
    assert H._ptr_io(None) is None
    x = torch.zeros(8, dtype=torch.float64)
    assert H._ptr_io(x) == x.data_ptr()
    with pytest.raises(ValueError):
        H._ptr_io(torch.zeros(8, dtype=torch.float32))
    with pytest.raises(ValueError):
        H._ptr_io(torch.zeros(8, 2, dtype=torch.float64)[:, 0])
