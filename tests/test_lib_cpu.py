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
    return sorted(set(re.findall(r"\b(hwfv1_[a-z_]+)\s*\(", txt)))


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
