"""Python binding of the HWFV1 C ABI (include/hwfv1.h).

Argument marshalling only: every function here calls the same-named entry
point of libhwfv1.so, and every step of the method runs in that library's
CUDA kernels.  Device arrays are torch CUDA tensors (float64, contiguous,
row-major over the finest 2^L x 2^L grid); torch is used for device memory
and streams only.  Loading fails loudly if the library is missing: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

_lock = threading.Lock()
_lib = None

OK = 0
STATUS = {0: "HWFV1_OK", 1: "HWFV1_ERR_INVALID_SPEC", 2: "HWFV1_ERR_OOM", 3: "HWFV1_ERR_CUDA",
          4: "HWFV1_ERR_NONFINITE", 5: "HWFV1_ERR_NEG_DEPTH", 6: "HWFV1_ERR_TIMEOUT",
          7: "HWFV1_ERR_STATE"}
BC = {"closed": 0, "transmissive": 1, "inflow": 2}
REG_PREDICT, REG_CLOSE, FULL_SWEEP, FLUX_MATCH = 1, 2, 4, 8


class Hwfv1Error(RuntimeError):
    def __init__(self, status, what, msg=""):
        super().__init__("%s: %s%s" % (what, STATUS.get(status, status), (" (%s)" % msg) if msg else ""))
        self.status = status


class Problem(C.Structure):
    """Mirror of struct hwfv1_problem."""
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("lx", C.c_double), ("ly", C.c_double),
                ("eps", C.c_double), ("cfl", C.c_double), ("g", C.c_double),
                ("manning_n", C.c_double), ("tol_h", C.c_double), ("dt_max", C.c_double),
                ("L", C.c_int32), ("precision", C.c_int32), ("bc", C.c_int32 * 4),
                ("inflow_a0", C.c_int32), ("inflow_a1", C.c_int32), ("inflow_n", C.c_int32),
                ("flags", C.c_uint32),
                ("inflow_t", C.POINTER(C.c_double)), ("inflow_Q", C.POINTER(C.c_double))]


_H = C.c_void_p
_dp = C.c_void_p        # device pointers are passed as integers


def library_path():
    return _build.LIB


def lib():
    """Load libhwfv1.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise OSError("libhwfv1.so not found at %s" % path)
            L = C.CDLL(path)
            L.hwfv1_version.restype = C.c_int32
            L.hwfv1_init.argtypes = [C.POINTER(Problem), _dp, _dp, _dp, _dp, C.c_void_p, C.POINTER(_H)]
            for name in ("encode", "flag", "step", "decode"):
                getattr(L, "hwfv1_" + name).argtypes = [_H]
            L.hwfv1_traverse.argtypes = [_H, C.POINTER(C.c_int64)]
            L.hwfv1_advance.argtypes = [_H, C.c_double, C.c_int64]
            L.hwfv1_advance_uniform.argtypes = [_H, C.c_double, C.c_int64]
            L.hwfv1_get_fields.argtypes = [_H, _dp, _dp, _dp]
            L.hwfv1_set_fields.argtypes = [_H, _dp, _dp, _dp]
            L.hwfv1_get_leaves.argtypes = [_H, _dp, C.c_int64, C.POINTER(C.c_int64)]
            L.hwfv1_get_flags.argtypes = [_H, C.c_int32, _dp, C.c_int64]
            L.hwfv1_get_level.argtypes = [_H, C.c_int32, C.c_int32, _dp]
            L.hwfv1_get_time.argtypes = [_H, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                         C.POINTER(C.c_int64)]
            L.hwfv1_set_time.argtypes = [_H, C.c_double, C.c_double]
            L.hwfv1_get_stats.argtypes = [_H, C.POINTER(C.c_int64), C.POINTER(C.c_double)]
            L.hwfv1_get_counters.argtypes = [_H] + [C.POINTER(C.c_int64)] * 5
            L.hwfv1_profile_step.argtypes = [_H, C.POINTER(C.c_float), C.POINTER(C.c_char_p), C.c_int32,
                                             C.POINTER(C.c_int32)]
            L.hwfv1_profile_update.argtypes = [_H, C.c_int32, C.POINTER(C.c_float)]
            L.hwfv1_fp64_throughput.argtypes = [C.POINTER(C.c_double)]
            L.hwfv1_save.argtypes = [_H, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]
            L.hwfv1_load.argtypes = [_H, C.c_void_p, C.c_size_t]
            L.hwfv1_last_error.argtypes = [_H]
            L.hwfv1_last_error.restype = C.c_char_p
            L.hwfv1_traverse_noalloc.argtypes = [_dp, C.c_int32, _dp, C.c_int64, _dp, C.c_void_p]
            _pp = C.POINTER(C.c_void_p)
            L.hwfv1_batch_init.argtypes = [C.POINTER(Problem), C.c_int32, _pp, _pp, _pp, _pp, C.c_void_p,
                                           C.POINTER(C.c_void_p)]
            L.hwfv1_batch_advance.argtypes = [C.c_void_p, C.c_double, C.c_int64]
            L.hwfv1_batch_autotune.argtypes = [C.c_void_p, C.c_int64, C.POINTER(C.c_int32)]
            L.hwfv1_batch_member.argtypes = [C.c_void_p, C.c_int32, C.POINTER(_H)]
            L.hwfv1_batch_launches_per_step.argtypes = [C.c_void_p]
            L.hwfv1_batch_launches_per_step.restype = C.c_int64
            L.hwfv1_batch_last_error.argtypes = [C.c_void_p]
            L.hwfv1_batch_last_error.restype = C.c_char_p
            L.hwfv1_batch_destroy.argtypes = [C.c_void_p]
            L.hwfv1_batch_destroy.restype = None
            L.hwfv1_skipnet_num_params.restype = C.c_int32
            L.hwfv1_skipnet_create.argtypes = [C.c_uint32, C.POINTER(C.c_void_p)]
            L.hwfv1_skipnet_set_params.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.c_int64]
            L.hwfv1_skipnet_get_params.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.c_int64]
            L.hwfv1_skipnet_forward.argtypes = [C.c_void_p, _dp, C.c_int32, C.c_int32, C.c_int32, _dp]
            L.hwfv1_skipnet_gradients.argtypes = [C.c_void_p, _dp, _dp, C.c_int32, C.c_int32, C.c_int32,
                                                  C.POINTER(C.c_double), C.POINTER(C.c_float)]
            L.hwfv1_skipnet_train.argtypes = [C.c_void_p, _dp, _dp, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                              C.c_int32, C.c_float, C.c_uint32, C.POINTER(C.c_double)]
            L.hwfv1_skipnet_destroy.argtypes = [C.c_void_p]
            L.hwfv1_skipnet_destroy.restype = None
            L.hwfv1_set_skipnet.argtypes = [_H, C.c_void_p, C.c_int32, C.c_float, C.c_int32]
            L.hwfv1_set_skip_levels.argtypes = [_H, C.c_void_p, C.c_int32]
            L.hwfv1_get_skip_levels.argtypes = [_H, C.c_int32, C.c_void_p, C.c_int64]
            L.hwfv1_set_leaf_store.argtypes = [_H, C.c_int32]
            L.hwfv1_get_features.argtypes = [_H, _dp, C.c_int64]
            L.hwfv1_get_labels.argtypes = [_H, _dp, C.c_int64]
            L.hwfv1_destroy.argtypes = [_H]
            L.hwfv1_destroy.restype = None
            _lib = L
    return _lib


def exported_symbols():
    return ["hwfv1_init", "hwfv1_encode", "hwfv1_flag", "hwfv1_traverse", "hwfv1_step",
            "hwfv1_decode", "hwfv1_advance", "hwfv1_advance_uniform", "hwfv1_get_fields", "hwfv1_set_fields",
            "hwfv1_get_leaves", "hwfv1_get_flags", "hwfv1_get_level", "hwfv1_get_time",
            "hwfv1_set_time", "hwfv1_get_stats", "hwfv1_get_counters", "hwfv1_profile_step",
            "hwfv1_profile_update", "hwfv1_fp64_throughput", "hwfv1_save", "hwfv1_load",
            "hwfv1_last_error", "hwfv1_destroy", "hwfv1_version", "hwfv1_traverse_noalloc",
            "hwfv1_batch_init", "hwfv1_batch_advance", "hwfv1_batch_autotune", "hwfv1_batch_member",
            "hwfv1_batch_launches_per_step", "hwfv1_batch_last_error", "hwfv1_batch_destroy",
            "hwfv1_skipnet_num_params", "hwfv1_skipnet_create", "hwfv1_skipnet_set_params",
            "hwfv1_skipnet_get_params", "hwfv1_skipnet_forward", "hwfv1_skipnet_gradients",
            "hwfv1_skipnet_train", "hwfv1_skipnet_destroy", "hwfv1_set_skipnet", "hwfv1_set_skip_levels",
            "hwfv1_get_skip_levels", "hwfv1_set_leaf_store", "hwfv1_get_features", "hwfv1_get_labels"]


def _check(st, what, hd=None):
    if st != OK:
        msg = ""
        if hd is not None:
            m = lib().hwfv1_last_error(hd)
            msg = m.decode() if m else ""
        raise Hwfv1Error(st, what, msg)


def _ptr(t):
    """Device pointer of a torch CUDA tensor (float64/uint32, contiguous)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _ptr_io(t):
    """Pointer of a contiguous float64 tensor on the device or on the host
    (pinned or not): hwfv1_init and hwfv1_get_fields take either."""
    if t is None:
        return None
    if not t.is_contiguous() or not t.is_floating_point() or t.element_size() != 8:
        raise ValueError("expected a contiguous float64 tensor")
    return t.data_ptr()


def make_problem(p, precision=64):
    """hwfv1_problem from a problem dict (see synth.problem); keeps the
    hydrograph arrays alive on the returned object."""
    s = Problem()
    s.x0, s.y0, s.lx, s.ly = p["x0"], p["y0"], p["lx"], p["ly"]
    s.eps, s.cfl, s.g = p["eps"], p["cfl"], p["g"]
    s.manning_n, s.tol_h, s.dt_max = p["manning_n"], p["tol_h"], p["dt_max"]
    s.L = p["L"]
    s.precision = precision
    for k in range(4):
        s.bc[k] = BC[p["bc"][k]]
    inf = p.get("inflow")
    if inf:
        n = len(inf["t"])
        t = (C.c_double * n)(*inf["t"])
        q = (C.c_double * n)(*inf["Q"])
        s._keep = (t, q)
        s.inflow_t = C.cast(t, C.POINTER(C.c_double))
        s.inflow_Q = C.cast(q, C.POINTER(C.c_double))
        s.inflow_n = n
        s.inflow_a0, s.inflow_a1 = inf["a0"], inf["a1"]
    s.flags = ((REG_PREDICT if p.get("reg_predict", True) else 0) | (REG_CLOSE if p.get("reg_close", True) else 0)
               | (FULL_SWEEP if p.get("full_sweep", False) else 0)
               | (FLUX_MATCH if p.get("flux_match", False) else 0))
    return s


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def hwfv1_init(spec, z, h, qx, qy, stream=None):
    """spec: Problem; z, h, qx, qy: float64 tensors on the device or on the
    host (a host field is copied in by the library); stream: a
    torch.cuda.Stream or None (the library's own stream).  Returns a handle."""
    hd = _H()
    sp = stream.cuda_stream if stream is not None else None
    st = lib().hwfv1_init(C.byref(spec), _ptr_io(z), _ptr_io(h), _ptr_io(qx), _ptr_io(qy), sp, C.byref(hd))
    _check(st, "hwfv1_init")
    return hd


def hwfv1_encode(hd):
    _check(lib().hwfv1_encode(hd), "hwfv1_encode", hd)


def hwfv1_flag(hd):
    _check(lib().hwfv1_flag(hd), "hwfv1_flag", hd)


def hwfv1_traverse(hd, want_count=False):
    n = C.c_int64(0)
    _check(lib().hwfv1_traverse(hd, C.byref(n) if want_count else None), "hwfv1_traverse", hd)
    return n.value if want_count else None


def hwfv1_step(hd):
    _check(lib().hwfv1_step(hd), "hwfv1_step", hd)


def hwfv1_decode(hd):
    _check(lib().hwfv1_decode(hd), "hwfv1_decode", hd)


def hwfv1_advance(hd, t_end, max_steps):
    _check(lib().hwfv1_advance(hd, float(t_end), int(max_steps)), "hwfv1_advance", hd)


def hwfv1_get_fields(hd, h=None, qx=None, qy=None):
    """Outputs on the device or on the host (written when the call returns)."""
    _check(lib().hwfv1_get_fields(hd, _ptr_io(h), _ptr_io(qx), _ptr_io(qy)), "hwfv1_get_fields", hd)


def hwfv1_set_fields(hd, h, qx, qy):
    _check(lib().hwfv1_set_fields(hd, _ptr(h), _ptr(qx), _ptr(qy)), "hwfv1_set_fields", hd)


def hwfv1_get_leaves(hd, out=None):
    """Returns the leaf count; fills `out` (CUDA int32/uint32 tensor) if given."""
    n = C.c_int64(0)
    cap = out.numel() if out is not None else 0
    _check(lib().hwfv1_get_leaves(hd, _ptr(out), cap, C.byref(n)), "hwfv1_get_leaves", hd)
    return n.value


def hwfv1_get_flags(hd, which, out):
    _check(lib().hwfv1_get_flags(hd, int(which), _ptr(out), out.numel()), "hwfv1_get_flags", hd)


def hwfv1_get_level(hd, field, level, out):
    _check(lib().hwfv1_get_level(hd, int(field), int(level), _ptr(out)), "hwfv1_get_level", hd)


def hwfv1_get_time(hd):
    t, dt, s = C.c_double(), C.c_double(), C.c_int64()
    _check(lib().hwfv1_get_time(hd, C.byref(t), C.byref(dt), C.byref(s)), "hwfv1_get_time", hd)
    return t.value, dt.value, s.value


def hwfv1_set_time(hd, t, dt):
    _check(lib().hwfv1_set_time(hd, float(t), float(dt)), "hwfv1_set_time", hd)


def hwfv1_get_stats(hd):
    m = C.c_int64()
    sm = (C.c_double * 3)()
    _check(lib().hwfv1_get_stats(hd, C.byref(m), sm), "hwfv1_get_stats", hd)
    return m.value, list(sm)


def hwfv1_profile_step(hd, cap=64):
    """[(kernel name, ms)] of one step launched kernel by kernel."""
    ms = (C.c_float * cap)()
    names = (C.c_char_p * cap)()
    n = C.c_int32()
    _check(lib().hwfv1_profile_step(hd, ms, names, cap, C.byref(n)), "hwfv1_profile_step", hd)
    return [(names[i].decode(), float(ms[i])) for i in range(min(n.value, cap))]


def hwfv1_fp64_throughput():
    """Measured FP64 add throughput of the current device (TFLOP/s)."""
    v = C.c_double()
    _check(lib().hwfv1_fp64_throughput(C.byref(v)), "hwfv1_fp64_throughput")
    return v.value


def hwfv1_profile_update(hd, reps=20):
    """Mean time (ms) of the full update of the queued leaves, replayed reps
    times inside one plain step (which the call then completes)."""
    ms = C.c_float()
    _check(lib().hwfv1_profile_update(hd, int(reps), C.byref(ms)), "hwfv1_profile_update", hd)
    return ms.value


def hwfv1_advance_uniform(hd, t_end=float("inf"), max_steps=1):
    _check(lib().hwfv1_advance_uniform(hd, float(t_end), int(max_steps)), "hwfv1_advance_uniform", hd)


def hwfv1_get_counters(hd):
    """(steps, leaf_updates, active_updates, wet_updates, kernels_per_step)."""
    v = [C.c_int64() for _ in range(5)]
    _check(lib().hwfv1_get_counters(hd, *[C.byref(x) for x in v]), "hwfv1_get_counters", hd)
    return tuple(x.value for x in v)


def hwfv1_save(hd):
    used = C.c_size_t()
    _check(lib().hwfv1_save(hd, None, 0, C.byref(used)), "hwfv1_save", hd)
    buf = C.create_string_buffer(used.value)
    _check(lib().hwfv1_save(hd, buf, used.value, C.byref(used)), "hwfv1_save", hd)
    return bytes(buf.raw)


def hwfv1_load(hd, data):
    buf = C.create_string_buffer(data, len(data))
    _check(lib().hwfv1_load(hd, buf, len(data)), "hwfv1_load", hd)


def hwfv1_traverse_noalloc(sig_bits, L, leaves, num_leaves, stream=None):
    """Leaf list of a significance bit array with no device allocation:
    sig_bits (CUDA int32/uint32, get_flags layout), leaves (CUDA
    int32/uint32 output), num_leaves (CUDA int32/uint32, one element)."""
    sp = stream.cuda_stream if stream is not None else None
    st = lib().hwfv1_traverse_noalloc(_ptr(sig_bits), int(L), _ptr(leaves), leaves.numel(),
                                      _ptr(num_leaves), sp)
    _check(st, "hwfv1_traverse_noalloc")


def hwfv1_last_error(hd):
    m = lib().hwfv1_last_error(hd)
    return m.decode() if m else ""


def hwfv1_destroy(hd):
    lib().hwfv1_destroy(hd)


def bits_words(L):
    """Words of a significance bit array with levels 0..L-1."""
    if L <= 3:
        return L
    return 3 + ((1 << (2 * L)) - 64) // 96


def word_off(n):
    return bits_words(n)


# ---------------------------------------------------------------------------
# Batched ensembles
# ---------------------------------------------------------------------------

def _check_batch(st, what, bt=None):
    if st != OK:
        msg = ""
        if bt is not None:
            m = lib().hwfv1_batch_last_error(bt)
            msg = m.decode() if m else ""
        raise Hwfv1Error(st, what, msg)


def hwfv1_batch_init(specs, z, h, qx, qy, stream=None):
    """specs: list of Problem (same precision); z, h, qx, qy: lists of CUDA
    float64 tensors.  Returns a batch handle."""
    n = len(specs)
    arr = (Problem * n)(*specs)
    ptrs = [(C.c_void_p * n)(*[_ptr(t) for t in xs]) for xs in (z, h, qx, qy)]
    bt = C.c_void_p()
    sp = stream.cuda_stream if stream is not None else None
    st = lib().hwfv1_batch_init(arr, n, *[C.cast(p, C.POINTER(C.c_void_p)) for p in ptrs], sp, C.byref(bt))
    _check_batch(st, "hwfv1_batch_init")
    return bt


def hwfv1_batch_advance(bt, t_end, max_steps):
    _check_batch(lib().hwfv1_batch_advance(bt, float(t_end), int(max_steps)), "hwfv1_batch_advance", bt)


def hwfv1_batch_autotune(bt, trial_steps):
    ch = (C.c_int32 * 2)()
    _check_batch(lib().hwfv1_batch_autotune(bt, int(trial_steps), ch), "hwfv1_batch_autotune", bt)
    return ch[0], ch[1]


def hwfv1_batch_member(bt, d):
    hd = _H()
    _check_batch(lib().hwfv1_batch_member(bt, int(d), C.byref(hd)), "hwfv1_batch_member", bt)
    return hd


def hwfv1_batch_launches_per_step(bt):
    return int(lib().hwfv1_batch_launches_per_step(bt))


def hwfv1_batch_last_error(bt):
    m = lib().hwfv1_batch_last_error(bt)
    return m.decode() if m else ""


def hwfv1_batch_destroy(bt):
    lib().hwfv1_batch_destroy(bt)


# ---------------------------------------------------------------------------
# Learned subtree skip (subtree CNN)
# ---------------------------------------------------------------------------

def hwfv1_skipnet_num_params():
    return int(lib().hwfv1_skipnet_num_params())


def hwfv1_skipnet_create(seed=0):
    net = C.c_void_p()
    _check(lib().hwfv1_skipnet_create(int(seed), C.byref(net)), "hwfv1_skipnet_create")
    return net


def hwfv1_skipnet_set_params(net, params):
    import numpy as np
    a = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib().hwfv1_skipnet_set_params(net, a.ctypes.data_as(C.POINTER(C.c_float)), a.size),
           "hwfv1_skipnet_set_params")


def hwfv1_skipnet_get_params(net):
    import numpy as np
    a = np.empty(hwfv1_skipnet_num_params(), dtype=np.float32)
    _check(lib().hwfv1_skipnet_get_params(net, a.ctypes.data_as(C.POINTER(C.c_float)), a.size),
           "hwfv1_skipnet_get_params")
    return a


def hwfv1_skipnet_forward(net, x, nimg, H, W, logits):
    """x: CUDA int16/bfloat16 tensor [nimg*H*W*4]; logits: CUDA float32 [nimg*H*W*16]."""
    _check(lib().hwfv1_skipnet_forward(net, _ptr(x), int(nimg), int(H), int(W), _ptr(logits)),
           "hwfv1_skipnet_forward")


def hwfv1_skipnet_gradients(net, x, labels, nimg, H, W):
    import numpy as np
    g = np.empty(hwfv1_skipnet_num_params(), dtype=np.float32)
    loss = C.c_double()
    _check(lib().hwfv1_skipnet_gradients(net, _ptr(x), _ptr(labels), int(nimg), int(H), int(W), C.byref(loss),
                                         g.ctypes.data_as(C.POINTER(C.c_float))), "hwfv1_skipnet_gradients")
    return loss.value, g


def hwfv1_skipnet_train(net, x, labels, nimg, H, W, batch, epochs, lr, seed=0):
    loss = C.c_double()
    _check(lib().hwfv1_skipnet_train(net, _ptr(x), _ptr(labels), int(nimg), int(H), int(W), int(batch),
                                     int(epochs), float(lr), int(seed), C.byref(loss)), "hwfv1_skipnet_train")
    return loss.value


def hwfv1_skipnet_destroy(net):
    lib().hwfv1_skipnet_destroy(net)


def hwfv1_set_skipnet(hd, net, audit_K=10, margin=0.02, predict_every=1):
    _check(lib().hwfv1_set_skipnet(hd, net, int(audit_K), float(margin), int(predict_every)),
           "hwfv1_set_skipnet", hd)


def hwfv1_set_skip_levels(hd, levels, audit_K=10):
    """levels: host uint8 array [2^(L-4), 2^(L-4)] (row-major, j major) or
    None to stop."""
    if levels is None:
        _check(lib().hwfv1_set_skip_levels(hd, None, int(audit_K)), "hwfv1_set_skip_levels", hd)
        return
    lv = np.ascontiguousarray(levels, dtype=np.uint8)
    _check(lib().hwfv1_set_skip_levels(hd, lv.ctypes.data, int(audit_K)), "hwfv1_set_skip_levels", hd)


def hwfv1_get_skip_levels(hd, which, L):
    """which = 0: predicted levels in use, 1: storage levels; host uint8
    array [2^(L-4), 2^(L-4)]."""
    S = 1 << (L - 4)
    out = np.empty((S, S), dtype=np.uint8)
    _check(lib().hwfv1_get_skip_levels(hd, int(which), out.ctypes.data, out.size), "hwfv1_get_skip_levels", hd)
    return out


def hwfv1_set_leaf_store(hd, on=True):
    _check(lib().hwfv1_set_leaf_store(hd, 1 if on else 0), "hwfv1_set_leaf_store", hd)


def hwfv1_get_features(hd, out):
    _check(lib().hwfv1_get_features(hd, _ptr(out), out.numel()), "hwfv1_get_features", hd)


def hwfv1_get_labels(hd, out):
    _check(lib().hwfv1_get_labels(hd, _ptr(out), out.numel()), "hwfv1_get_labels", hd)

