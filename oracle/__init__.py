"""Loader for the HWFV1 CPU oracle (oracle/hwfv1_oracle.c).

TEST INFRASTRUCTURE ONLY: the oracle is the plain, slow statement of the
method that the CUDA library is checked against.  Only tests/,
``__graft_entry__.smoke()`` and bench.py's cpu_baseline / ``--impl reference``
legs may import this package; the library in paper_2206_05761_gb300/ never
does.  It is compiled with gcc on first use (or by ``build()``) with
``-ffp-contract=off`` so that its operation order is exactly the one written
in the C source.

All arrays here are numpy, row-major over a level (index j*2^n + i).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HWFV1_ORACLE_SRC / HWFV1_ORACLE_BUILD_DIR point the loader at another copy
# of the C source and build folder: the mutation test plants mistakes in
# such a copy to show that the pins catch them.
_SRC = os.environ.get("HWFV1_ORACLE_SRC") or os.path.join(_HERE, "hwfv1_oracle.c")
_OUT_DIR = os.environ.get("HWFV1_ORACLE_BUILD_DIR") or os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc_hwfv1.so")
_lock = threading.Lock()
_lib = None

BC = {"closed": 0, "transmissive": 1, "inflow": 2}


def build(force=False):
    """Compile the oracle shared library with gcc (no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Problem(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("lx", C.c_double), ("ly", C.c_double),
                ("L", C.c_int), ("reg_predict", C.c_int), ("reg_close", C.c_int),
                ("inflow_a0", C.c_int), ("inflow_a1", C.c_int), ("inflow_n", C.c_int),
                ("bc", C.c_int * 4),
                ("eps", C.c_double), ("cfl", C.c_double), ("g", C.c_double),
                ("manning_n", C.c_double), ("tol_h", C.c_double), ("dt_max", C.c_double),
                ("inflow_t", C.POINTER(C.c_double)), ("inflow_Q", C.POINTER(C.c_double)),
                ("flux_match", C.c_int)]


class StepOut(C.Structure):
    _fields_ = [("T", C.POINTER(C.c_uint8)), ("S", C.POINTER(C.c_uint8)),
                ("leaves", C.POINTER(C.c_uint32)), ("leaves_cap", C.c_int64),
                ("hier_out", C.POINTER(C.c_double)),
                ("num_leaves", C.c_int64), ("dt_next", C.c_double)]


_dp = C.POINTER(C.c_double)
_u8p = C.POINTER(C.c_uint8)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            L.orc_version.restype = C.c_int
            L.orc_morton.restype = C.c_uint64
            L.orc_morton.argtypes = [C.c_uint32, C.c_uint32]
            L.orc_demorton.argtypes = [C.c_uint64, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.orc_zindex.restype = C.c_int64
            L.orc_zindex.argtypes = [C.c_int, C.c_uint64]
            L.orc_encode_parent.argtypes = [_dp, _dp]
            L.orc_decode_parent.argtypes = [_dp, _dp]
            L.orc_encode.argtypes = [C.c_int, _dp, _dp, _dp]
            L.orc_decode_all.argtypes = [C.c_int, _dp, _dp, _dp]
            L.orc_smax.restype = C.c_double
            L.orc_smax.argtypes = [C.c_int, _dp]
            L.orc_threshold_flags.argtypes = [C.c_int, C.c_double, C.POINTER(_dp), _dp, _u8p]
            L.orc_regularise.argtypes = [C.c_int, C.c_int, C.c_int, _u8p, _u8p]
            L.orc_leaves_dft.restype = C.c_int64
            L.orc_leaves_dft.argtypes = [C.c_int, _u8p, C.POINTER(C.c_uint32), C.c_int64]
            L.orc_leaves_ptt.argtypes = [C.c_int, _u8p, C.POINTER(C.c_int64)]
            L.orc_hll_x.argtypes = [C.c_double, C.c_double, _dp, _dp, _dp]
            L.orc_star_estimate.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, _dp, _dp]
            L.orc_cfl_rmin.restype = C.c_double
            L.orc_cfl_rmin.argtypes = [C.POINTER(Problem), _dp, _dp, _dp]
            L.orc_next_dt.restype = C.c_double
            L.orc_next_dt.argtypes = [C.POINTER(Problem), _dp, _dp, _dp]
            L.orc_hwfv1_step.restype = C.c_int
            L.orc_hwfv1_step.argtypes = [C.POINTER(Problem), _dp, _dp, _dp, _dp, C.c_double,
                                         C.c_double, C.POINTER(StepOut)]
            L.orc_fv1_step.restype = C.c_int
            L.orc_fv1_step.argtypes = [C.POINTER(Problem), _dp, _dp, _dp, _dp, C.c_double,
                                       C.c_double]
            L.orc_skip_step.restype = C.c_int
            L.orc_skip_step.argtypes = [C.POINTER(Problem), C.POINTER(_dp), _u8p, _u8p, _dp, C.c_double,
                                        C.c_double, C.POINTER(StepOut)]
            L.orc_skip_audit_step.restype = C.c_int
            L.orc_skip_audit_step.argtypes = [C.POINTER(Problem), C.POINTER(_dp), _u8p, _dp, C.c_double,
                                              C.c_double, C.POINTER(StepOut)]
            L.orc_skip_prolong_all.restype = C.c_int
            L.orc_skip_prolong_all.argtypes = [C.POINTER(Problem), C.POINTER(_dp), _u8p, _dp]
            L.orc_run.restype = C.c_int
            L.orc_run.argtypes = [C.POINTER(Problem), _dp, _dp, _dp, _dp, _dp, _dp, C.c_double,
                                  C.c_int64, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    return _lib


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def level_start(n):
    return ((1 << (2 * n)) - 1) // 3


def make_problem(p):
    """ctypes Problem from a synth.problem() dict (keeps the hydrograph
    arrays alive on the returned object)."""
    s = Problem()
    s.x0, s.y0, s.lx, s.ly = p["x0"], p["y0"], p["lx"], p["ly"]
    s.L = p["L"]
    s.reg_predict = int(p["reg_predict"])
    s.reg_close = int(p["reg_close"])
    s.flux_match = int(p.get("flux_match", False))
    for k in range(4):
        s.bc[k] = BC[p["bc"][k]]
    s.eps, s.cfl, s.g = p["eps"], p["cfl"], p["g"]
    s.manning_n, s.tol_h, s.dt_max = p["manning_n"], p["tol_h"], p["dt_max"]
    inf = p.get("inflow")
    if inf:
        t = np.ascontiguousarray(inf["t"], dtype=np.float64)
        q = np.ascontiguousarray(inf["Q"], dtype=np.float64)
        s._keep = (t, q)
        s.inflow_t, s.inflow_Q = _d(t), _d(q)
        s.inflow_n = len(t)
        s.inflow_a0, s.inflow_a1 = inf["a0"], inf["a1"]
    else:
        s.inflow_n = 0
    return s


# ---------------------------------------------------------------------------
# Thin wrappers
# ---------------------------------------------------------------------------

def morton(i, j):
    return int(lib().orc_morton(int(i), int(j)))


def demorton(code):
    a, b = C.c_uint32(), C.c_uint32()
    lib().orc_demorton(int(code), C.byref(a), C.byref(b))
    return a.value, b.value


def zindex(n, code):
    return int(lib().orc_zindex(int(n), int(code)))



def encode_parent(c):
    c = np.ascontiguousarray(c, dtype=np.float64)
    o = np.empty(4)
    lib().orc_encode_parent(_d(c), _d(o))
    return o


def decode_parent(p):
    p = np.ascontiguousarray(p, dtype=np.float64)
    o = np.empty(4)
    lib().orc_decode_parent(_d(p), _d(o))
    return o


def encode(L, fine):
    """Return (hier, det): hier has all levels 0..L (length (4^(L+1)-1)/3),
    det the three details of every parent (shape (P, 3))."""
    fine = np.ascontiguousarray(fine, dtype=np.float64).reshape(-1)
    hier = np.empty(level_start(L + 1))
    det = np.empty(3 * max(level_start(L), 1))
    lib().orc_encode(L, _d(fine), _d(hier), _d(det))
    return hier, det[: 3 * level_start(L)].reshape(-1, 3)


def decode_all(L, hier, det):
    det = np.ascontiguousarray(det, dtype=np.float64).reshape(-1)
    out = np.empty(1 << (2 * L))
    c0 = np.ascontiguousarray(hier[:1], dtype=np.float64)
    lib().orc_decode_all(L, _d(c0), _d(det), _d(out))
    return out.reshape(1 << L, 1 << L)


def level(hier, n):
    s = 1 << n
    return hier[level_start(n): level_start(n) + s * s].reshape(s, s)


def smax(L, fine):
    return float(lib().orc_smax(L, _d(np.ascontiguousarray(fine, dtype=np.float64).reshape(-1))))


def threshold_flags(L, eps, dets, smaxes):
    """dets: four detail arrays (P, 3) for h, qx, qy, z; smaxes: four s_max."""
    dets = [np.ascontiguousarray(d, dtype=np.float64).reshape(-1) for d in dets]
    arr = (_dp * 4)(*[_d(d) for d in dets])
    sm = np.ascontiguousarray(smaxes, dtype=np.float64)
    T = np.zeros(max(level_start(L), 1), dtype=np.uint8)
    lib().orc_threshold_flags(L, float(eps), arr, _d(sm), T.ctypes.data_as(_u8p))
    return T[: level_start(L)]


def regularise(L, T, predict=True, close=True):
    T = np.ascontiguousarray(T, dtype=np.uint8)
    S = np.zeros(max(level_start(L), 1), dtype=np.uint8)
    Tb = T if T.size else np.zeros(1, np.uint8)
    lib().orc_regularise(L, int(predict), int(close), Tb.ctypes.data_as(_u8p), S.ctypes.data_as(_u8p))
    return S[: level_start(L)]


def leaves_dft(L, S):
    S = np.ascontiguousarray(S, dtype=np.uint8)
    Sb = S if S.size else np.zeros(1, np.uint8)
    n = lib().orc_leaves_dft(L, Sb.ctypes.data_as(_u8p), None, 0)
    out = np.empty(n, dtype=np.uint32)
    lib().orc_leaves_dft(L, Sb.ctypes.data_as(_u8p), out.ctypes.data_as(C.POINTER(C.c_uint32)), n)
    return out


def leaves_ptt(L, S):
    S = np.ascontiguousarray(S, dtype=np.uint8)
    Sb = S if S.size else np.zeros(1, np.uint8)
    out = np.empty(1 << (2 * L), dtype=np.int64)
    lib().orc_leaves_ptt(L, Sb.ctypes.data_as(_u8p), out.ctypes.data_as(C.POINTER(C.c_int64)))
    return out


def hll_x(g, tol_h, left, right):
    a = np.ascontiguousarray(left, dtype=np.float64)
    b = np.ascontiguousarray(right, dtype=np.float64)
    F = np.empty(3)
    lib().orc_hll_x(float(g), float(tol_h), _d(a), _d(b), _d(F))
    return F


def star_estimate(unL, aL, unR, aR):
    """Two-rarefaction estimate (us, as) of the star region of a wet face
    (hydrostatic reconstruction already applied: a = sqrt(g h*))."""
    us, as_ = C.c_double(), C.c_double()
    lib().orc_star_estimate(float(unL), float(aL), float(unR), float(aR), C.byref(us), C.byref(as_))
    return us.value, as_.value


class State:
    """Finest-grid state (h, qx, qy, z row-major) plus time and next dt."""

    def __init__(self, p, fields, t=0.0, dt=None):
        self.p = p
        self.cp = make_problem(p)
        self.h = np.ascontiguousarray(fields["h"], dtype=np.float64).copy()
        self.qx = np.ascontiguousarray(fields["qx"], dtype=np.float64).copy()
        self.qy = np.ascontiguousarray(fields["qy"], dtype=np.float64).copy()
        self.z = np.ascontiguousarray(fields["z"], dtype=np.float64).copy()
        self.t = float(t)
        self.dt = self.next_dt() if dt is None else float(dt)
        self.steps = 0
        self.leaf_updates = 0

    def next_dt(self):
        return float(lib().orc_next_dt(C.byref(self.cp), _d(self.h), _d(self.qx), _d(self.qy)))


    def step(self, dt=None, want=()):
        """One HWFV1 step of size dt (default: the current dt).  `want` may
        hold "T", "S", "leaves", "hier" to return those intermediates."""
        L = self.p["L"]
        P, N = level_start(L), 1 << (2 * L)
        dt = self.dt if dt is None else float(dt)
        o = StepOut()
        res = {}
        if "T" in want:
            res["T"] = np.zeros(max(P, 1), np.uint8)
            o.T = res["T"].ctypes.data_as(_u8p)
        if "S" in want:
            res["S"] = np.zeros(max(P, 1), np.uint8)
            o.S = res["S"].ctypes.data_as(_u8p)
        if "leaves" in want:
            res["leaves"] = np.zeros(N, np.uint32)
            o.leaves = res["leaves"].ctypes.data_as(C.POINTER(C.c_uint32))
            o.leaves_cap = N
        if "hier" in want:
            res["hier"] = np.zeros(3 * (N + P))
            o.hier_out = _d(res["hier"])
        rc = lib().orc_hwfv1_step(C.byref(self.cp), _d(self.h), _d(self.qx), _d(self.qy),
                                  _d(self.z), self.t, dt, C.byref(o))
        if rc:
            raise RuntimeError("oracle step failed (%d)" % rc)
        if "T" in res:
            res["T"] = res["T"][:P]
        if "S" in res:
            res["S"] = res["S"][:P]
        if "leaves" in res:
            res["leaves"] = res["leaves"][: o.num_leaves]
        if "hier" in res:
            res["hier"] = res["hier"].reshape(3, N + P)
        self.t += dt
        self.dt = o.dt_next
        self.steps += 1
        self.leaf_updates += o.num_leaves
        res["num_leaves"] = int(o.num_leaves)
        return res

    def fv1_step(self, dt=None):
        dt = self.dt if dt is None else float(dt)
        lib().orc_fv1_step(C.byref(self.cp), _d(self.h), _d(self.qx), _d(self.qy), _d(self.z),
                           self.t, dt)
        self.t += dt
        self.dt = self.next_dt()
        self.steps += 1
        self.leaf_updates += 1 << (2 * self.p["L"])

    def run(self, t_end=np.inf, max_steps=1 << 62, uniform=False):
        t, dt = C.c_double(self.t), C.c_double(self.dt)
        steps, lu = C.c_int64(0), C.c_int64(0)
        rc = lib().orc_run(C.byref(self.cp), _d(self.h), _d(self.qx), _d(self.qy), _d(self.z),
                           C.byref(t), C.byref(dt), float(t_end), int(max_steps), int(uniform),
                           C.byref(steps), C.byref(lu))
        if rc:
            raise MemoryError("oracle run failed")
        self.t, self.dt = t.value, dt.value
        self.steps += steps.value
        self.leaf_updates += lu.value
        return steps.value


class SkipState:
    """State of the learned subtree skip (reading R-skip in the C source):
    full hierarchies of h, qx, qy with each level-(L-4) subtree's state at
    its storage level m (row-major [j, i] over level L-4), the bed, time and
    next dt.  `skip_step(levels)` takes the predicted level of every subtree
    (an integer array [j, i] over level L-4, values in [L-4, L]);
    `plain_step()` is the exact audit step; `fields()` the finest fields."""

    def __init__(self, p, fields, t=0.0, dt=None):
        self.p = p
        self.cp = make_problem(p)
        L = p["L"]
        self.L, self.Ls = L, L - 4
        H = level_start(L + 1)
        self.hier = np.zeros((3, H))
        for q, k in enumerate(("h", "qx", "qy")):
            self.hier[q, level_start(L):] = np.asarray(fields[k], dtype=np.float64).reshape(-1)
        self.z = np.ascontiguousarray(fields["z"], dtype=np.float64).reshape(-1).copy()
        self.m = np.full(1 << (2 * self.Ls), L, dtype=np.uint8)
        self.t = float(t)
        fin = self.hier[:, level_start(L):]
        self.dt = (float(lib().orc_next_dt(C.byref(self.cp), _d(np.ascontiguousarray(fin[0])),
                                           _d(np.ascontiguousarray(fin[1])), _d(np.ascontiguousarray(fin[2]))))
                   if dt is None else float(dt))
        self.steps = 0
        self.leaf_updates = 0

    def _rows(self, hier=None):
        h = self.hier if hier is None else hier
        return (_dp * 3)(*[h[q].ctypes.data_as(_dp) for q in range(3)])

    def _out(self, want, res):
        L = self.L
        P, N = level_start(L), 1 << (2 * L)
        o = StepOut()
        if "T" in want:
            res["T"] = np.zeros(max(P, 1), np.uint8)
            o.T = res["T"].ctypes.data_as(_u8p)
        if "S" in want:
            res["S"] = np.zeros(max(P, 1), np.uint8)
            o.S = res["S"].ctypes.data_as(_u8p)
        res["leaves"] = np.zeros(N, np.uint32)
        o.leaves = res["leaves"].ctypes.data_as(C.POINTER(C.c_uint32))
        o.leaves_cap = N
        return o

    def _finish(self, o, res, dt):
        P = level_start(self.L)
        for k in ("T", "S"):
            if k in res:
                res[k] = res[k][:P]
        res["leaves"] = res["leaves"][: o.num_leaves]
        res["num_leaves"] = int(o.num_leaves)
        self.t += dt
        self.dt = o.dt_next
        self.steps += 1
        self.leaf_updates += o.num_leaves
        return res

    def skip_step(self, levels, dt=None, want=()):
        levels = np.ascontiguousarray(levels, dtype=np.uint8).reshape(-1)
        assert levels.size == self.m.size
        dt = self.dt if dt is None else float(dt)
        res = {}
        o = self._out(want, res)
        rc = lib().orc_skip_step(C.byref(self.cp), self._rows(), self.m.ctypes.data_as(_u8p),
                                 levels.ctypes.data_as(_u8p), _d(self.z), self.t, dt, C.byref(o))
        if rc:
            raise RuntimeError("oracle skip step failed (%d)" % rc)
        return self._finish(o, res, dt)

    def to_finest(self):
        """Bring every subtree to level L in place (before a plain step)."""
        rc = lib().orc_skip_prolong_all(C.byref(self.cp), self._rows(), self.m.ctypes.data_as(_u8p), _d(self.z))
        if rc:
            raise RuntimeError("oracle prolongation failed (%d)" % rc)

    def plain_step(self, dt=None, want=()):
        """The exact audit step: s_max over the stored state, every subtree
        brought to level L, then the plain step."""
        dt = self.dt if dt is None else float(dt)
        res = {}
        o = self._out(want, res)
        rc = lib().orc_skip_audit_step(C.byref(self.cp), self._rows(), self.m.ctypes.data_as(_u8p),
                                       _d(self.z), self.t, dt, C.byref(o))
        if rc:
            raise RuntimeError("oracle audit step failed (%d)" % rc)
        return self._finish(o, res, dt)

    def fields(self):
        """Finest h, qx, qy ([j, i]) of the state, formed on a copy."""
        L = self.L
        hier = self.hier.copy()
        m = self.m.copy()
        rc = lib().orc_skip_prolong_all(C.byref(self.cp), self._rows(hier), m.ctypes.data_as(_u8p), _d(self.z))
        if rc:
            raise RuntimeError("oracle prolongation failed (%d)" % rc)
        n = 1 << L
        return {k: hier[q, level_start(L):].reshape(n, n).copy() for q, k in enumerate(("h", "qx", "qy"))}

    def stored(self):
        """The stored state: per subtree its level and its level-m cells
        (a list of (level, h, qx, qy) blocks, row-major over level L-4)."""
        out = []
        Ls = self.Ls
        for sj in range(1 << Ls):
            for si in range(1 << Ls):
                ms = int(self.m[sj * (1 << Ls) + si])
                w = 1 << (ms - Ls)
                lv = [self.hier[q, level_start(ms): level_start(ms) + (1 << (2 * ms))].reshape(1 << ms, 1 << ms)
                      [sj * w:(sj + 1) * w, si * w:(si + 1) * w] for q in range(3)]
                out.append((ms, *lv))
        return out
