"""Convenience wrapper over the C ABI for tests and benchmarks: owns the
torch CUDA tensors handed to the library and converts results to numpy.
Every computation happens in libhwfv1.so."""
from __future__ import annotations

import numpy as np
import torch

from . import hwfv1 as H


class Simulation:
    def __init__(self, p, fields, precision=64, stream=None, device="cuda"):
        if not torch.cuda.is_available():
            raise RuntimeError("HWFV1 needs a CUDA device; there is no CPU fallback")
        self.p = p
        self.L = p["L"]
        self.N = 1 << (2 * self.L)
        self.dev = torch.device(device)
        self.stream = stream
        self.spec = H.make_problem(p, precision)
        dt = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1),
                                       device=self.dev)
        z, h, qx, qy = (dt(fields[k]) for k in ("z", "h", "qx", "qy"))
        self.hd = H.hwfv1_init(self.spec, z, h, qx, qy, stream)
        self._bufs = [torch.empty(self.N, dtype=torch.float64, device=self.dev) for _ in range(3)]

    def _wait(self):
        """Wait for the library's stream before torch touches a tensor the
        library wrote (torch copies on its own current stream)."""
        if self.stream is not None:
            self.stream.synchronize()
        else:
            torch.cuda.synchronize()

    # -- the five phases of a step and the loop ---------------------------
    def encode(self):
        H.hwfv1_encode(self.hd)

    def flag(self):
        H.hwfv1_flag(self.hd)

    def traverse(self, want_count=False):
        return H.hwfv1_traverse(self.hd, want_count)

    def fv1(self):
        H.hwfv1_step(self.hd)

    def decode(self):
        H.hwfv1_decode(self.hd)

    def step(self):
        self.encode()
        self.flag()
        self.traverse()
        self.fv1()
        self.decode()

    def advance(self, t_end=float("inf"), max_steps=1):
        H.hwfv1_advance(self.hd, t_end, max_steps)

    def advance_uniform(self, t_end=float("inf"), max_steps=1):
        """Uniform FV1 on the finest grid (the GPU-FV1 comparison solver)."""
        H.hwfv1_advance_uniform(self.hd, t_end, max_steps)

    # -- results ------------------------------------------------------------
    def fields(self):
        h, qx, qy = self._bufs
        H.hwfv1_get_fields(self.hd, h, qx, qy)
        self._wait()
        s = 1 << self.L
        return {k: v.cpu().numpy().reshape(s, s).copy() for k, v in zip(("h", "qx", "qy"), (h, qx, qy))}

    def set_fields(self, f):
        t = [torch.as_tensor(np.ascontiguousarray(f[k], dtype=np.float64).reshape(-1), device=self.dev)
             for k in ("h", "qx", "qy")]
        H.hwfv1_set_fields(self.hd, *t)
        self._wait()                      # before t is released

    def leaves(self):
        n = H.hwfv1_get_leaves(self.hd)
        out = torch.empty(max(n, 1), dtype=torch.int32, device=self.dev)
        H.hwfv1_get_leaves(self.hd, out)
        self._wait()
        return out[:n].cpu().numpy().view(np.uint32).copy()

    def flags(self, which):
        w = H.bits_words(self.L)
        out = torch.zeros(max(w, 1), dtype=torch.int32, device=self.dev)
        H.hwfv1_get_flags(self.hd, which, out)
        self._wait()
        return out[:w].cpu().numpy().view(np.uint32).copy()

    def level(self, field, n):
        out = torch.empty(1 << (2 * n), dtype=torch.float64, device=self.dev)
        H.hwfv1_get_level(self.hd, field, n, out)
        self._wait()
        return out.cpu().numpy()

    def time(self):
        return H.hwfv1_get_time(self.hd)

    def set_time(self, t, dt):
        H.hwfv1_set_time(self.hd, t, dt)

    def stats(self):
        return H.hwfv1_get_stats(self.hd)

    def counters(self):
        """(steps, leaf_updates, active_updates, wet_updates, kernels_per_step)."""
        return H.hwfv1_get_counters(self.hd)

    def save(self):
        return H.hwfv1_save(self.hd)

    def load(self, blob):
        H.hwfv1_load(self.hd, blob)

    def features(self):
        """CNN input of the current state (call after encode): float32
        array [S, S, 4] of the bf16 values."""
        S = 1 << (self.L - 4)
        out = torch.empty(S * S * 4, dtype=torch.bfloat16, device=self.dev)
        H.hwfv1_get_features(self.hd, out)
        self._wait()
        return out.float().cpu().numpy().reshape(S, S, 4)

    def features_dev(self, out):
        H.hwfv1_get_features(self.hd, out)

    def labels(self):
        S = 1 << (self.L - 4)
        out = torch.empty(S * S, dtype=torch.uint8, device=self.dev)
        H.hwfv1_get_labels(self.hd, out)
        self._wait()
        return out.cpu().numpy().reshape(S, S)

    def labels_dev(self, out):
        H.hwfv1_get_labels(self.hd, out)

    def set_skipnet(self, net, audit_K=10, margin=0.02, predict_every=1):
        H.hwfv1_set_skipnet(self.hd, net, audit_K, margin, predict_every)

    def set_skip_levels(self, levels, audit_K=10):
        """The learned subtree skip with the given levels ([j, i] over level
        L-4; None stops it)."""
        H.hwfv1_set_skip_levels(self.hd, levels, audit_K)

    def set_leaf_store(self, on=True):
        """The exact leaf-value store (flat-bed subtrees stored at their
        deepest leaf level; results identical to the plain step)."""
        H.hwfv1_set_leaf_store(self.hd, on)

    def skip_levels(self, which=1):
        """Storage levels (which=1) or predicted levels in use (which=0)."""
        return H.hwfv1_get_skip_levels(self.hd, which, self.L)

    def close(self):
        if self.hd is not None:
            H.hwfv1_destroy(self.hd)
            self.hd = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unpack_bits(words, L):
    """Significance bits (get_flags layout) -> per-level uint8 arrays in
    Morton order."""
    out = []
    for n in range(L):
        w0 = H.word_off(n)
        cnt = 1 << (2 * n)
        nw = max(1, cnt // 32)
        bits = np.unpackbits(words[w0:w0 + nw].astype("<u4").view(np.uint8), bitorder="little")
        out.append(bits[:cnt].astype(np.uint8))
    return out


class Ensemble:
    """Many independent domains advanced together (hwfv1_batch_*)."""

    def __init__(self, cases, precision=64, stream=None, device="cuda"):
        if not torch.cuda.is_available():
            raise RuntimeError("HWFV1 needs a CUDA device; there is no CPU fallback")
        self.dev = torch.device(device)
        self.specs = [H.make_problem(p, precision) for p, _ in cases]
        self.L = [p["L"] for p, _ in cases]
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64).reshape(-1), device=self.dev)
        self._inputs = {k: [t(f[k]) for _, f in cases] for k in ("z", "h", "qx", "qy")}
        self.stream = stream
        self.bt = H.hwfv1_batch_init(self.specs, self._inputs["z"], self._inputs["h"], self._inputs["qx"],
                                     self._inputs["qy"], stream)
        self._wait()
        self._inputs = None

    def _wait(self):
        """Wait for the library's stream before torch touches a tensor the
        library read or wrote."""
        if self.stream is not None:
            self.stream.synchronize()
        else:
            torch.cuda.synchronize()

    def advance(self, t_end=float("inf"), max_steps=1):
        H.hwfv1_batch_advance(self.bt, t_end, max_steps)

    def autotune(self, trial_steps=3):
        return H.hwfv1_batch_autotune(self.bt, trial_steps)

    def member_fields(self, d):
        hd = H.hwfv1_batch_member(self.bt, d)
        n = 1 << (2 * self.L[d])
        bufs = [torch.empty(n, dtype=torch.float64, device=self.dev) for _ in range(3)]
        H.hwfv1_get_fields(hd, *bufs)
        self._wait()
        s = 1 << self.L[d]
        return {k: v.cpu().numpy().reshape(s, s) for k, v in zip(("h", "qx", "qy"), bufs)}

    def member_leaves(self, d):
        hd = H.hwfv1_batch_member(self.bt, d)
        n = H.hwfv1_get_leaves(hd)
        out = torch.empty(max(n, 1), dtype=torch.int32, device=self.dev)
        H.hwfv1_get_leaves(hd, out)
        self._wait()
        return out[:n].cpu().numpy().view(np.uint32).copy()

    def member_time(self, d):
        return H.hwfv1_get_time(H.hwfv1_batch_member(self.bt, d))

    def member_stats(self, d):
        return H.hwfv1_get_stats(H.hwfv1_batch_member(self.bt, d))

    def launches_per_step(self):
        return H.hwfv1_batch_launches_per_step(self.bt)

    def close(self):
        if self.bt is not None:
            H.hwfv1_batch_destroy(self.bt)
            self.bt = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
