"""Thin Python binding of the C ABI in include/nbgpu.h.

Argument marshalling only: every step of the regular-force path runs in the CUDA
kernels of libnbgpu.so.  PyTorch supplies device memory and the stream.  There is
no CPU fallback: if the library is missing or CUDA is unavailable, calls raise.

Names follow the C ABI (nb_init -> Context, nb_set_particles -> set_particles,
nb_predict -> predict, nb_regular_force -> regular_force, nb_regular_force_backward
-> regular_force_backward).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

NB_OK, NB_ERR_ARG, NB_ERR_STATE, NB_ERR_OOM, NB_ERR_CUDA, NB_ERR_NB_OVERFLOW, NB_ERR_TIMEOUT, NB_ERR_DEVICE = range(8)
STATUS_NAMES = {0: "NB_OK", 1: "NB_ERR_ARG", 2: "NB_ERR_STATE", 3: "NB_ERR_OOM", 4: "NB_ERR_CUDA",
                5: "NB_ERR_NB_OVERFLOW", 6: "NB_ERR_TIMEOUT", 7: "NB_ERR_DEVICE"}
NB_FP64, NB_MIXED = 0, 1
PRECISIONS = {"fp64": NB_FP64, "mixed": NB_MIXED}

# every symbol include/nbgpu.h declares
EXPORTS = ("nb_version", "nb_init", "nb_free", "nb_set_stream", "nb_set_particles", "nb_predict",
           "nb_set_predicted", "nb_get_predicted", "nb_get_records", "nb_regular_force", "nb_regular_force_backward",
           "nb_sync", "nb_last_error", "nb_plan", "nb_plan_for", "nb_set_plan_override", "nb_set_timing",
           "nb_get_timings", "nb_regular_force_noalloc", "nb_batch_plan", "nb_regular_force_batched",
           "nb_set_plan_table", "nb_set_source_range", "nb_irregular_force", "nb_sched_init", "nb_sched_free",
           "nb_sched_next", "nb_sched_update", "nb_sched_get", "nb_sched_counts", "nb_sched_last_error",
           "nb_sched_peek", "nb_ac_init", "nb_ac_step", "nb_ac_run", "nb_ac_get", "nb_ac_free", "nb_ac_last_error",
           "nb_inject_fault", "nb_sched_set_time", "nb_ac_snapshot_bytes", "nb_ac_save", "nb_ac_restore",
           "nb_row_order", "nb_hermite_predict", "nb_hermite_predict_backward", "nb_hermite_correct",
           "nb_hermite_correct_backward")
NB_FAULT_ALLOC, NB_FAULT_SYNC, NB_FAULT_STATUS = 1, 2, 3
NB_SOURCE_ALIGN = 256


def _torch():
    import torch
    return torch


class NBError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class NBOverflow(UserWarning):
    """Neighbour lists were cut at nb_cap or at the CSR capacity (results otherwise valid)."""


class _Config(ctypes.Structure):
    _fields_ = [("n_max", ctypes.c_int64), ("precision", ctypes.c_int32), ("nb_cap", ctypes.c_int32),
                ("device", ctypes.c_int32), ("flags", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class _ACParams(ctypes.Structure):
    _fields_ = [("eta_irr", ctypes.c_double), ("eta_reg", ctypes.c_double), ("eta_s", ctypes.c_double),
                ("dt_max", ctypes.c_double), ("nb_opt", ctypes.c_int32), ("level_max", ctypes.c_int32)]


_lib = None


def load_library(build_if_needed: bool = True):
    """Load libnbgpu.so (building it in-tree with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed and _build.needs_build():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library {_build.LIB} is missing; run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    P, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    st = ctypes.c_int
    sig = {
        "nb_version": (i32, []),
        "nb_init": (st, [ctypes.POINTER(P), ctypes.POINTER(_Config)]),
        "nb_free": (st, [P]),
        "nb_set_stream": (st, [P, P]),
        "nb_set_particles": (st, [P, i64, P, P, P, P, P, P, i32]),
        "nb_predict": (st, [P, dbl]),
        "nb_set_predicted": (st, [P, i64, P, P, P, i32]),
        "nb_get_predicted": (st, [P, P, P, i32]),
        "nb_get_records": (st, [P, P, i32]),
        "nb_regular_force": (st, [P, i64, P, P, i32, P, P, P, P, P, i64, P, i32]),
        "nb_regular_force_backward": (st, [P, i64, P, P, P, P, P, P, P, i32]),
        "nb_sync": (st, [P]),
        "nb_last_error": (ctypes.c_char_p, [P]),
        "nb_plan": (st, [P, i64, i64, P]),
        "nb_row_order": (st, [P, i64, P, P]),
        "nb_hermite_predict": (st, [P, i64, dbl, P, P, P, P, P, P, P]),
        "nb_hermite_predict_backward": (st, [P, i64, dbl, P, P, P, P, P, P, P]),
        "nb_hermite_correct": (st, [P, i64, dbl, P, P, P, P, P, P, P, P, P]),
        "nb_hermite_correct_backward": (st, [P, i64, dbl, P, P, P, P, P, P, P, P, P]),
        "nb_plan_for": (st, [i32, i32, P, i64, i64, i32, P]),
        "nb_set_plan_override": (st, [P, i32, i32, i32]),
        "nb_batch_plan": (st, [P, i64, P, P, i32]),
        "nb_set_plan_table": (st, [P, i32, P, P, P, P]),
        "nb_set_source_range": (st, [P, i64, i64]),
        "nb_inject_fault": (st, [P, i32, i32]),
        "nb_sched_init": (st, [ctypes.POINTER(P), i64, P, i32, i32, i32, P, i32]),
        "nb_sched_free": (st, [P]),
        "nb_sched_next": (st, [P, ctypes.POINTER(dbl), ctypes.POINTER(i64), ctypes.POINTER(P)]),
        "nb_sched_update": (st, [P, P, P, i32]),
        "nb_sched_get": (st, [P, P, P, ctypes.POINTER(dbl), i32]),
        "nb_sched_counts": (st, [P, P]),
        "nb_sched_last_error": (ctypes.c_char_p, [P]),
        "nb_sched_peek": (st, [P, ctypes.POINTER(dbl)]),
        "nb_ac_init": (st, [ctypes.POINTER(P), P, i64, P, P, P, P, ctypes.POINTER(_ACParams), i32]),
        "nb_ac_step": (st, [P, ctypes.POINTER(dbl), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "nb_ac_run": (st, [P, dbl, i64, P]),
        "nb_ac_get": (st, [P, P, P, P, P, P, P, P, P, P, i32]),
        "nb_ac_free": (st, [P]),
        "nb_sched_set_time": (st, [P, dbl]),
        "nb_ac_snapshot_bytes": (st, [P, ctypes.POINTER(ctypes.c_size_t)]),
        "nb_ac_save": (st, [P, P, ctypes.c_size_t]),
        "nb_ac_restore": (st, [ctypes.POINTER(P), P, P, ctypes.c_size_t]),
        "nb_ac_last_error": (ctypes.c_char_p, [P]),
        "nb_irregular_force": (st, [P, dbl, i64, P, P, P, P, P, P, P, P, P, i32]),
        "nb_regular_force_batched": (st, [P, P, P, P, P, P, P, P, i64, P]),
        "nb_set_timing": (st, [P, i32]),
        "nb_get_timings": (st, [P, P, P]),
        "nb_regular_force_noalloc": (st, [i64, P, P, P, i64, P, P, P, P, P, ctypes.c_char_p, i32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def plan_for(precision: str, num_sms: int, ctas_per_sm, n: int, n_i: int, nb_cap: int = 512) -> dict:
    """Host-only launch plan (no GPU needed)."""
    lib = load_library()
    out = (ctypes.c_int64 * 6)()
    occ = (ctypes.c_int32 * 21)(*ctas_per_sm) if ctas_per_sm is not None else None
    s = lib.nb_plan_for(PRECISIONS[precision], num_sms, ctypes.cast(occ, ctypes.c_void_p) if occ else None,
                        n, n_i, nb_cap, ctypes.cast(out, ctypes.c_void_p))
    if s != NB_OK:
        raise NBError(s, "nb_plan_for rejected its arguments")
    return dict(kernel=out[0], i_per_cta=out[1], splits=out[2], ctas=out[3], tile=out[4], variant=out[5])


def _ptr(t):
    """(pointer, on_device) of a contiguous torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None, None
    if isinstance(t, np.ndarray):
        if not t.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return t.ctypes.data, 0
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return t.data_ptr(), 1 if t.is_cuda else 0


@dataclass
class ForceResult:
    acc: object
    jerk: object
    pot: object
    nb_off: object = None
    nb_idx: object = None
    nb_count: object = None

    def neighbour_lists(self):
        """Per-row neighbour index arrays (host numpy; synchronises)."""
        off = self.nb_off.cpu().numpy() if hasattr(self.nb_off, "cpu") else self.nb_off
        idx = self.nb_idx.cpu().numpy() if hasattr(self.nb_idx, "cpu") else self.nb_idx
        return [idx[off[k]:off[k + 1]] for k in range(len(off) - 1)]


class Context:
    """One nb_ctx: device state of up to n_max particles at a fixed precision."""

    def __init__(self, n_max: int, precision: str = "mixed", nb_cap: int = 512, device: int = 0,
                 stream=None):
        import torch
        self._torch = torch
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available: the regular-force library has no CPU path")
        self.precision = precision
        self.nb_cap = nb_cap
        self.device = device
        self._stream = stream  # None: follow torch's current stream
        cfg = _Config(n_max=n_max, precision=PRECISIONS[precision], nb_cap=nb_cap, device=device, flags=0,
                      stream=None)
        h = ctypes.c_void_p()
        s = self.lib.nb_init(ctypes.byref(h), ctypes.byref(cfg))
        if s != NB_OK:
            raise NBError(s, f"nb_init(n_max={n_max}, precision={precision}, nb_cap={nb_cap}) failed")
        self.h = h
        self.n = 0

    # -- plumbing ------------------------------------------------------------------------
    def _check(self, s, what, allow_overflow=True):
        if s == NB_OK:
            return s
        msg = self.lib.nb_last_error(self.h).decode()
        if s == NB_ERR_NB_OVERFLOW and allow_overflow:
            import warnings
            warnings.warn(f"{what}: {msg}", NBOverflow, stacklevel=3)
            return s
        raise NBError(s, f"{what}: {msg}")

    def _bind_stream(self):
        torch = self._torch
        st = self._stream if self._stream is not None else torch.cuda.current_stream(self.device)
        self.lib.nb_set_stream(self.h, ctypes.c_void_p(st.cuda_stream))

    def close(self):
        if getattr(self, "h", None):
            self.lib.nb_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI mirrors --------------------------------------------------------------------
    def set_particles(self, x, v, a, jerk, m, t_last):
        ptrs = [_ptr(q) for q in (x, v, a, jerk, m, t_last)]
        dev = {p[1] for p in ptrs}
        if len(dev) != 1:
            raise ValueError("all arrays must live on the same side (host or device)")
        self._bind_stream()
        n = int(m.shape[0])
        s = self.lib.nb_set_particles(self.h, n, *[p[0] for p in ptrs], dev.pop())
        self._check(s, "nb_set_particles")
        self.n = n

    def predict(self, t: float):
        self._bind_stream()
        self._check(self.lib.nb_predict(self.h, float(t)), "nb_predict")

    def set_predicted(self, xp, vp, m):
        ptrs = [_ptr(q) for q in (xp, vp, m)]
        dev = {p[1] for p in ptrs}
        if len(dev) != 1:
            raise ValueError("all arrays must live on the same side (host or device)")
        self._bind_stream()
        n = int(m.shape[0])
        self._check(self.lib.nb_set_predicted(self.h, n, *[p[0] for p in ptrs], dev.pop()), "nb_set_predicted")
        self.n = n

    def get_predicted(self):
        torch = self._torch
        xp = torch.empty((self.n, 3), dtype=torch.float64, device=f"cuda:{self.device}")
        vp = torch.empty_like(xp)
        self._bind_stream()
        self._check(self.lib.nb_get_predicted(self.h, xp.data_ptr(), vp.data_ptr(), 1), "nb_get_predicted")
        return xp, vp

    def get_records(self):
        """The j-records of the predicted particles: (n, 12) float32 (mixed) or (n, 8) float64."""
        torch = self._torch
        mixed = self.precision == "mixed"
        rec = torch.empty((self.n, 12 if mixed else 8), dtype=torch.float32 if mixed else torch.float64,
                          device=f"cuda:{self.device}")
        self._bind_stream()
        self._check(self.lib.nb_get_records(self.h, rec.data_ptr(), 1), "nb_get_records")
        return rec

    def regular_force(self, idx, rs2, neighbours: bool = True, nb_capacity: int | None = None,
                      out: ForceResult | None = None) -> ForceResult:
        """Regular force, jerk, potential (+ CSR neighbour lists) of the active block idx.

        idx: int32 tensor (device) or numpy array (host); rs2: scalar float or per-row
        array.  Device inputs give device outputs (asynchronous; nb_sync() reports the
        deferred status); host inputs give host outputs (synchronous).
        """
        torch = self._torch
        on_dev = isinstance(idx, torch.Tensor) and idx.is_cuda
        n_i = int(idx.shape[0])
        scalar = np.isscalar(rs2) or (hasattr(rs2, "ndim") and rs2.ndim == 0)
        if on_dev:
            dev = idx.device
            if isinstance(rs2, torch.Tensor) and rs2.is_cuda and rs2.dtype == torch.float64:
                # a device tensor: one entry = the same r_s^2 for every row
                rs2_t = rs2.reshape(-1).contiguous()
                scalar = rs2_t.numel() == 1
            elif scalar:
                rs2_t = torch.full((1,), float(rs2), dtype=torch.float64, device=dev)
            else:
                rs2_t = torch.as_tensor(rs2, dtype=torch.float64, device=dev).contiguous()
            if out is None:
                cap = (nb_capacity if nb_capacity is not None else n_i * self.nb_cap) if neighbours else 0
                out = ForceResult(
                    acc=torch.empty((n_i, 3), dtype=torch.float64, device=dev),
                    jerk=torch.empty((n_i, 3), dtype=torch.float64, device=dev),
                    pot=torch.empty((n_i,), dtype=torch.float64, device=dev),
                    nb_off=torch.empty((n_i + 1,), dtype=torch.int64, device=dev) if neighbours else None,
                    nb_idx=torch.empty((max(cap, 1),), dtype=torch.int32, device=dev) if neighbours else None,
                    nb_count=torch.empty((n_i,), dtype=torch.int32, device=dev) if neighbours else None)
            self._bind_stream()
            cap_elems = int(out.nb_idx.numel()) if out.nb_idx is not None else 0
            s = self.lib.nb_regular_force(
                self.h, n_i, idx.data_ptr(), rs2_t.data_ptr(), 1 if scalar else 0, out.acc.data_ptr(),
                out.jerk.data_ptr(), out.pot.data_ptr(), _ptr(out.nb_off)[0], _ptr(out.nb_idx)[0], cap_elems,
                _ptr(out.nb_count)[0], 1)
            self._check(s, "nb_regular_force")
            out._rs2_keepalive = rs2_t
            return out
        idx_np = np.ascontiguousarray(np.asarray(idx), dtype=np.int32)
        rs2_np = np.ascontiguousarray(np.atleast_1d(np.asarray(rs2, dtype=np.float64)))
        cap = (nb_capacity if nb_capacity is not None else n_i * self.nb_cap) if neighbours else 0
        res = ForceResult(acc=np.empty((n_i, 3)), jerk=np.empty((n_i, 3)), pot=np.empty(n_i),
                          nb_off=np.empty(n_i + 1, np.int64) if neighbours else None,
                          nb_idx=np.empty(max(cap, 1), np.int32) if neighbours else None,
                          nb_count=np.empty(n_i, np.int32) if neighbours else None)
        self._bind_stream()
        s = self.lib.nb_regular_force(
            self.h, n_i, idx_np.ctypes.data, rs2_np.ctypes.data, 1 if scalar else 0, res.acc.ctypes.data,
            res.jerk.ctypes.data, res.pot.ctypes.data, _ptr(res.nb_off)[0], _ptr(res.nb_idx)[0],
            cap if neighbours else 0, _ptr(res.nb_count)[0], 0)
        res.status = self._check(s, "nb_regular_force")
        return res

    def regular_force_backward(self, idx, g_acc, g_jerk, g_pot):
        """(g_x, g_v, g_m) for all n particles (device tensors in, device tensors out)."""
        torch = self._torch
        dev = idx.device
        gx = torch.empty((self.n, 3), dtype=torch.float64, device=dev)
        gv = torch.empty_like(gx)
        gm = torch.empty((self.n,), dtype=torch.float64, device=dev)
        self._bind_stream()
        s = self.lib.nb_regular_force_backward(self.h, int(idx.shape[0]), idx.data_ptr(), g_acc.data_ptr(),
                                               g_jerk.data_ptr(), g_pot.data_ptr(), gx.data_ptr(), gv.data_ptr(),
                                               gm.data_ptr(), 1)
        self._check(s, "nb_regular_force_backward")
        return gx, gv, gm

    def irregular_force(self, t: float, idx, nb_off, nb_idx, regular: ForceResult | None = None):
        """nb_irregular_force: (acc, jerk, pot) of the rows idx over their CSR neighbour lists,
        i and its neighbours predicted to time t from the loaded Hermite state.  With
        `regular` (the all-j result of regular_force for the same rows, same side), its
        acc / jerk / pot are replaced in place by the part from outside the lists.  Device
        tensors give device outputs (asynchronous), numpy arrays host outputs."""
        torch = self._torch
        on_dev = isinstance(idx, torch.Tensor) and idx.is_cuda
        n_i = int(idx.shape[0])
        reg = (regular.acc, regular.jerk, regular.pot) if regular is not None else (None, None, None)
        if on_dev:
            dev = idx.device
            acc = torch.empty((n_i, 3), dtype=torch.float64, device=dev)
            jerk = torch.empty_like(acc)
            pot = torch.empty((n_i,), dtype=torch.float64, device=dev)
            ptr = lambda q: q.data_ptr() if q is not None else None
            self._bind_stream()
            s = self.lib.nb_irregular_force(self.h, float(t), n_i, idx.data_ptr(), nb_off.data_ptr(),
                                            nb_idx.data_ptr(), acc.data_ptr(), jerk.data_ptr(), pot.data_ptr(),
                                            *[ptr(q) for q in reg], 1)
            self._check(s, "nb_irregular_force")
            return acc, jerk, pot
        idx_np = np.ascontiguousarray(np.asarray(idx), dtype=np.int32)
        off_np = np.ascontiguousarray(np.asarray(nb_off), dtype=np.int64)
        nb_np = np.ascontiguousarray(np.asarray(nb_idx), dtype=np.int32)
        if nb_np.size == 0:
            nb_np = np.zeros(1, np.int32)
        acc, jerk, pot = np.empty((n_i, 3)), np.empty((n_i, 3)), np.empty(n_i)
        for q in reg:
            if q is not None and not (isinstance(q, np.ndarray) and q.flags.c_contiguous and q.dtype == np.float64):
                raise ValueError("regular results must be contiguous float64 numpy arrays in host mode")
        self._bind_stream()
        s = self.lib.nb_irregular_force(self.h, float(t), n_i, idx_np.ctypes.data, off_np.ctypes.data,
                                        nb_np.ctypes.data, acc.ctypes.data, jerk.ctypes.data, pot.ctypes.data,
                                        *[q.ctypes.data if q is not None else None for q in reg], 0)
        self._check(s, "nb_irregular_force")
        return acc, jerk, pot

    def set_timing(self, enable: bool = True):
        self._check(self.lib.nb_set_timing(self.h, 1 if enable else 0), "nb_set_timing")

    PHASES = ("predict", "force", "reduce", "neighbours", "backward", "irregular", "order")

    def timings(self) -> dict:
        """{phase: (device ms, kernel launches)} since the last call; synchronises."""
        ms = (ctypes.c_double * len(self.PHASES))()
        ln = (ctypes.c_int64 * len(self.PHASES))()
        self._check(self.lib.nb_get_timings(self.h, ctypes.cast(ms, ctypes.c_void_p),
                                            ctypes.cast(ln, ctypes.c_void_p)), "nb_get_timings")
        return {p: (ms[q], ln[q]) for q, p in enumerate(self.PHASES)}

    def sync(self, allow_overflow: bool = True) -> int:
        return self._check(self.lib.nb_sync(self.h), "nb_sync", allow_overflow)

    # ---- Hermite predictor / corrector over device arrays, and their VJPs ----------------
    @staticmethod
    def _dev64(*ts):
        for t in ts:
            if not (t.is_cuda and t.dtype == _torch().float64 and t.is_contiguous()):
                raise ValueError("Hermite arrays must be contiguous float64 device tensors")

    def hermite_predict(self, t: float, x, v, a, jerk, t_last):
        """nb_hermite_predict: (xp, vp) at time t of the (n,3) states, t_last (n)."""
        self._dev64(x, v, a, jerk, t_last)
        xp, vp = _torch().empty_like(x), _torch().empty_like(v)
        self._check(self.lib.nb_hermite_predict(self.h, x.shape[0], float(t), x.data_ptr(), v.data_ptr(), a.data_ptr(),
                                                jerk.data_ptr(), t_last.data_ptr(), xp.data_ptr(), vp.data_ptr()),
                    "nb_hermite_predict")
        return xp, vp

    def hermite_predict_backward(self, t: float, t_last, g_xp, g_vp):
        """nb_hermite_predict_backward: (g_x, g_v, g_a, g_jerk)."""
        self._dev64(t_last, g_xp, g_vp)
        out = [_torch().empty_like(g_xp) for _ in range(4)]
        self._check(self.lib.nb_hermite_predict_backward(self.h, g_xp.shape[0], float(t), t_last.data_ptr(),
                                                         g_xp.data_ptr(), g_vp.data_ptr(),
                                                         *[o.data_ptr() for o in out]), "nb_hermite_predict_backward")
        return tuple(out)

    def hermite_correct(self, t: float, t_last, xp, vp, a0, j0, a1, j1):
        """nb_hermite_correct: (x1, v1) of rows stepping from t_last (n) to t."""
        self._dev64(t_last, xp, vp, a0, j0, a1, j1)
        x1, v1 = _torch().empty_like(xp), _torch().empty_like(vp)
        self._check(self.lib.nb_hermite_correct(self.h, xp.shape[0], float(t), t_last.data_ptr(), xp.data_ptr(),
                                                vp.data_ptr(), a0.data_ptr(), j0.data_ptr(), a1.data_ptr(),
                                                j1.data_ptr(), x1.data_ptr(), v1.data_ptr()), "nb_hermite_correct")
        return x1, v1

    def hermite_correct_backward(self, t: float, t_last, g_x1, g_v1):
        """nb_hermite_correct_backward: (g_xp, g_vp, g_a0, g_j0, g_a1, g_j1)."""
        self._dev64(t_last, g_x1, g_v1)
        out = [_torch().empty_like(g_x1) for _ in range(6)]
        self._check(self.lib.nb_hermite_correct_backward(self.h, g_x1.shape[0], float(t), t_last.data_ptr(),
                                                         g_x1.data_ptr(), g_v1.data_ptr(),
                                                         *[o.data_ptr() for o in out]), "nb_hermite_correct_backward")
        return tuple(out)

    def row_order(self, idx):
        """nb_row_order: the spatial (Morton) order of the rows idx (device int32 tensor) that
        the anchored force kernel takes; returns the permutation as a device int32 tensor."""
        import torch
        perm = torch.empty_like(idx)
        self._check(self.lib.nb_row_order(self.h, int(idx.shape[0]), idx.data_ptr(), perm.data_ptr()), "nb_row_order")
        return perm

    def plan(self, n: int, n_i: int) -> dict:
        out = (ctypes.c_int64 * 6)()
        self._check(self.lib.nb_plan(self.h, n, n_i, ctypes.cast(out, ctypes.c_void_p)), "nb_plan")
        return dict(kernel=out[0], i_per_cta=out[1], splits=out[2], ctas=out[3], tile=out[4], variant=out[5])

    def batch_plan(self, cluster_off, active_off, variant: int = -1):
        """nb_batch_plan: describe the clusters (host int64 offset arrays of C+1 entries)."""
        co = np.ascontiguousarray(np.asarray(cluster_off), dtype=np.int64)
        ao = np.ascontiguousarray(np.asarray(active_off), dtype=np.int64)
        if co.shape != ao.shape:
            raise ValueError("cluster_off and active_off must have the same length")
        self._bind_stream()
        self._check(self.lib.nb_batch_plan(self.h, co.shape[0] - 1, co.ctypes.data, ao.ctypes.data, int(variant)),
                    "nb_batch_plan")
        self._batch_rows = int(ao[-1])

    def regular_force_batched(self, idx, rs2, neighbours: bool = True, nb_capacity: int | None = None,
                              out: ForceResult | None = None) -> ForceResult:
        """One launch for all clusters of the batch plan (device tensors in and out)."""
        torch = self._torch
        rows = self._batch_rows
        dev = idx.device
        if out is None:
            cap = (nb_capacity if nb_capacity is not None else rows * self.nb_cap) if neighbours else 0
            out = ForceResult(
                acc=torch.empty((rows, 3), dtype=torch.float64, device=dev),
                jerk=torch.empty((rows, 3), dtype=torch.float64, device=dev),
                pot=torch.empty((rows,), dtype=torch.float64, device=dev),
                nb_off=torch.empty((rows + 1,), dtype=torch.int64, device=dev) if neighbours else None,
                nb_idx=torch.empty((max(cap, 1),), dtype=torch.int32, device=dev) if neighbours else None,
                nb_count=torch.empty((rows,), dtype=torch.int32, device=dev) if neighbours else None)
        self._bind_stream()
        cap_elems = int(out.nb_idx.numel()) if out.nb_idx is not None else 0
        s = self.lib.nb_regular_force_batched(self.h, idx.data_ptr(), rs2.data_ptr(), out.acc.data_ptr(),
                                              out.jerk.data_ptr(), out.pot.data_ptr(), _ptr(out.nb_off)[0],
                                              _ptr(out.nb_idx)[0], cap_elems, _ptr(out.nb_count)[0])
        self._check(s, "nb_regular_force_batched")
        return out

    def apply_tuned(self, n: int | None = None) -> bool:
        """Install the autotuner's plan table for this GPU, precision and particle count
        (tuned_plans.json, written by paper_1504_03687_gb300.tune); False if none exists."""
        from . import tune
        key = tune.device_key(self.precision, n if n is not None else max(self.n, 1))
        table = tune.load_table(key)
        if not table:
            return False
        tune.apply_table(self, table)
        return True

    def set_plan_table(self, entries):
        """nb_set_plan_table from [(ni_max, kernel, variant, splits), ...] (sorted by ni_max)."""
        e = sorted(entries)
        nim = np.array([x[0] for x in e], np.int64)
        ker = np.array([x[1] for x in e], np.int32)
        var = np.array([x[2] for x in e], np.int32)
        spl = np.array([x[3] for x in e], np.int32)
        self._check(self.lib.nb_set_plan_table(self.h, len(e), nim.ctypes.data, ker.ctypes.data, var.ctypes.data,
                                               spl.ctypes.data), "nb_set_plan_table")

    def set_source_range(self, j_lo: int = 0, j_hi: int = 0):
        """nb_set_source_range: later regular_force calls sum over source particles j in
        [j_lo, j_hi) only; (0, 0) = all particles."""
        self._check(self.lib.nb_set_source_range(self.h, int(j_lo), int(j_hi)), "nb_set_source_range")

    def inject_fault(self, kind: int, after: int = 0):
        """nb_inject_fault: arm a simulated allocation / synchronisation / status-read failure."""
        self._check(self.lib.nb_inject_fault(self.h, int(kind), int(after)), "nb_inject_fault")

    def set_plan_override(self, kernel: int = -1, variant: int = 0, splits: int = 1):
        """Force (kernel, variant, splits) for later regular_force calls; kernel < 0 = automatic."""
        self._check(self.lib.nb_set_plan_override(self.h, kernel, variant, splits), "nb_set_plan_override")


class _DeviceView:
    """Zero-copy CUDA array view of library-owned device memory (int32)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4", "data": (ptr, False), "version": 3,
                                         "strides": None}


class Scheduler:
    """nb_sched: the block-step sorting list (Sec. 3.3.1) on the device.

    levels: initial level of every particle (step 2^-level), host array or device tensor.
    next() -> (t_block, n_active); active() is a zero-copy int32 device view of the active
    particles (the list prefix), valid until update(); update(want) commits the step with
    the requested levels (list order) and returns the granted ones."""

    def __init__(self, levels, level_min: int, level_max: int, device: int = 0):
        import torch
        self._torch = torch
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available: the scheduler has no CPU path")
        self.device = device
        st = torch.cuda.current_stream(device)
        self._stream = st
        on_dev = isinstance(levels, torch.Tensor) and levels.is_cuda
        lv = levels.to(torch.int32).contiguous() if on_dev else np.ascontiguousarray(levels, dtype=np.int32)
        self.n = int(lv.shape[0])
        h = ctypes.c_void_p()
        s = self.lib.nb_sched_init(ctypes.byref(h), self.n, lv.data_ptr() if on_dev else lv.ctypes.data,
                                   int(level_min), int(level_max), device, ctypes.c_void_p(st.cuda_stream),
                                   1 if on_dev else 0)
        if s != NB_OK:
            raise NBError(s, f"nb_sched_init(n={self.n}, levels in [{level_min}, {level_max}]) failed")
        self.h = h
        self.n_active = 0
        self._list = None

    def _check(self, s, what):
        if s != NB_OK:
            raise NBError(s, f"{what}: {self.lib.nb_sched_last_error(self.h).decode()}")

    def next(self):
        t = ctypes.c_double()
        na = ctypes.c_int64()
        ptr = ctypes.c_void_p()
        self._check(self.lib.nb_sched_next(self.h, ctypes.byref(t), ctypes.byref(na), ctypes.byref(ptr)),
                    "nb_sched_next")
        self.n_active = na.value
        self._list = ptr.value
        return t.value, na.value

    def active(self):
        """int32 device tensor viewing the active particles (no copy)."""
        return self._torch.as_tensor(_DeviceView(self._list, self.n_active), device=f"cuda:{self.device}")

    def update(self, want, granted: bool = True):
        torch = self._torch
        if isinstance(want, torch.Tensor) and want.is_cuda:
            w = want.to(torch.int32).contiguous()
            g = torch.empty_like(w) if granted else None
            self._check(self.lib.nb_sched_update(self.h, w.data_ptr(), g.data_ptr() if g is not None else None, 1),
                        "nb_sched_update")
            return g
        w = np.ascontiguousarray(want, dtype=np.int32)
        g = np.empty_like(w) if granted else None
        self._check(self.lib.nb_sched_update(self.h, w.ctypes.data, g.ctypes.data if g is not None else None, 0),
                    "nb_sched_update")
        return g

    def get(self):
        """(list, levels, t_now) on the host."""
        lst, lev = np.empty(self.n, np.int32), np.empty(self.n, np.int32)
        t = ctypes.c_double()
        self._check(self.lib.nb_sched_get(self.h, lst.ctypes.data, lev.ctypes.data, ctypes.byref(t), 0),
                    "nb_sched_get")
        return lst, lev, t.value

    def counts(self):
        c = np.empty(64, np.int64)
        self._check(self.lib.nb_sched_counts(self.h, c.ctypes.data), "nb_sched_counts")
        return c

    def close(self):
        if getattr(self, "h", None):
            self.lib.nb_sched_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ACIntegrator:
    """nb_ac: the Ahmad-Cohen Hermite block-step integrator on the device, driving the
    context `ctx` (its precision and nb_cap) and its own block-step scheduler."""

    def __init__(self, ctx: Context, m, x, v, rs2, eta_irr=0.02, eta_reg=0.03, eta_s=0.01, dt_max=0.125,
                 nb_opt=0, level_max=40):
        self.ctx, self.lib = ctx, ctx.lib
        n = int(np.asarray(m).shape[0])
        self.n, self.cap = n, ctx.nb_cap
        m_, x_, v_ = (np.ascontiguousarray(q, dtype=np.float64) for q in (m, x, v))
        r_ = np.ascontiguousarray(np.broadcast_to(np.asarray(rs2, np.float64), (n,)))
        prm = _ACParams(eta_irr, eta_reg, eta_s, dt_max, int(nb_opt), int(level_max))
        ctx._bind_stream()
        h = ctypes.c_void_p()
        s = self.lib.nb_ac_init(ctypes.byref(h), ctx.h, n, m_.ctypes.data, x_.ctypes.data, v_.ctypes.data,
                                r_.ctypes.data, ctypes.byref(prm), 0)
        if s != NB_OK:
            raise NBError(s, f"nb_ac_init: {self.lib.nb_ac_last_error(h).decode() if h.value else ''}")
        self.h = h
        ctx.n = n

    def _check(self, s, what, allow=()):
        if s != NB_OK and s not in allow:
            raise NBError(s, f"{what}: {self.lib.nb_ac_last_error(self.h).decode()}")
        return s

    def step(self):
        t, na, nr = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.nb_ac_step(self.h, ctypes.byref(t), ctypes.byref(na), ctypes.byref(nr)), "nb_ac_step")
        return t.value, na.value, nr.value

    def run(self, t_end: float, max_blocks: int = 0) -> dict:
        st = np.zeros(6)
        self._check(self.lib.nb_ac_run(self.h, float(t_end), int(max_blocks), st.ctypes.data), "nb_ac_run",
                    allow=(NB_ERR_STATE,) if max_blocks else ())
        return dict(blocks=int(st[0]), irregular_steps=int(st[1]), regular_steps=int(st[2]),
                    neighbour_pairs=st[3], all_pairs=st[4], device_blocks=int(st[5]))

    def get(self) -> dict:
        n, cap = self.n, self.cap
        out = dict(x=np.empty((n, 3)), v=np.empty((n, 3)), t=np.empty(n), dt=np.empty(n), DT=np.empty(n),
                   T=np.empty(n), rs2=np.empty(n), nb_count=np.empty(n, np.int32),
                   nb_lists=np.empty((n, cap), np.int32))
        self._check(self.lib.nb_ac_get(self.h, *[out[k].ctypes.data for k in
                                                 ("x", "v", "t", "dt", "DT", "T", "rs2", "nb_count", "nb_lists")], 0),
                    "nb_ac_get")
        return out

    def save(self) -> bytes:
        """nb_ac_save: the complete integrator state as bytes (a checkpoint)."""
        nb = ctypes.c_size_t()
        self._check(self.lib.nb_ac_snapshot_bytes(self.h, ctypes.byref(nb)), "nb_ac_snapshot_bytes")
        buf = np.empty(nb.value, np.uint8)
        self._check(self.lib.nb_ac_save(self.h, buf.ctypes.data, nb.value), "nb_ac_save")
        return buf.tobytes()

    @classmethod
    def restore(cls, ctx: Context, blob: bytes) -> "ACIntegrator":
        """nb_ac_restore: an integrator on ctx resumed from a checkpoint of save()."""
        self = cls.__new__(cls)
        self.ctx, self.lib = ctx, ctx.lib
        buf = np.frombuffer(blob, np.uint8)
        self.n = int(np.frombuffer(blob[8:16], np.int64)[0])
        self.cap = ctx.nb_cap
        ctx._bind_stream()
        h = ctypes.c_void_p()
        s = self.lib.nb_ac_restore(ctypes.byref(h), ctx.h, buf.ctypes.data, buf.size)
        if s != NB_OK:
            raise NBError(s, "nb_ac_restore failed")
        self.h = h
        ctx.n = self.n
        return self

    def close(self):
        if getattr(self, "h", None):
            self.lib.nb_ac_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
