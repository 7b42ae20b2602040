"""ctypes binding of libsph (include/sph.h): argument marshalling only.

Every step of the SPH path runs in the CUDA kernels of ``libsph.so``; this module
only turns torch CUDA tensors into the pointer structs the C-ABI takes.  There is
no CPU fallback: if the library is missing or cannot load, :func:`lib` raises.

The C entry points are exposed under their C names (``sph_init``,
``sph_build_cells``, ``sph_density``, ``sph_force``, ``sph_step``, ...);
:class:`Context` and :class:`Particles` are small conveniences on top.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

SPH_OK = 0
SPH_ERR_INVALID_ARG = 1
SPH_ERR_CUDA = 2
SPH_ERR_NOT_CONVERGED = 3
SPH_ERR_H_EXCEEDS_CELL = 4
SPH_ERR_TIMEOUT = 5
SPH_ERR_NAN = 6
SPH_ERR_STATE = 7
SPH_ERR_CAPACITY = 8
SPH_ERR_PRECISION = 9
SPH_FRAME_RATIO = 64
SPH_FLAG_TIMING = 1
SPH_FLAG_NGB_HASH = 2
SPH_FLAG_AUTOTUNE = 4
SPH_FLAG_ADAPTIVE = 8
SPH_FLAG_TREE_H_GUESS = 16
SPH_FLAG_HPREDICT = 32
SPH_FLAG_AXIS_SWEEP = 64
SPH_FLAG_SYMMETRIC = 128
SPH_FLAG_BIN_LIMITER = 256
SPH_BIN_LIMIT_LEVELS = 2
SPH_HP_NBF16 = 4544
SPH_HP_NF32 = 143
SPH_HP_NPARAM = 4673
SPH_SORT_STATIC_MAX_N = 262144

_NAMES = {0: "SPH_OK", 1: "SPH_ERR_INVALID_ARG", 2: "SPH_ERR_CUDA", 3: "SPH_ERR_NOT_CONVERGED",
          4: "SPH_ERR_H_EXCEEDS_CELL", 5: "SPH_ERR_TIMEOUT", 6: "SPH_ERR_NAN", 7: "SPH_ERR_STATE",
          8: "SPH_ERR_CAPACITY", 9: "SPH_ERR_PRECISION"}

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "sph.h")


class SphError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class sph_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("box_size", ctypes.c_double), ("gamma", ctypes.c_float),
                ("n_ngb", ctypes.c_float), ("h_tol", ctypes.c_float), ("alpha_visc", ctypes.c_float),
                ("cfl", ctypes.c_float), ("cell_factor", ctypes.c_float),
                ("max_h_iter", ctypes.c_int32), ("use_balsara", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("tile_width", ctypes.c_int32), ("n_boxes", ctypes.c_int32),
                ("box_offsets", ctypes.c_void_p), ("leaf_max", ctypes.c_int32),
                ("list_reserve", ctypes.c_int64)]


_PFIELDS = ["x", "y", "z", "vx", "vy", "vz", "m", "u", "h", "rho", "P", "c", "f", "divv", "curl",
            "n_ngb", "ax", "ay", "az", "dudt", "vsig"]


class sph_particles(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in _PFIELDS]


class sph_conserved(ctypes.Structure):
    _fields_ = [("momentum", ctypes.c_double * 3), ("e_kin", ctypes.c_double),
                ("e_th", ctypes.c_double), ("dt_next", ctypes.c_double),
                ("u_floors", ctypes.c_int64)]


SPH_MAX_BINS = 24


class sph_bin_stats(ctypes.Structure):
    _fields_ = [("substeps", ctypes.c_int64), ("updates", ctypes.c_int64), ("cfl_over", ctypes.c_int64),
                ("bin_count", ctypes.c_int64 * (SPH_MAX_BINS + 1)), ("limited", ctypes.c_int64),
                ("woken", ctypes.c_int64), ("limit_sweeps", ctypes.c_int64)]


class sph_stats(ctypes.Structure):
    _fields_ = [("nc", ctypes.c_int32), ("rebuilds", ctypes.c_int32), ("n_cells", ctypes.c_int64),
                ("cell_size", ctypes.c_double), ("density_passes", ctypes.c_int64),
                ("force_passes", ctypes.c_int64), ("density_pairs", ctypes.c_int64),
                ("density_targets", ctypes.c_int64), ("force_pairs", ctypes.c_int64),
                ("density_candidates", ctypes.c_int64), ("force_candidates", ctypes.c_int64),
                ("t_density_ms", ctypes.c_double), ("t_force_ms", ctypes.c_double),
                ("t_build_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("tile_width", ctypes.c_int32), ("cell_factor", ctypes.c_float),
                ("graph_steps", ctypes.c_int64), ("leaf_max", ctypes.c_int32),
                ("hp_samples", ctypes.c_int64), ("grav_passes", ctypes.c_int64),
                ("grav_pairs", ctypes.c_int64), ("t_grav_ms", ctypes.c_double),
                ("force_symmetric", ctypes.c_int32), ("axis_sweep", ctypes.c_int32),
                ("density_streamed", ctypes.c_int64),
                ("density_staged", ctypes.c_int64), ("force_streamed", ctypes.c_int64),
                ("force_staged", ctypes.c_int64)]


_lock = threading.Lock()
_lib = None


def lib(build_if_missing: bool = True):
    """Load libsph.so (building it with nvcc first when asked).  Raises when the
    library cannot be built or loaded -- there is no other implementation."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libsph.so not built ({path}); run paper_1508_00115_gb300.build")
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        C = ctypes.c_int
        sig = {
            "sph_default_params": (C, [ctypes.POINTER(sph_params)]),
            "sph_init": (C, [ctypes.POINTER(P), ctypes.POINTER(sph_params), C, P]),
            "sph_set_n": (C, [P, ctypes.c_int64]),
            "sph_build_cells": (C, [P, ctypes.POINTER(sph_particles)]),
            "sph_density": (C, [P, ctypes.POINTER(sph_particles), ctypes.POINTER(ctypes.c_int32)]),
            "sph_force": (C, [P, ctypes.POINTER(sph_particles)]),
            "sph_step": (C, [P, ctypes.POINTER(sph_particles), ctypes.c_double,
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(sph_conserved)]),
            "sph_step_host": (C, [P, ctypes.POINTER(sph_particles), ctypes.c_double,
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(sph_conserved)]),
            "sph_steps": (C, [P, ctypes.POINTER(sph_particles), ctypes.c_int32, ctypes.c_double,
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(sph_conserved)]),
            "sph_step_bins": (C, [P, ctypes.POINTER(sph_particles), ctypes.c_double, ctypes.c_int32,
                                  ctypes.POINTER(sph_conserved), ctypes.POINTER(sph_bin_stats)]),
            "sph_get_bins": (C, [P, P]),
            "sph_get_permutation": (C, [P, P]),
            "sph_reset_ids": (C, [P]),
            "sph_get_cell_keys": (C, [P, P]),
            "sph_get_ngb_hash": (C, [P, P]),
            "sph_sort_keys_static": (C, [P, P, P, ctypes.c_int64, ctypes.c_int32, P]),
            "sph_hpredict_init": (C, [P, ctypes.c_uint64]),
            "sph_hpredict_load": (C, [P, P, P]),
            "sph_hpredict_save": (C, [P, P, P]),
            "sph_hpredict_params": (C, [P, P]),
            "sph_hpredict_features": (C, [P, ctypes.POINTER(sph_particles), ctypes.c_double, P]),
            "sph_hpredict_targets": (C, [P, ctypes.POINTER(sph_particles), P]),
            "sph_hpredict_eval": (C, [P, P, ctypes.c_int64, P]),
            "sph_hpredict_train": (C, [P, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_uint64,
                                       ctypes.POINTER(ctypes.c_float)]),
            "sph_hpredict_collect": (C, [P, P, P, ctypes.c_int64]),
            "sph_gravity_p2p": (C, [P, ctypes.c_double, ctypes.c_double, P, P, P, P]),
            "sph_fp32_peak": (C, [P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_float)]),
            "sph_get_stats": (C, [P, ctypes.POINTER(sph_stats)]),
            "sph_reset_stats": (C, [P]),
            "sph_last_error": (ctypes.c_char_p, [P]),
            "sph_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def header_symbols() -> list[str]:
    """Entry points declared in include/sph.h."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(sph_\w+)\s*\(", text,
                                 flags=re.M)))


# ------------------------------------------------------------------ C names


def sph_default_params() -> sph_params:
    p = sph_params()
    lib().sph_default_params(ctypes.byref(p))
    return p


def _check(rc: int, ctx=None, allow=()):
    if rc != SPH_OK and rc not in allow:
        msg = lib().sph_last_error(ctx).decode() if ctx else ""
        raise SphError(rc, msg)
    return rc


def sph_init(params: sph_params, device: int = 0, stream: int | None = None):
    h = ctypes.c_void_p()
    rc = lib().sph_init(ctypes.byref(h), ctypes.byref(params), int(device),
                        ctypes.c_void_p(stream or 0))
    if rc != SPH_OK:
        raise SphError(rc, "sph_init failed (check parameters / device)")
    return h


def sph_build_cells(ctx, parts: sph_particles) -> int:
    return _check(lib().sph_build_cells(ctx, ctypes.byref(parts)), ctx)


def sph_density(ctx, parts: sph_particles, allow_not_converged: bool = False) -> int:
    it = ctypes.c_int32(0)
    allow = (SPH_ERR_NOT_CONVERGED,) if allow_not_converged else ()
    _check(lib().sph_density(ctx, ctypes.byref(parts), ctypes.byref(it)), ctx, allow)
    return int(it.value)


def sph_force(ctx, parts: sph_particles) -> int:
    return _check(lib().sph_force(ctx, ctypes.byref(parts)), ctx)


def sph_step(ctx, parts: sph_particles, dt: float = 0.0, allow=()):
    used = ctypes.c_double(0)
    cons = sph_conserved()
    _check(lib().sph_step(ctx, ctypes.byref(parts), float(dt), ctypes.byref(used),
                          ctypes.byref(cons)), ctx, allow)
    return float(used.value), _cons_dict(cons)


def sph_steps(ctx, parts: sph_particles, n_steps: int, dt: float = 0.0, allow=()):
    last = ctypes.c_double(0)
    cons = sph_conserved()
    _check(lib().sph_steps(ctx, ctypes.byref(parts), int(n_steps), float(dt), ctypes.byref(last),
                           ctypes.byref(cons)), ctx, allow)
    return float(last.value), _cons_dict(cons)


def sph_step_host(ctx, parts: sph_particles, dt: float = 0.0):
    used = ctypes.c_double(0)
    cons = sph_conserved()
    _check(lib().sph_step_host(ctx, ctypes.byref(parts), float(dt), ctypes.byref(used),
                               ctypes.byref(cons)), ctx)
    return float(used.value), _cons_dict(cons)


def sph_step_bins(ctx, parts: sph_particles, dt_max: float, n_bins: int):
    cons = sph_conserved()
    bs = sph_bin_stats()
    _check(lib().sph_step_bins(ctx, ctypes.byref(parts), float(dt_max), int(n_bins), ctypes.byref(cons),
                               ctypes.byref(bs)), ctx)
    stats = dict(substeps=int(bs.substeps), updates=int(bs.updates), cfl_over=int(bs.cfl_over),
                 bin_count=np.array(list(bs.bin_count), dtype=np.int64), limited=int(bs.limited),
                 woken=int(bs.woken), limit_sweeps=int(bs.limit_sweeps))
    return _cons_dict(cons), stats


def _cons_dict(c: sph_conserved) -> dict:
    return dict(momentum=np.array(list(c.momentum)), e_kin=c.e_kin, e_th=c.e_th,
                e_tot=c.e_kin + c.e_th, dt_next=c.dt_next, u_floors=int(c.u_floors))


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def sph_hpredict_init(ctx, seed: int = 1) -> int:
    return _check(lib().sph_hpredict_init(ctx, int(seed)), ctx)


def sph_hpredict_load(ctx, w_bf16: np.ndarray, f32: np.ndarray) -> int:
    w = np.ascontiguousarray(w_bf16, dtype=np.uint16)
    f = np.ascontiguousarray(f32, dtype=np.float32)
    assert w.size == SPH_HP_NBF16 and f.size == SPH_HP_NF32
    return _check(lib().sph_hpredict_load(ctx, w.ctypes.data_as(ctypes.c_void_p),
                                          f.ctypes.data_as(ctypes.c_void_p)), ctx)


def sph_hpredict_save(ctx):
    w = np.zeros(SPH_HP_NBF16, np.uint16)
    f = np.zeros(SPH_HP_NF32, np.float32)
    _check(lib().sph_hpredict_save(ctx, w.ctypes.data_as(ctypes.c_void_p), f.ctypes.data_as(ctypes.c_void_p)), ctx)
    return w, f


def sph_hpredict_params(ctx) -> np.ndarray:
    p = np.zeros(SPH_HP_NPARAM, np.float32)
    _check(lib().sph_hpredict_params(ctx, p.ctypes.data_as(ctypes.c_void_p)), ctx)
    return p


def sph_hpredict_features(ctx, parts: sph_particles, dt: float, feats) -> int:
    return _check(lib().sph_hpredict_features(ctx, ctypes.byref(parts), float(dt),
                                              _ptr(feats) if feats is not None else None), ctx)


def sph_hpredict_targets(ctx, parts: sph_particles, target) -> int:
    return _check(lib().sph_hpredict_targets(ctx, ctypes.byref(parts), _ptr(target)), ctx)


def sph_hpredict_eval(ctx, feats, n: int, out) -> int:
    return _check(lib().sph_hpredict_eval(ctx, _ptr(feats), int(n), _ptr(out)), ctx)


def sph_hpredict_train(ctx, feats, target, n: int, epochs: int, lr: float, seed: int = 0) -> float:
    loss = ctypes.c_float(0)
    _check(lib().sph_hpredict_train(ctx, _ptr(feats), _ptr(target), int(n), int(epochs), float(lr), int(seed),
                                    ctypes.byref(loss)), ctx)
    return float(loss.value)


def sph_hpredict_collect(ctx, feats, target, capacity: int) -> int:
    return _check(lib().sph_hpredict_collect(ctx, _ptr(feats) if feats is not None else None,
                                             _ptr(target) if target is not None else None, int(capacity)), ctx)


def sph_gravity_p2p(ctx, G: float, eps: float, ax, ay, az, phi=None) -> int:
    return _check(lib().sph_gravity_p2p(ctx, float(G), float(eps), _ptr(ax), _ptr(ay), _ptr(az),
                                        _ptr(phi) if phi is not None else None), ctx)


def sph_fp32_peak(stream: int | None = None, iters: int = 1 << 15, reps: int = 3) -> tuple[float, float]:
    """Measured FP32 FMA throughput of the current device: (TFLOP/s, ms of the
    fastest launch)."""
    tf = ctypes.c_double(0)
    ms = ctypes.c_float(0)
    _check(lib().sph_fp32_peak(ctypes.c_void_p(stream or 0), int(iters), int(reps), ctypes.byref(tf),
                               ctypes.byref(ms)))
    return float(tf.value), float(ms.value)


def sph_get_stats(ctx) -> dict:
    s = sph_stats()
    _check(lib().sph_get_stats(ctx, ctypes.byref(s)), ctx)
    return {k: getattr(s, k) for k, _ in sph_stats._fields_}


def sph_reset_stats(ctx) -> int:
    return _check(lib().sph_reset_stats(ctx), ctx)


def sph_destroy(ctx) -> None:
    if ctx:
        lib().sph_destroy(ctx)


# ------------------------------------------------------------ conveniences


class Particles:
    """Caller-owned device SoA (torch CUDA tensors) in the layout of sph_particles."""

    F64 = ("x", "y", "z", "vx", "vy", "vz")
    F32 = ("m", "u", "h", "rho", "P", "c", "f", "divv", "curl", "ax", "ay", "az", "dudt", "vsig")

    def __init__(self, d: dict, device: str = "cuda", pin: bool = False):
        import torch
        n = int(np.asarray(d["x"]).size)
        self.n = n
        self.t = {}
        for k in self.F64:
            self.t[k] = self._mk(d.get(k), n, torch.float64, device, pin)
        for k in self.F32:
            self.t[k] = self._mk(d.get(k), n, torch.float32, device, pin)
        self.t["n_ngb"] = self._mk(d.get("n_ngb"), n, torch.int32, device, pin)

    @staticmethod
    def _mk(v, n, dtype, device, pin):
        import torch
        if device == "cpu":
            t = torch.zeros(n, dtype=dtype, pin_memory=pin)
            if v is not None:
                t.copy_(torch.as_tensor(np.asarray(v)).to(dtype))
            return t
        if v is None:
            return torch.zeros(n, dtype=dtype, device=device)
        return torch.as_tensor(np.asarray(v)).to(dtype).to(device)

    def struct(self) -> sph_particles:
        p = sph_particles()
        for k in _PFIELDS:
            setattr(p, k, ctypes.c_void_p(self.t[k].data_ptr()))
        return p

    def numpy(self) -> dict:
        return {k: v.detach().cpu().numpy() for k, v in self.t.items()}


class Context:
    """Owns an sph_ctx; methods mirror the C entry points."""

    def __init__(self, n: int, device: int = 0, stream=None, box_offsets=None, **overrides):
        import torch
        self.params = sph_default_params()
        self.params.n = int(n)
        for k, v in overrides.items():
            setattr(self.params, k, v)
        self._offs = None
        if box_offsets is not None and len(box_offsets) > 2:
            self._offs = (ctypes.c_int64 * len(box_offsets))(*[int(v) for v in box_offsets])
            self.params.n_boxes = len(box_offsets) - 1
            self.params.box_offsets = ctypes.cast(self._offs, ctypes.c_void_p)
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.stream = stream
        self.h = sph_init(self.params, device, stream)

    def build_cells(self, parts: Particles):
        self._p = parts.struct()
        return sph_build_cells(self.h, self._p)

    def density(self, parts: Particles, allow_not_converged=False) -> int:
        return sph_density(self.h, parts.struct(), allow_not_converged)

    def force(self, parts: Particles):
        return sph_force(self.h, parts.struct())

    def step(self, parts: Particles, dt: float = 0.0, allow=()):
        """One KDK step; `allow`: statuses returned instead of raised (the step
        completes under SPH_ERR_NOT_CONVERGED and SPH_ERR_PRECISION)."""
        return sph_step(self.h, parts.struct(), dt, allow)

    def steps(self, parts: Particles, n_steps: int, dt: float = 0.0, allow=()):
        return sph_steps(self.h, parts.struct(), n_steps, dt, allow)

    def step_bins(self, parts: Particles, dt_max: float, n_bins: int):
        """Individual time-steps over dt_max: (conserved dict, bin stats dict)."""
        return sph_step_bins(self.h, parts.struct(), dt_max, n_bins)

    def bins(self) -> np.ndarray:
        import torch
        n = int(self.params.n)
        t = torch.empty(max(n, 1), dtype=torch.int8, device="cuda")
        _check(lib().sph_get_bins(self.h, ctypes.c_void_p(t.data_ptr())), self.h)
        torch.cuda.synchronize()
        return t[:n].cpu().numpy()

    def step_host(self, parts: Particles, dt: float = 0.0):
        return sph_step_host(self.h, parts.struct(), dt)

    def gravity(self, G: float = 1.0, eps: float = 0.0, out=None, with_phi: bool = True):
        """Near-field gravity on the current cells (sph_gravity_p2p) into device
        tensors (a dict ax, ay, az, phi of FP32 CUDA tensors, allocated if None);
        returns that dict."""
        import torch
        n = int(self.params.n)
        if out is None:
            out = {k: torch.zeros(max(n, 1), dtype=torch.float32, device="cuda") for k in ("ax", "ay", "az", "phi")}
        sph_gravity_p2p(self.h, G, eps, out["ax"], out["ay"], out["az"], out["phi"] if with_phi else None)
        return out

    def permutation(self) -> np.ndarray:
        import torch
        n = int(self.params.n)
        t = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        _check(lib().sph_get_permutation(self.h, ctypes.c_void_p(t.data_ptr())), self.h)
        torch.cuda.synchronize()
        return t[:n].cpu().numpy()

    def cell_keys(self) -> np.ndarray:
        import torch
        n = int(self.params.n)
        t = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        _check(lib().sph_get_cell_keys(self.h, ctypes.c_void_p(t.data_ptr())), self.h)
        torch.cuda.synchronize()
        return t[:n].cpu().numpy()

    def ngb_hash(self) -> np.ndarray:
        import torch
        n = int(self.params.n)
        t = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        _check(lib().sph_get_ngb_hash(self.h, ctypes.c_void_p(t.data_ptr())), self.h)
        torch.cuda.synchronize()
        return t[:n].cpu().numpy().view(np.uint64)

    # learned initial h (device tensors in, device tensors out)
    def hp_init(self, seed: int = 1):
        return sph_hpredict_init(self.h, seed)

    def hp_load(self, w_bf16, f32):
        return sph_hpredict_load(self.h, w_bf16, f32)

    def hp_save(self):
        return sph_hpredict_save(self.h)

    def hp_params(self) -> np.ndarray:
        return sph_hpredict_params(self.h)

    def hp_features(self, parts: Particles, dt: float):
        import torch
        f = torch.empty((max(parts.n, 1), 6), dtype=torch.float32, device="cuda")
        sph_hpredict_features(self.h, parts.struct(), dt, f)
        return f[: parts.n]

    def hp_targets(self, parts: Particles):
        import torch
        t = torch.empty(max(parts.n, 1), dtype=torch.float32, device="cuda")
        sph_hpredict_targets(self.h, parts.struct(), t)
        return t[: parts.n]

    def hp_eval(self, feats):
        import torch
        n = int(feats.shape[0])
        out = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
        sph_hpredict_eval(self.h, feats.contiguous(), n, out)
        return out[:n]

    def hp_train(self, feats, target, epochs: int = 1, lr: float = 1e-3, seed: int = 0) -> float:
        return sph_hpredict_train(self.h, feats.contiguous(), target.contiguous(), int(target.shape[0]), epochs,
                                  lr, seed)

    def hp_collect(self, feats, target, capacity: int):
        self._hp_bufs = (feats, target)  # keep the buffers alive while collecting
        return sph_hpredict_collect(self.h, feats, target, capacity)

    def stats(self) -> dict:
        return sph_get_stats(self.h)

    def reset_stats(self):
        return sph_reset_stats(self.h)

    def last_error(self) -> str:
        return lib().sph_last_error(self.h).decode()

    def close(self):
        if self.h:
            sph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
