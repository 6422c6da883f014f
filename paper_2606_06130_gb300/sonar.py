"""Thin ctypes binding of libsonar.so (the C ABI declared in include/sonar.h).

Argument marshalling only: every step of the echo-formation path runs in the library's
CUDA kernels. PyTorch provides device memory and streams. The library must have been
built (``__graft_entry__.build()`` or ``python -m paper_2606_06130_gb300.build``);
loading fails loudly otherwise, there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

SONAR_OK = 0
SONAR_E_ARG = -1
SONAR_E_NOMEM = -2
SONAR_E_CUDA = -3
SONAR_E_CAPACITY = -4
SONAR_E_TIMEOUT = -5
SONAR_E_NOSCENE = -6
SONAR_E_UNSUPPORTED = -7

SONAR_FP32 = 0
SONAR_BF16 = 1
SONAR_FP16 = 2

SONAR_OPT_DEBUG = 1
SONAR_OPT_TIMING = 2
SONAR_OPT_GRAPH = 3
SONAR_OPT_TILE_N = 4
SONAR_OPT_SYNTH = 5
SONAR_OPT_RAW = 6
SONAR_OPT_BVH = 7
SONAR_OPT_CROSS = 8
SONAR_OPT_AUTOTUNE = 9
SONAR_OPT_TRAVERSAL = 10
SONAR_OPT_TTD = 11
SONAR_OPT_GEMM_CLUSTER = 12
SONAR_OPT_BEAMFORM = 13

SONAR_SUR_N_PARAMS = 150657

PRECISIONS = {"fp32": SONAR_FP32, "bf16": SONAR_BF16, "fp16": SONAR_FP16}


class sonar_pose(C.Structure):
    _fields_ = [("t", C.c_double * 3), ("q", C.c_double * 4)]


class sonar_ssp(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("z", C.POINTER(C.c_double)), ("c", C.POINTER(C.c_double))]


class sonar_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("pitch_m", C.c_double), ("f0_hz", C.c_double),
                ("bw_hz", C.c_double), ("pulse_s", C.c_double), ("c_ref", C.c_double),
                ("hfov_rad", C.c_double), ("vfov_rad", C.c_double), ("n_beam_az", C.c_int32),
                ("n_beam_el", C.c_int32), ("n_range", C.c_int32), ("r_min_m", C.c_double),
                ("r_max_m", C.c_double), ("r_blank_m", C.c_double), ("n_ray_az", C.c_int32),
                ("n_ray_el", C.c_int32), ("n_sub", C.c_int32), ("max_bounces", C.c_int32),
                ("surface_z", C.c_double), ("r_surface", C.c_double), ("r_seabed", C.c_double),
                ("alpha_np_per_m", C.c_double), ("seed", C.c_uint64), ("precision", C.c_int32),
                ("thr_mode", C.c_int32), ("thr", C.c_double), ("taper", C.POINTER(C.c_float))]


class sonar_volume(C.Structure):
    _fields_ = [("n", C.c_int64), ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("s_v", C.c_double)]


class sonar_field(C.Structure):
    _fields_ = [("nx", C.c_int32), ("nz", C.c_int32), ("x0", C.c_double), ("dx", C.c_double), ("z0", C.c_double),
                ("dz", C.c_double), ("c", C.POINTER(C.c_double)), ("step_m", C.c_double)]


class sonar_point(C.Structure):
    _fields_ = [("x", C.c_float), ("y", C.c_float), ("z", C.c_float), ("intensity", C.c_float),
                ("beam", C.c_int32), ("bin", C.c_int32)]


class sonar_hit(C.Structure):
    _fields_ = [("key", C.c_uint32), ("prim", C.c_int32), ("tau", C.c_double), ("amp", C.c_float),
                ("phi", C.c_float), ("uy", C.c_float), ("uz", C.c_float)]


class sonar_stats(C.Structure):
    _fields_ = [("n_hits", C.c_int64), ("hit_capacity", C.c_int64), ("n_pings", C.c_int32),
                ("taps", C.c_int32), ("kernels", C.c_int32), ("ms_trace", C.c_float), ("ms_bin", C.c_float),
                ("ms_synth", C.c_float), ("ms_convert", C.c_float), ("ms_beamform", C.c_float),
                ("ms_peaks", C.c_float), ("tile_n", C.c_int32), ("synth_cols", C.c_int32), ("autotuned", C.c_int32),
                ("synth_mma_flop", C.c_double), ("gemm_cluster", C.c_int32),
                ("beam_sep", C.c_int32)]


class sonar_sur_metrics(C.Structure):
    _fields_ = [("nl2", C.c_double), ("lit_beams", C.c_int64), ("peak_bin_mean", C.c_double),
                ("peak_within_1", C.c_double), ("peak_within_4", C.c_double), ("cells", C.c_int64),
                ("si", C.c_double), ("si_ref", C.c_double)]


POINT_DTYPE = np.dtype([("x", "<f4"), ("y", "<f4"), ("z", "<f4"), ("intensity", "<f4"),
                        ("beam", "<i4"), ("bin", "<i4")])
HIT_DTYPE = np.dtype([("key", "<u4"), ("prim", "<i4"), ("tau", "<f8"), ("amp", "<f4"), ("phi", "<f4"),
                      ("uy", "<f4"), ("uz", "<f4")])

_lib = None

# name -> (restype, argtypes); the same names as include/sonar.h
_SIGS = {
    "sonar_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "sonar_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sonar_destroy": (C.c_int, [C.c_void_p]),
    "sonar_last_error": (C.c_char_p, [C.c_void_p]),
    "sonar_set_option": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64]),
    "sonar_set_volume": (C.c_int, [C.c_void_p, C.POINTER(sonar_volume)]),
    "sonar_set_field": (C.c_int, [C.c_void_p, C.POINTER(sonar_field)]),
    "sonar_scene_upload": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64]),
    "sonar_ping": (C.c_int, [C.c_void_p, C.POINTER(sonar_pose), C.POINTER(sonar_params), C.POINTER(sonar_ssp),
                             C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "sonar_ping_batch": (C.c_int, [C.c_void_p, C.POINTER(sonar_pose), C.c_int32, C.POINTER(sonar_params),
                                   C.POINTER(sonar_ssp), C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "sonar_ping_async": (C.c_int, [C.c_void_p, C.POINTER(sonar_pose), C.c_int32, C.POINTER(sonar_params),
                                   C.POINTER(sonar_ssp), C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "sonar_wait": (C.c_int, [C.c_void_p]),
    "sonar_probe_wait_limit": (C.c_int, [C.c_void_p, C.c_int64]),
    "sonar_get_hits": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    "sonar_get_echoes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "sonar_get_raw": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64]),
    "sonar_get_stats": (C.c_int, [C.c_void_p, C.POINTER(sonar_stats)]),
    "sonar_sur_set_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double]),
    "sonar_sur_get_weights": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "sonar_sur_render": (C.c_int, [C.c_void_p, C.POINTER(sonar_pose), C.c_int32, C.POINTER(sonar_params),
                                   C.POINTER(sonar_ssp), C.c_void_p]),
    "sonar_sur_ping": (C.c_int, [C.c_void_p, C.POINTER(sonar_pose), C.c_int32, C.POINTER(sonar_params),
                                 C.POINTER(sonar_ssp), C.c_void_p]),
    "sonar_sur_geometric": (C.c_int, [C.c_void_p, C.POINTER(sonar_pose), C.c_int32, C.POINTER(sonar_params),
                                      C.POINTER(sonar_ssp), C.c_void_p]),
    "sonar_sur_train_step": (C.c_int, [C.c_void_p, C.POINTER(sonar_pose), C.c_int32, C.POINTER(sonar_params),
                                       C.POINTER(sonar_ssp), C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_int32,
                                       C.POINTER(C.c_double), C.c_void_p]),
    "sonar_sur_compare": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(sonar_params),
                                    C.c_double, C.POINTER(sonar_sur_metrics)]),
    "sonar_cloud_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(sonar_params), C.POINTER(sonar_pose),
                                      C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p]),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """Loads libsonar.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(the echo-formation path has no CPU fallback)")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class SonarError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sonar error {code}: {msg}")
        self.code = code


# ------------------------------------------------------------------ marshalling helpers
_PARAM_MAP = {"pitch": "pitch_m", "f0": "f0_hz", "bw": "bw_hz", "pulse": "pulse_s", "hfov": "hfov_rad",
              "vfov": "vfov_rad", "r_min": "r_min_m", "r_max": "r_max_m", "r_blank": "r_blank_m",
              "alpha": "alpha_np_per_m"}


def make_params(p: dict, precision="fp32", taper=None) -> sonar_params:
    """sonar_params from a parameter dict (input-generator names or sonar.h names)."""
    sp = sonar_params()
    for k, v in p.items():
        name = _PARAM_MAP.get(k, k)
        if name in ("taper", "precision"):
            continue
        if name == "surface_z" and v is None:
            v = math.nan
        setattr(sp, name, v)
    prec = p.get("precision", precision)
    sp.precision = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    if taper is not None:
        arr = np.ascontiguousarray(taper, np.float32)
        sp._taper_keep = arr
        sp.taper = arr.ctypes.data_as(C.POINTER(C.c_float))
    return sp


def make_pose(pose: dict) -> sonar_pose:
    return sonar_pose((C.c_double * 3)(*map(float, pose["t"])), (C.c_double * 4)(*map(float, pose["q"])))


def make_ssp(ssp: dict) -> sonar_ssp:
    z = np.ascontiguousarray(ssp.get("z", []), np.float64)
    c = np.ascontiguousarray(ssp.get("c", []), np.float64)
    s = sonar_ssp(len(c), z.ctypes.data_as(C.POINTER(C.c_double)) if len(z) else None,
                  c.ctypes.data_as(C.POINTER(C.c_double)) if len(c) else None)
    s._keep = (z, c)
    return s


def _ptr(x):
    """Address of a torch tensor or numpy array (device or host)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


class Sonar:
    """One library context on one CUDA device; a convenience wrapper over the C ABI."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.device = device
        self.h = C.c_void_p()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        rc = lib().sonar_create(C.byref(self.h), device, C.c_void_p(stream.cuda_stream))
        if rc != SONAR_OK:
            raise SonarError(rc, "sonar_create failed (an sm_103 GPU is required)")
        self._pending = []  # point-count arrays of asynchronous calls not yet retired

    def close(self):
        if self.h:
            lib().sonar_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != SONAR_OK:
            raise SonarError(rc, lib().sonar_last_error(self.h).decode())

    def set_option(self, option: int, value: int):
        self._check(lib().sonar_set_option(self.h, option, int(value)))

    def set_volume(self, n: int, lo=(0.0, 0.0, 0.0), hi=(0.0, 0.0, 0.0), s_v: float = 0.0):
        """Water-column scatterers of the following pings (n = 0: none)."""
        v = sonar_volume(int(n), (C.c_double * 3)(*map(float, lo)), (C.c_double * 3)(*map(float, hi)), float(s_v))
        self._check(lib().sonar_set_volume(self.h, C.byref(v)))

    def set_field(self, field: dict | None):
        """Range-dependent sound speed of the following pings: {"x0", "dx", "z0", "dz",
        "c": [nz][nx] m/s, "h": integration step in m}, or None to remove it."""
        if field is None:
            self._check(lib().sonar_set_field(self.h, None))
            return
        c = np.ascontiguousarray(field["c"], np.float64)
        f = sonar_field(c.shape[1], c.shape[0], float(field["x0"]), float(field["dx"]), float(field["z0"]),
                        float(field["dz"]), c.ctypes.data_as(C.POINTER(C.c_double)), float(field["h"]))
        self._check(lib().sonar_set_field(self.h, C.byref(f)))

    def upload(self, scene):
        v = np.ascontiguousarray(scene.verts, np.float32)
        t = np.ascontiguousarray(scene.tris, np.int32)
        mu = np.ascontiguousarray(scene.mu, np.float32)
        fl = np.ascontiguousarray(scene.flags, np.uint8)
        pts = np.ascontiguousarray(scene.points, np.float32).reshape(-1, 3)
        sg = np.ascontiguousarray(scene.sigma, np.float32)
        pl = np.ascontiguousarray(scene.planes, np.float64).reshape(-1, 4)
        self._check(lib().sonar_scene_upload(self.h, _ptr(v) if len(v) else None, len(v), _ptr(t) if len(t) else None,
                                             len(t), _ptr(mu) if len(mu) else None, _ptr(fl) if len(fl) else None,
                                             _ptr(pts) if len(pts) else None, _ptr(sg) if len(sg) else None, len(pts),
                                             _ptr(pl) if len(pl) else None, len(pl)))

    def ping_batch(self, poses, params: dict, ssp: dict, precision="fp32", taper=None, env=None, cloud=None,
                   cloud_cap: int | None = None):
        """Returns (env, cloud, n_cloud). env/cloud default to new device tensors."""
        torch = self.torch
        P = len(poses)
        nb = params["n_beam_az"] * params["n_beam_el"]
        if cloud_cap is None:
            cloud_cap = nb
        if env is None:
            env = torch.empty((P, params["n_beam_el"], params["n_beam_az"], params["n_range"]),
                              dtype=torch.float32, device=f"cuda:{self.device}")
        if cloud is None:
            cloud = torch.empty((P, cloud_cap, 6), dtype=torch.int32, device=f"cuda:{self.device}")
        arr = (sonar_pose * P)(*[make_pose(p) for p in poses])
        sp = make_params(params, precision, taper)
        ss = make_ssp(ssp)
        n = (C.c_int64 * P)()
        self._check(lib().sonar_ping_batch(self.h, arr, P, C.byref(sp), C.byref(ss), _ptr(env), _ptr(cloud),
                                           cloud_cap, n))
        return env, cloud, np.array(n[:], np.int64)

    def ping_async(self, poses, params: dict, ssp: dict, precision="fp32", taper=None, env=None, cloud=None,
                   cloud_cap: int | None = None):
        """Enqueues the pings without waiting (sonar_ping_async). env/cloud: device tensors
        or pinned host tensors (default: new device tensors). Returns (env, cloud, n_cloud);
        they are complete once the call is retired: by the second following ping_async,
        by wait(), or by any other call on this context."""
        torch = self.torch
        P = len(poses)
        nb = params["n_beam_az"] * params["n_beam_el"]
        if cloud_cap is None:
            cloud_cap = nb
        if env is None:
            env = torch.empty((P, params["n_beam_el"], params["n_beam_az"], params["n_range"]),
                              dtype=torch.float32, device=f"cuda:{self.device}")
        if cloud is None:
            cloud = torch.empty((P, cloud_cap, 6), dtype=torch.int32, device=f"cuda:{self.device}")
        arr = (sonar_pose * P)(*[make_pose(p) for p in poses])
        sp = make_params(params, precision, taper)
        ss = make_ssp(ssp)
        n = np.zeros(P, np.int64)
        self._pending.append(n)
        try:
            self._check(lib().sonar_ping_async(self.h, arr, P, C.byref(sp), C.byref(ss), _ptr(env), _ptr(cloud),
                                               cloud_cap, n.ctypes.data_as(C.POINTER(C.c_int64))))
        finally:
            # the call retired the one made two calls earlier; its count array is final
            del self._pending[:-2]
        return env, cloud, n

    def wait(self):
        """Retires every asynchronous call in flight (sonar_wait)."""
        try:
            self._check(lib().sonar_wait(self.h))
        finally:
            self._pending.clear()

    def probe_wait_limit(self, limit_cycles: int) -> int:
        """One bounded device-side wait that nothing completes (sonar_probe_wait_limit).
        Returns the status code: SONAR_E_TIMEOUT when the wait gave up at its limit."""
        self._pending.clear()
        return int(lib().sonar_probe_wait_limit(self.h, int(limit_cycles)))

    def ping(self, pose, params: dict, ssp: dict, **kw):
        env, cloud, n = self.ping_batch([pose], params, ssp, **kw)
        return env[0], cloud[0], int(n[0])

    def hits(self) -> np.ndarray:
        n = C.c_int64()
        lib().sonar_get_hits(self.h, None, 0, C.byref(n))
        out = np.zeros(int(n.value), HIT_DTYPE)
        self._check(lib().sonar_get_hits(self.h, out.ctypes.data if len(out) else None, len(out), C.byref(n)))
        return out

    def echoes(self, params: dict, n_pings: int = 1) -> np.ndarray:
        M = params["nx"] * params["ny"]
        out = np.zeros((n_pings, params["n_range"], M, 2), np.float32)
        self._check(lib().sonar_get_echoes(self.h, out.ctypes.data, out.size))
        return out[..., 0] + 1j * out[..., 1]

    def raw(self, params: dict, phase: int, n_pings: int = 1) -> np.ndarray:
        """Raw element series of the last call at phase s (samples t_n + s dt / U); after a
        true-time-delay ping, the wideband element echoes at that phase."""
        M = params["nx"] * params["ny"]
        out = np.zeros((n_pings, params["n_range"], M, 2), np.float32)
        self._check(lib().sonar_get_raw(self.h, phase, out.ctypes.data, out.size))
        return out[..., 0] + 1j * out[..., 1]

    # ------------------------------------------------------------ learned surrogate
    def sur_set_weights(self, params, e_scale: float):
        """Network parameters (SONAR_SUR_N_PARAMS floats) and output scale; resets Adam."""
        a = np.ascontiguousarray(params, np.float32)
        self._check(lib().sonar_sur_set_weights(self.h, a.ctypes.data, a.size, float(e_scale)))

    def sur_get_weights(self) -> np.ndarray:
        out = np.zeros(SONAR_SUR_N_PARAMS, np.float32)
        self._check(lib().sonar_sur_get_weights(self.h, out.ctypes.data, out.size))
        return out

    def sur_render(self, poses, params: dict, ssp: dict) -> np.ndarray:
        """Beam-centre geometric rendering: [P, beams, 8] (L, kappa, mu, Gamma of two hits)."""
        P = len(poses)
        nb = params["n_beam_az"] * params["n_beam_el"]
        out = np.zeros((P, nb, 8), np.float32)
        arr = (sonar_pose * P)(*[make_pose(p) for p in poses])
        sp, ss = make_params(params), make_ssp(ssp)
        self._check(lib().sonar_sur_render(self.h, arr, P, C.byref(sp), C.byref(ss), out.ctypes.data))
        return out

    def sur_ping(self, poses, params: dict, ssp: dict, env=None):
        """The surrogate's envelope volumes [P, n_beam_el, n_beam_az, n_range] (device tensor)."""
        torch = self.torch
        P = len(poses)
        if env is None:
            env = torch.empty((P, params["n_beam_el"], params["n_beam_az"], params["n_range"]), dtype=torch.float32,
                              device=f"cuda:{self.device}")
        arr = (sonar_pose * P)(*[make_pose(p) for p in poses])
        sp, ss = make_params(params), make_ssp(ssp)
        self._check(lib().sonar_sur_ping(self.h, arr, P, C.byref(sp), C.byref(ss), _ptr(env)))
        return env

    def sur_geometric(self, poses, params: dict, ssp: dict, env=None):
        """Envelope of the geometric rendering without the network (device tensor)."""
        torch = self.torch
        P = len(poses)
        if env is None:
            env = torch.empty((P, params["n_beam_el"], params["n_beam_az"], params["n_range"]), dtype=torch.float32,
                              device=f"cuda:{self.device}")
        arr = (sonar_pose * P)(*[make_pose(p) for p in poses])
        sp, ss = make_params(params), make_ssp(ssp)
        self._check(lib().sonar_sur_geometric(self.h, arr, P, C.byref(sp), C.byref(ss), _ptr(env)))
        return env

    def sur_train_step(self, poses, params: dict, ssp: dict, target, beams=None, lr: float = 1e-3,
                       update: bool = True, want_grad: bool = False):
        """One training step against device envelopes `target` of the same poses; beams: a
        device int32 tensor of selected beam indices (None: all). Returns (loss, grad)."""
        P = len(poses)
        arr = (sonar_pose * P)(*[make_pose(p) for p in poses])
        sp, ss = make_params(params), make_ssp(ssp)
        loss = C.c_double()
        grad = np.zeros(SONAR_SUR_N_PARAMS, np.float32) if want_grad else None
        n_sel = 0 if beams is None else int(beams.numel())
        self._check(lib().sonar_sur_train_step(self.h, arr, P, C.byref(sp), C.byref(ss), _ptr(target), _ptr(beams),
                                               n_sel, float(lr), 1 if update else 0, C.byref(loss),
                                               grad.ctypes.data if want_grad else None))
        return loss.value, grad

    def sur_compare(self, env, ref, params: dict, rel_thr: float = 0.1) -> dict:
        """Metrics of envelope volumes env against ref (device tensors of the same shape)."""
        m = sonar_sur_metrics()
        P = int(env.shape[0]) if env.dim() == 4 else 1
        sp = make_params(params)
        self._check(lib().sonar_sur_compare(self.h, _ptr(env), _ptr(ref), P, C.byref(sp), float(rel_thr), C.byref(m)))
        return {k: getattr(m, k) for k, _ in sonar_sur_metrics._fields_}

    def stats(self) -> dict:
        s = sonar_stats()
        self._check(lib().sonar_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in sonar_stats._fields_}


def cloud_records(cloud, n: int) -> np.ndarray:
    """Device or host cloud buffer [cap, 6] (int32 view) -> structured points."""
    a = cloud.cpu().numpy() if hasattr(cloud, "cpu") else np.asarray(cloud)
    return np.ascontiguousarray(a[:n]).view(POINT_DTYPE).reshape(-1)
