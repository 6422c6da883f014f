"""FP64 CPU oracle for per-ping coherent echo formation (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may
import this package. It wraps oracle/sonar_oracle.c (built with gcc by oracle/build.py)
through ctypes; it imports nothing from the CUDA product package, and the product
package imports nothing from here. Inputs are plain numpy arrays and dicts as produced
by the seeded input generators.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

_lib = None


class OrcParams(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("pitch", C.c_double), ("f0", C.c_double),
                ("bw", C.c_double), ("pulse", C.c_double), ("c_ref", C.c_double),
                ("hfov", C.c_double), ("vfov", C.c_double), ("n_beam_az", C.c_int32),
                ("n_beam_el", C.c_int32), ("n_range", C.c_int32), ("r_min", C.c_double),
                ("r_max", C.c_double), ("r_blank", C.c_double), ("n_ray_az", C.c_int32),
                ("n_ray_el", C.c_int32), ("n_sub", C.c_int32), ("max_bounces", C.c_int32),
                ("surface_z", C.c_double), ("r_surface", C.c_double), ("r_seabed", C.c_double),
                ("alpha", C.c_double), ("seed", C.c_uint64), ("thr_mode", C.c_int32),
                ("thr", C.c_double), ("cross", C.c_int32), ("vol_n", C.c_int64),
                ("vol_lo", C.c_double * 3), ("vol_hi", C.c_double * 3), ("vol_sv", C.c_double),
                ("fld_nx", C.c_int32), ("fld_nz", C.c_int32), ("fld_x0", C.c_double), ("fld_dx", C.c_double),
                ("fld_z0", C.c_double), ("fld_dz", C.c_double), ("fld_c", C.c_void_p), ("fld_h", C.c_double)]


_PARAM_DEFAULTS = {"cross": 0, "vol_n": 0, "vol_lo": (0.0, 0.0, 0.0), "vol_hi": (0.0, 0.0, 0.0), "vol_sv": 0.0}


class OrcScene(C.Structure):
    _fields_ = [("n_verts", C.c_int64), ("verts", C.c_void_p), ("n_tris", C.c_int64),
                ("tris", C.c_void_p), ("mu", C.c_void_p), ("flags", C.c_void_p),
                ("n_points", C.c_int64), ("points", C.c_void_p), ("sigma", C.c_void_p),
                ("n_planes", C.c_int64), ("planes", C.c_void_p)]


_HIT_I32 = ("ray", "sub", "seg", "prim")
_HIT_F64 = ("tau", "len", "amp", "psi", "phi", "ux", "uy", "uz", "cr", "ci", "margin", "gap", "kinc", "gam")


class OrcHits(C.Structure):
    _fields_ = ([("cap", C.c_int64), ("n", C.c_int64)]
                + [(k, C.c_void_p) for k in _HIT_I32] + [(k, C.c_void_p) for k in _HIT_F64]
                + [("c_ref", C.c_double)])


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        _lib.orc_trace.argtypes = [vp, vp, vp, vp, vp, vp, i32, C.c_int, vp]
        _lib.orc_synth.argtypes = [vp, vp, vp, i64, vp]
        _lib.orc_raw.argtypes = [vp, vp, i32, i32, vp, i64, vp]
        _lib.orc_pulse.argtypes = [d, d, d, vp, vp]
        _lib.orc_beamform.argtypes = [vp, d, vp, vp, i64, vp, i64, vp]
        _lib.orc_synth_wb.argtypes = [vp, vp, d, vp, i64, vp]
        _lib.orc_ttd.argtypes = [vp, vp, vp, vp, i64, vp, i64, vp]
        _lib.orc_envelope.argtypes = [vp, vp, vp, i64, i64, vp]
        _lib.orc_peaks.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        _lib.orc_peaks.restype = i64
        _lib.orc_pulse_acf.argtypes = [d, d, d, vp, vp]
        _lib.orc_pcg4d.argtypes = [vp]
        _lib.orc_closest_hit.argtypes = [vp, vp, vp, d, d, i32, C.c_int, vp, vp, vp]
        _lib.orc_field_ray.argtypes = [vp, vp, vp, d, i32, vp]
        _lib.orc_closest_hit.restype = i32
        _lib.orc_arc_nodes.argtypes = [vp, vp, i32, vp, vp, d, i32, vp, vp, vp]
        _lib.orc_eigen_arc.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp]
        _lib.orc_eigen_arc.restype = C.c_int
        _lib.orc_num_threads.restype = C.c_int
        _lib.orc_set_threads.argtypes = [C.c_int]
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None and a.size else None


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def make_params(p: dict) -> OrcParams:
    """OrcParams from a parameter dict. A range-dependent sound speed comes as
    p["field"] = {"x0", "dx", "z0", "dz", "c": [nz][nx] m/s, "h": RK4 step in m}."""
    o = OrcParams()
    fld = p.get("field")
    for name, _ in OrcParams._fields_:
        if name.startswith("fld_"):
            continue
        v = p.get(name, _PARAM_DEFAULTS[name]) if name in _PARAM_DEFAULTS else p[name]
        if name in ("vol_lo", "vol_hi"):
            v = (C.c_double * 3)(*[float(x) for x in v])
        if name == "surface_z" and v is None:
            v = math.nan
        setattr(o, name, v)
    if fld is not None:
        cf = np.ascontiguousarray(fld["c"], np.float64)
        o.fld_nz, o.fld_nx = cf.shape
        o.fld_x0, o.fld_dx, o.fld_z0, o.fld_dz = (float(fld[k]) for k in ("x0", "dx", "z0", "dz"))
        o.fld_h = float(fld["h"])
        o.fld_c = cf.ctypes.data
        o._keep = cf  # the grid must outlive the call
    return o


class _SceneHold:
    """Keeps the numpy arrays referenced by an OrcScene alive."""

    def __init__(self, sc):
        self.verts = np.ascontiguousarray(sc.verts, np.float32)
        self.tris = np.ascontiguousarray(sc.tris, np.int32)
        self.mu = np.ascontiguousarray(sc.mu, np.float32)
        self.flags = np.ascontiguousarray(sc.flags, np.uint8)
        self.points = np.ascontiguousarray(sc.points, np.float32).reshape(-1, 3)
        self.sigma = np.ascontiguousarray(sc.sigma, np.float32)
        self.planes = np.ascontiguousarray(sc.planes, np.float64).reshape(-1, 4)
        self.s = OrcScene(len(self.verts), _ptr(self.verts), len(self.tris), _ptr(self.tris),
                          _ptr(self.mu), _ptr(self.flags), len(self.points), _ptr(self.points),
                          _ptr(self.sigma), len(self.planes), _ptr(self.planes))


def field_ray(params: dict, o, d, h: float, n: int) -> np.ndarray:
    """n RK4 steps of the field-route integrator (Sec. II.A refraction in a 2-D field):
    (x, y, z, tx, ty, tz, T) after an arc length n h from o along d."""
    L = lib()
    op = make_params(params)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    out = np.zeros(7, np.float64)
    rc = L.orc_field_ray(C.byref(op), _ptr(o), _ptr(d), C.c_double(h), C.c_int32(n), _ptr(out))
    if rc != 0:
        raise RuntimeError(f"orc_field_ray failed with code {rc}")
    return out


def trace(scene, params: dict, pose: dict, ssp: dict, use_bvh: bool = True) -> dict:
    """Hit list of one ping (Sec. II.A ray casting + Sec. II.B per-hit backscatter)."""
    L = lib()
    sh = _SceneHold(scene)
    op = make_params(params)
    t = np.ascontiguousarray(pose["t"], np.float64)
    q = np.ascontiguousarray(pose["q"], np.float64)
    z = np.ascontiguousarray(ssp["z"], np.float64)
    c = np.ascontiguousarray(ssp["c"], np.float64)
    cap = 1 << 16
    while True:
        arrs = {k: np.zeros(cap, np.int32) for k in _HIT_I32}
        arrs.update({k: np.zeros(cap, np.float64) for k in _HIT_F64})
        h = OrcHits(cap, 0, *[_ptr(arrs[k]) for k in _HIT_I32], *[_ptr(arrs[k]) for k in _HIT_F64], 0.0)
        rc = L.orc_trace(C.byref(sh.s), C.byref(op), _ptr(t), _ptr(q), _ptr(z), _ptr(c), len(z),
                         1 if use_bvh else 0, C.byref(h))
        if rc < 0:
            cap = int(h.n) + 16
            continue
        if rc != 0:
            raise RuntimeError(f"orc_trace failed with code {rc}")
        n = int(h.n)
        out = {k: v[:n].copy() for k, v in arrs.items()}
        out["n"] = n
        out["c_ref"] = float(h.c_ref)
        return out


def _hits_struct(h: dict):
    keep = {k: np.ascontiguousarray(h[k], np.int32) for k in _HIT_I32}
    # kinc and gam are trace outputs only (nothing downstream reads them): hand-made
    # hit lists may leave them out
    keep.update({k: np.ascontiguousarray(h[k] if k in h else np.zeros(h["n"]), np.float64) for k in _HIT_F64})
    s = OrcHits(h["n"], h["n"], *[_ptr(keep[k]) for k in _HIT_I32],
                *[_ptr(keep[k]) for k in _HIT_F64], h["c_ref"])
    return s, keep


def synth(params: dict, hits: dict, ns) -> np.ndarray:
    """Element echoes s_m[n] for the requested samples: complex128 [len(ns), M]."""
    ns = np.ascontiguousarray(ns, np.int32)
    M = params["nx"] * params["ny"]
    out = np.zeros((len(ns), M, 2), np.float64)
    hs, keep = _hits_struct(hits)
    lib().orc_synth(C.byref(make_params(params)), C.byref(hs), _ptr(ns), len(ns), _ptr(out))
    return out[..., 0] + 1j * out[..., 1]


def beamform(params: dict, c_ref: float, s: np.ndarray, beams=None, taper=None) -> np.ndarray:
    """Beams B[b, i] for element echoes s [n_ns, M]: complex128 [n_beams, n_ns]."""
    nb = params["n_beam_az"] * params["n_beam_el"]
    beams = np.arange(nb, dtype=np.int32) if beams is None else np.ascontiguousarray(beams, np.int32)
    s = np.ascontiguousarray(s, np.complex128)
    sr = np.ascontiguousarray(np.stack([s.real, s.imag], -1))
    out = np.zeros((len(beams), s.shape[0], 2), np.float64)
    tp = None if taper is None else np.ascontiguousarray(taper, np.float32)
    lib().orc_beamform(C.byref(make_params(params)), c_ref, _ptr(tp), _ptr(sr), s.shape[0],
                       _ptr(beams), len(beams), _ptr(out))
    return out[..., 0] + 1j * out[..., 1]


def envelope(params: dict, B: np.ndarray, ns) -> np.ndarray:
    ns = np.ascontiguousarray(ns, np.int32)
    Br = np.ascontiguousarray(np.stack([B.real, B.imag], -1))
    out = np.zeros(B.shape, np.float64)
    lib().orc_envelope(C.byref(make_params(params)), _ptr(Br), _ptr(ns), len(ns), B.shape[0], _ptr(out))
    return out


def volume(params: dict, hits: dict, ns=None, beams=None, taper=None):
    """Envelope E[b, i] (and beams B, element echoes s) for the requested samples/beams."""
    ns = np.arange(params["n_range"], dtype=np.int32) if ns is None else np.asarray(ns, np.int32)
    s = synth(params, hits, ns)
    B = beamform(params, hits["c_ref"], s, beams, taper)
    E = envelope(params, B, ns)
    return E, B, s


def peaks(params: dict, pose: dict, E: np.ndarray) -> dict:
    """Point cloud from a full envelope volume E [Nb, Nr]."""
    E = np.ascontiguousarray(E, np.float64)
    nb = E.shape[0]
    pts = np.zeros((nb, 4), np.float64)
    pb = np.zeros(nb, np.int32)
    pn = np.zeros(nb, np.int32)
    t = np.ascontiguousarray(pose["t"], np.float64)
    q = np.ascontiguousarray(pose["q"], np.float64)
    n = lib().orc_peaks(C.byref(make_params(params)), _ptr(t), _ptr(q), _ptr(E), _ptr(pts), _ptr(pb), _ptr(pn))
    return {"xyzi": pts[:n], "beam": pb[:n], "bin": pn[:n]}


def raw_echoes(params: dict, hits: dict, U: int, ns) -> np.ndarray:
    """Raw element series r_m(t_n + s dt / U), s = 0..U-1, for the requested samples n (any
    integers, also outside [0, n_range)): complex128 [U, len(ns), M]. The echo before
    pulse compression (Sec. II.B time series)."""
    ns = np.ascontiguousarray(ns, np.int32)
    M = params["nx"] * params["ny"]
    hs, keep = _hits_struct(hits)
    out = np.zeros((U, len(ns), M, 2), np.float64)
    for s in range(U):
        lib().orc_raw(C.byref(make_params(params)), C.byref(hs), U, s, _ptr(ns), len(ns), _ptr(out[s]))
    return out[..., 0] + 1j * out[..., 1]


def matched_filter(params: dict, hits: dict, U: int, ns) -> np.ndarray:
    """Matched filter of the raw series (Sec. II.B): y_m(t_n) = (dt / (U E)) sum over the raw
    samples t_i = t_j + s dt / U of r_m(t_i) conj(p(t_i - t_n)), E = 3T/8 the pulse energy.
    A rectangle-rule quadrature of the correlation integral that defines R, so y tends to
    the compressed echoes s_m[n] as U grows. complex128 [len(ns), M]."""
    ns = np.asarray(ns, np.int64)
    T, B = params["pulse"], params["bw"]
    dt = 2.0 * (params["r_max"] - params["r_min"]) / params["n_range"] / hits["c_ref"]
    D = int(math.ceil(T / 2 / dt)) + 1
    d = np.arange(-D, D + 1)
    rows = np.unique((ns[:, None] + d[None, :]).ravel())
    raw = raw_echoes(params, hits, U, rows)
    idx = {int(r): i for i, r in enumerate(rows)}
    E = 3.0 * T / 8.0
    y = np.zeros((len(ns), params["nx"] * params["ny"]), np.complex128)
    for s in range(U):
        h = np.conj(pulse(d * dt + s * dt / U, T, B))
        for a, n in enumerate(ns):
            for k, dd in enumerate(d):
                if h[k] != 0:
                    y[a] += raw[s, idx[int(n + dd)]] * h[k]
    return y * (dt / (U * E))


def pulse(t, T: float, B: float) -> np.ndarray:
    """The transmitted pulse p(t) (Hann-windowed linear chirp, |t| <= T/2)."""
    t = np.atleast_1d(np.asarray(t, np.float64))
    out = np.zeros(t.shape, np.complex128)
    re, im = C.c_double(), C.c_double()
    for i, x in enumerate(t.ravel()):
        lib().orc_pulse(float(x), T, B, C.byref(re), C.byref(im))
        out.ravel()[i] = re.value + 1j * im.value
    return out


def pulse_acf(u, T: float, B: float) -> np.ndarray:
    u = np.atleast_1d(np.asarray(u, np.float64))
    out = np.zeros(u.shape, np.complex128)
    re, im = C.c_double(), C.c_double()
    for i, x in enumerate(u.ravel()):
        lib().orc_pulse_acf(float(x), T, B, C.byref(re), C.byref(im))
        out.ravel()[i] = re.value + 1j * im.value
    return out


def pcg4d(v) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(v, np.uint32).copy())
    lib().orc_pcg4d(_ptr(a))
    return a


def closest_hit(scene, o, d, tmin=1e-7, tmax=math.inf, exclude=-1, use_bvh=True):
    sh = _SceneHold(scene)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    t, m, t2 = C.c_double(), C.c_double(), C.c_double()
    prim = lib().orc_closest_hit(C.byref(sh.s), _ptr(o), _ptr(d), tmin, tmax, exclude,
                                 1 if use_bvh else 0, C.byref(t), C.byref(m), C.byref(t2))
    return prim, t.value, m.value, t2.value


def arc_nodes(ssp: dict, o, d, h: float, n: int):
    z = np.ascontiguousarray(ssp["z"], np.float64)
    c = np.ascontiguousarray(ssp["c"], np.float64)
    pos = np.zeros((n, 3))
    tt = np.zeros(n)
    th = np.zeros(n)
    lib().orc_arc_nodes(_ptr(z), _ptr(c), len(z), _ptr(np.asarray(o, np.float64)),
                        _ptr(np.asarray(d, np.float64)), h, n, _ptr(pos), _ptr(tt), _ptr(th))
    return pos, tt, th


def eigen_arc(ssp: dict, o, x):
    z = np.ascontiguousarray(ssp["z"], np.float64)
    c = np.ascontiguousarray(ssp["c"], np.float64)
    d = np.zeros(3)
    t, s = C.c_double(), C.c_double()
    rc = lib().orc_eigen_arc(_ptr(z), _ptr(c), len(z), _ptr(np.asarray(o, np.float64)),
                             _ptr(np.asarray(x, np.float64)), _ptr(d), C.byref(t), C.byref(s))
    if rc != 0:
        raise RuntimeError("eigen_arc failed")
    return d, t.value, s.value


def synth_wideband(params: dict, hits: dict, ns, shift: float = 0.0) -> np.ndarray:
    """Wideband element echoes s_m(t_n + shift): the plane-wave delay u_k . p_m / c across
    the aperture in the envelope as well as in the phase. complex128 [len(ns), M]."""
    ns = np.ascontiguousarray(ns, np.int32)
    M = params["nx"] * params["ny"]
    out = np.zeros((len(ns), M, 2), np.float64)
    hs, keep = _hits_struct(hits)
    lib().orc_synth_wb(C.byref(make_params(params)), C.byref(hs), float(shift), _ptr(ns), len(ns), _ptr(out))
    return out[..., 0] + 1j * out[..., 1]


def ttd_exact(params: dict, hits: dict, ns, beams, taper=None) -> np.ndarray:
    """True-time-delay beams of the wideband echoes, exact in time: complex128
    [len(beams), len(ns)]."""
    ns = np.ascontiguousarray(ns, np.int32)
    beams = np.ascontiguousarray(beams, np.int32)
    out = np.zeros((len(beams), len(ns), 2), np.float64)
    hs, keep = _hits_struct(hits)
    tp = None if taper is None else np.ascontiguousarray(taper, np.float32)
    lib().orc_ttd(C.byref(make_params(params)), C.byref(hs), _ptr(tp), _ptr(ns), len(ns), _ptr(beams), len(beams),
                  _ptr(out))
    return out[..., 0] + 1j * out[..., 1]


def ttd_levels(params: dict, c_ref: float, U: int) -> tuple:
    """The fractional-delay grid of the true-time-delay beamformer: per (beam, element)
    the steering delay -u_b . p_m / c in units of dt / U, x [Nb, M], and the level range
    Q (levels q = -Q .. Q cover floor(x) - 1 .. floor(x) + 2 for every pair)."""
    nba, nbe, nx, ny = params["n_beam_az"], params["n_beam_el"], params["nx"], params["ny"]
    dt = 2.0 * (params["r_max"] - params["r_min"]) / params["n_range"] / c_ref
    i, j = np.arange(nba), np.arange(nbe)
    az = -params["hfov"] / 2 + (i + 0.5) * params["hfov"] / nba
    el = -params["vfov"] / 2 + (j + 0.5) * params["vfov"] / nbe
    uy = (np.cos(el)[:, None] * np.sin(az)[None, :]).ravel()
    uz = np.repeat(np.sin(el), nba)
    m = np.arange(nx * ny)
    ym = (m % nx - (nx - 1) / 2.0) * params["pitch"]
    zm = (m // nx - (ny - 1) / 2.0) * params["pitch"]
    x = -(uy[:, None] * ym[None, :] + uz[:, None] * zm[None, :]) / c_ref / (dt / U)
    Q = int(np.ceil(np.abs(x).max())) + 2
    return x, Q


def lagrange4(y) -> np.ndarray:
    """The 4-point Lagrange interpolation kernel: the weight of a sample at distance y
    (in samples) from the point read; cubic pieces on |y| < 1 and 1 <= |y| < 2, zero
    beyond; reproduces cubic polynomials exactly."""
    a = np.abs(np.asarray(y, np.float64))
    return np.where(a < 1.0, (a * a - 1.0) * (a - 2.0) / 2.0,
                    np.where(a < 2.0, -(a - 1.0) * (a - 2.0) * (a - 3.0) / 6.0, 0.0))


def ttd_interpolated(params: dict, hits: dict, ns, U: int, beams=None, taper=None) -> np.ndarray:
    """True-time-delay beams as the fractional-delay beamformer forms them: each element's
    wideband echo read at its steering delay by 4-point Lagrange interpolation between the
    samples of a grid U times finer than the range grid,
    B[b][n] = sum_m W[b][m] sum_q h(x_bm - q) s_m(t_n + q dt / U) with h = lagrange4 and W
    the phase-shift weights. complex128 [len(beams), len(ns)]."""
    nb = params["n_beam_az"] * params["n_beam_el"]
    beams = np.arange(nb) if beams is None else np.asarray(beams)
    c_ref = hits["c_ref"]
    x, Q = ttd_levels(params, c_ref, U)
    dt = 2.0 * (params["r_max"] - params["r_min"]) / params["n_range"] / c_ref
    M = params["nx"] * params["ny"]
    w = np.ones(M) if taper is None else np.asarray(taper, np.float64).ravel()
    m = np.arange(M)
    ym = (m % params["nx"] - (params["nx"] - 1) / 2.0) * params["pitch"]
    zm = (m // params["nx"] - (params["ny"] - 1) / 2.0) * params["pitch"]
    ka = 2 * math.pi * params["f0"] / c_ref
    nba = params["n_beam_az"]
    out = np.zeros((len(beams), len(ns)), np.complex128)
    for q in range(-Q, Q + 1):
        s_q = synth_wideband(params, hits, ns, shift=q * dt / U)  # [n, M]
        for a, b in enumerate(beams):
            i, j = b % nba, b // nba
            az = -params["hfov"] / 2 + (i + 0.5) * params["hfov"] / nba
            el = -params["vfov"] / 2 + (j + 0.5) * params["vfov"] / params["n_beam_el"]
            uy, uz = math.cos(el) * math.sin(az), math.sin(el)
            Wb = w * np.exp(-1j * ka * (uy * ym + uz * zm)) / w.sum()
            hq = lagrange4(x[b] - q)
            out[a] += s_q @ (Wb * hq)
    return out
