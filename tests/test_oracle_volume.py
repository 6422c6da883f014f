"""Pins of the oracle's water-column (volume) reverberation (Sec. II.B volumetric
backscatter paths).

Independent routes to the same quantities: the scatterer positions from a numpy
implementation of the published pcg4d hash (Jarzynski & Olano 2020); the mean
reverberation power per range shell from the volume integral of s_v / r^4; the
shadowing from a brute-force segment test over every triangle; the speckle statistics
of fully developed reverberation (exponential intensity, <I^2> / <I>^2 = 2).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_06130_gb300 import inputs

VOL_TAG = 0x564F4C


def _pcg4d(x, y, z, w):
    """pcg4d on uint32 arrays, from its published definition."""
    m = np.uint32(1664525)
    a = np.uint32(1013904223)
    with np.errstate(over="ignore"):
        x, y, z, w = (v.astype(np.uint32) * m + a for v in (x, y, z, w))
        x = x + y * w; y = y + z * x; z = z + x * y; w = w + y * z
        x ^= x >> np.uint32(16); y ^= y >> np.uint32(16); z ^= z >> np.uint32(16); w ^= w >> np.uint32(16)
        x = x + y * w; y = y + z * x; z = z + x * y; w = w + y * z
    return x, y, z, w


def _positions(n, lo, hi, seed):
    i = np.arange(n, dtype=np.uint64)
    s32 = np.uint32((seed ^ (seed >> 32)) & 0xFFFFFFFF)
    x, y, z, _ = _pcg4d((i & np.uint64(0xFFFFFFFF)).astype(np.uint32), (i >> np.uint64(32)).astype(np.uint32),
                        np.full(n, VOL_TAG, np.uint32), np.full(n, s32, np.uint32))
    u = np.stack([(v >> np.uint32(8)).astype(np.float64) / 2.0 ** 24 for v in (x, y, z)], 1)
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    return lo + (hi - lo) * u


def _empty_scene():
    return inputs.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.float32),
                        np.zeros(0, np.uint8))


def _vol_params(n, lo, hi, sv, **kw):
    p = dict(inputs.sensor_params("c1"), surface_z=None, max_bounces=0, n_ray_az=4, n_ray_el=2,
             vol_n=n, vol_lo=lo, vol_hi=hi, vol_sv=sv)
    p.update(kw)
    return p


def _vol_hits(h):
    sel = (h["prim"] < 0) & (h["sub"] == 0x20000)
    return sel


def test_positions_follow_the_hash_and_the_direct_route():
    pose = inputs.pose((0.5, -0.3, -2.0), yaw_deg=20, tilt_down_deg=15)
    lo, hi = (-4.0, -5.0, -6.0), (6.0, 4.0, 1.0)
    p = _vol_params(5000, lo, hi, 1e-3, r_max=8.0)
    h = oracle.trace(_empty_scene(), p, pose, inputs.ssp("c1"))
    sel = _vol_hits(h)
    X = _positions(5000, lo, hi, p["seed"])
    idx = h["ray"][sel]
    c = h["c_ref"]
    L = np.linalg.norm(X[idx] - pose["t"], axis=1)
    assert np.max(np.abs(h["tau"][sel] * c / 2 - L) / L) < 1e-13
    w, x, y, z = pose["q"] / np.linalg.norm(pose["q"])
    R = np.array([[w * w + x * x - y * y - z * z, 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), w * w - x * x + y * y - z * z, 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), w * w - x * x - y * y + z * z]])
    u = ((X[idx] - pose["t"]) / L[:, None]) @ R
    assert np.max(np.abs(np.stack([h["ux"][sel], h["uy"][sel], h["uz"][sel]], 1) - u)) < 1e-12
    # every scatterer within reach echoes (no mesh), and none beyond it
    L_all = np.linalg.norm(X - pose["t"], axis=1)
    T_stop = p["r_max"] / c + p["pulse"] / 2
    assert np.array_equal(np.sort(idx), np.nonzero(L_all <= T_stop * c)[0])


def test_mean_power_per_range_shell_follows_the_volume_integral():
    """E[sum over shell of amp^2] = sigma^2 n / V int_shell r^-4 dV = 4 pi s_v (1/r1 - 1/r2)
    for a box that contains every shell."""
    sv, n, a = 2e-3, 400_000, 6.0
    pose = inputs.pose((0.0, 0.0, -10.0))
    p = _vol_params(n, (-a, -a, -10 - a), (a, a, -10 + a), sv, r_max=5.5, alpha=0.0)
    h = oracle.trace(_empty_scene(), p, pose, inputs.ssp("c1"))
    sel = _vol_hits(h)
    L = h["tau"][sel] * h["c_ref"] / 2
    a2 = h["amp"][sel] ** 2
    for r1 in np.arange(1.0, 5.0, 0.5):
        r2 = r1 + 0.5
        got = a2[(L >= r1) & (L < r2)].sum()
        want = 4 * math.pi * sv * (1 / r1 - 1 / r2)
        assert abs(got / want - 1) < 0.06, (r1, got / want)


def test_attenuation_and_amplitude_law():
    """The same scatterers with alpha > 0: every amplitude scales by exp(-2 alpha L)."""
    pose = inputs.pose((0.0, 0.0, -10.0))
    base = _vol_params(3000, (-4, -4, -14), (4, 4, -6), 1e-3, r_max=6.0)
    h0 = oracle.trace(_empty_scene(), dict(base, alpha=0.0), pose, inputs.ssp("c1"))
    h1 = oracle.trace(_empty_scene(), dict(base, alpha=0.05), pose, inputs.ssp("c1"))
    assert np.array_equal(h0["ray"], h1["ray"])
    L = h0["tau"] * h0["c_ref"] / 2
    assert np.allclose(h1["amp"] / h0["amp"], np.exp(-0.1 * L), rtol=1e-13, atol=0)
    X = _positions(3000, (-4, -4, -14), (4, 4, -6), base["seed"])
    sigma = math.sqrt(1e-3 * 8 * 8 * 8 / 3000)
    Lx = np.linalg.norm(X[h0["ray"]] - pose["t"], axis=1)
    assert np.allclose(h0["amp"], sigma / Lx ** 2, rtol=1e-13, atol=0)


def test_shadowing_matches_brute_force():
    sc, p, ps, ssp = inputs.workload("wall_mirror")
    lo, hi = (-1.0, -4.0, -4.0), (8.0, 4.0, 0.0)
    n = 6000
    pv = dict(p, vol_n=n, vol_lo=lo, vol_hi=hi, vol_sv=1e-3)
    h = oracle.trace(sc, pv, ps[0], ssp)
    got = set(h["ray"][_vol_hits(h)].tolist())
    X = _positions(n, lo, hi, p["seed"])
    o = ps[0]["t"]
    v0, v1, v2 = (sc.verts[sc.tris[:, k]].astype(np.float64) for k in range(3))
    e1, e2 = v1 - v0, v2 - v0
    T_stop = p["r_max"] / h["c_ref"] + p["pulse"] / 2
    hidden = shown = 0
    for i in range(n):
        d = X[i] - o
        L = np.linalg.norm(d)
        if L > T_stop * h["c_ref"]:
            assert i not in got
            continue
        d /= L
        pv_ = np.cross(d, e2)
        det = np.einsum("ij,ij->i", e1, pv_)
        tv = o - v0
        u = np.einsum("ij,ij->i", tv, pv_) / det
        qv = np.cross(tv, e1)
        w = (qv @ d) / det
        t = np.einsum("ij,ij->i", e2, qv) / det
        inside = (t > 1e-6) & (t < L - 1e-6)
        marg = np.minimum(np.minimum(u, w), 1 - u - w)
        if np.min(np.abs(marg[inside]), initial=np.inf) < 1e-9 or np.min(np.abs(t - (L - 1e-6)), initial=1) < 1e-9:
            continue
        blocked = bool(np.any(inside & (marg >= 0)))
        assert (i in got) == (not blocked), i
        hidden += blocked
        shown += not blocked
    assert hidden > 300 and shown > 1000, (hidden, shown)


def test_reverberation_speckle_is_fully_developed():
    """Many random scatterers per resolution cell: the beam intensity is exponentially
    distributed (circular Gaussian field), so <I^2> / <I>^2 = 2 (a K-distributed excess
    of about 1 / N_cell remains)."""
    pose = inputs.pose((0.0, 0.0, -10.0))
    p = _vol_params(300_000, (-3.5, -3.5, -13.5), (3.5, 3.5, -6.5), 1e-3, r_max=3.0, n_range=128)
    h = oracle.trace(_empty_scene(), p, pose, inputs.ssp("c1"))
    dr = p["r_max"] / p["n_range"]
    ns = np.arange(int(1.5 / dr), int(2.9 / dr), dtype=np.int32)
    E, _, _ = oracle.volume(p, h, ns=ns)
    I = E.astype(np.float64) ** 2
    ratio = np.mean(I ** 2) / np.mean(I) ** 2
    assert 1.85 < ratio < 2.3, ratio


def test_volume_rejects_bad_boxes_and_refraction():
    pose = inputs.pose((0.0, 0.0, -10.0))
    with pytest.raises(RuntimeError):
        oracle.trace(_empty_scene(), _vol_params(10, (0, 0, 0), (1, -1, 1), 1e-3), pose, inputs.ssp("c1"))
    sc, p, ps, ssp = inputs.workload("c3")
    with pytest.raises(RuntimeError):
        oracle.trace(sc, dict(p, vol_n=10, vol_lo=(-1, -1, -3), vol_hi=(1, 1, -1), vol_sv=1e-3), ps[0], ssp)
