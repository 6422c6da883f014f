"""Pins of the oracle's out/back cross-term multipath (Sec. II.B multi-bounce paths,
with outgoing and returning legs allowed to differ).

Each pin reaches the same quantity by another route than the oracle's ray walk: the
image method for reflected routes, a brute-force segment test over every triangle for
the shadowing, and the two-ray (Lloyd's mirror) closed form for point scatterers.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_06130_gb300 import inputs

SEABED_Z = -4.0


def _rot(q):
    """Rotation matrix of a unit quaternion (w, x, y, z)."""
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[w * w + x * x - y * y - z * z, 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), w * w - x * x + y * y - z * z, 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), w * w - x * x - y * y + z * z]])


@pytest.fixture(scope="module")
def wm():
    sc, p, ps, ssp = inputs.workload("wall_mirror")
    h = oracle.trace(sc, dict(p, cross=1), ps[0], ssp)
    return sc, p, ps[0], ssp, h


def _by_key(h, seg):
    sel = np.nonzero((h["prim"] >= 0) & (h["seg"] == seg))[0]
    return {(int(h["ray"][i]), int(h["sub"][i])): i for i in sel}


def _seabed_route_geometry(h, i, pose):
    """Hit point X of a one-bounce seabed route by the image method: the unfolded ray
    from the sonar along the launch direction, L_r long, mirrored back across the seabed."""
    R = _rot(pose["q"])
    us = np.array([h["ux"][i], h["uy"][i], h["uz"][i]])
    d0 = R @ us
    L_r = h["len"][i]
    xp = pose["t"] + L_r * d0
    X = np.array([xp[0], xp[1], 2 * SEABED_Z - xp[2]])
    d_in = np.array([d0[0], d0[1], -d0[2]])
    return X, d_in, L_r, us


def test_cross_pairs_follow_the_image_method(wm):
    sc, p, pose, ssp, h = wm
    c = h["c_ref"]
    R = _rot(pose["q"])
    route, back_direct, back_route = _by_key(h, 1), _by_key(h, 17), _by_key(h, 33)
    assert len(back_direct) > 300 and back_direct.keys() == back_route.keys()
    n_wall = np.array([-1.0, 0.0, 0.0])
    for key, j in back_direct.items():
        i, k = route[key], back_route[key]
        X, d_in, L_r, us = _seabed_route_geometry(h, i, pose)
        assert abs(X[0] - 6.0) < 1e-9 and -4.0 <= X[2] <= 0.0
        v = X - pose["t"]
        L_d = np.linalg.norm(v)
        assert abs(h["tau"][j] * c - (L_r + L_d)) < 1e-12 * (L_r + L_d)
        u_d = R.T @ (v / L_d)
        assert np.allclose([h["ux"][j], h["uy"][j], h["uz"][j]], u_d, rtol=0, atol=1e-12)
        assert np.allclose([h["ux"][k], h["uy"][k], h["uz"][k]], us, rtol=0, atol=0)
        # bistatic Lambert over the route's footprint: the ratio to the route's own
        # monostatic echo cancels mu and the solid angle
        cos_d = abs(n_wall @ v) / L_d
        cos_r = abs(n_wall @ d_in)
        ratio = math.sqrt(cos_d / cos_r) * L_r / (p["r_seabed"] * L_d)
        assert abs(h["amp"][j] / h["amp"][i] - ratio) < 1e-12 * ratio
        # reciprocal partner: same delay, amplitude and phase
        for f in ("tau", "amp", "phi", "psi"):
            assert h[f][k] == h[f][j]
        assert h["psi"][j] != h["psi"][i]


def _segment_blocked(verts, tris, a, b, skip):
    """Brute force: does the open segment a -> b (minus 1e-4 m at b) cross any triangle
    other than `skip`? Moller-Trumbore over every triangle; also returns the smallest
    barycentric margin among triangles the segment's line meets within the segment."""
    d = b - a
    L = np.linalg.norm(d)
    d = d / L
    v0, v1, v2 = (verts[tris[:, k]].astype(np.float64) for k in range(3))
    e1, e2 = v1 - v0, v2 - v0
    pv = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, pv)
    ok = np.abs(det) > 1e-300
    inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
    tv = a - v0
    u = np.einsum("ij,ij->i", tv, pv) * inv
    qv = np.cross(tv, e1)
    w = (qv @ d) * inv
    t = np.einsum("ij,ij->i", e2, qv) * inv
    inside_t = ok & (t > 1e-7) & (t < L - 1e-4)
    inside_t[skip] = False
    margin = np.minimum(np.minimum(u, w), 1.0 - u - w)
    hit = inside_t & (margin >= 0)
    near = np.min(np.abs(margin[inside_t]), initial=np.inf)
    return bool(hit.any()), near


def test_cross_shadowing_matches_brute_force(wm):
    sc, p, pose, ssp, h = wm
    route, back_direct = _by_key(h, 1), _by_key(h, 17)
    shadowed = visible = 0
    for key, i in route.items():
        X, _, L_r, _ = _seabed_route_geometry(h, i, pose)
        if not abs(X[0] - 6.0) < 1e-9:
            continue
        L_d = np.linalg.norm(X - pose["t"])
        if (L_r + L_d) / h["c_ref"] > 2 * (p["r_max"] / h["c_ref"] + p["pulse"] / 2):
            continue
        blocked, near = _segment_blocked(sc.verts, sc.tris, pose["t"], X, int(h["prim"][i]))
        if near < 1e-9:
            continue  # a near-tie: either answer is correct
        assert (key in back_direct) == (not blocked), key
        shadowed += blocked
        visible += not blocked
    # the plate must hide part of the seabed-lit wall band, and leave the rest
    assert shadowed > 20 and visible > 300, (shadowed, visible)


def test_cross_bvh_equals_brute_force_traversal(wm):
    sc, p, pose, ssp, h = wm
    b = oracle.trace(sc, dict(p, cross=1), pose, ssp, use_bvh=False)
    o1 = np.lexsort((h["seg"], h["sub"], h["ray"], h["prim"]))
    o2 = np.lexsort((b["seg"], b["sub"], b["ray"], b["prim"]))
    for f in ("ray", "sub", "seg", "prim", "tau", "amp", "phi"):
        assert np.array_equal(h[f][o1], b[f][o2]), f


def test_cross_off_leaves_monostatic_hits(wm):
    sc, p, pose, ssp, h = wm
    h0 = oracle.trace(sc, dict(p, cross=0), pose, ssp)
    mono = ~(((h["prim"] >= 0) & (h["seg"] >= 16)) | ((h["prim"] < 0) & (h["sub"] >= 0x10000)))
    assert h0["n"] == int(mono.sum())
    for f in ("ray", "sub", "seg", "prim", "tau", "amp", "phi"):
        assert np.array_equal(h0[f], h[f][mono]), f


def test_points_follow_the_two_ray_model(wm):
    """Lloyd's mirror, squared: with routes direct (Gamma 1, L_1) and seabed (Gamma, L_2),
    out and back, the sum of a point's coefficients c_k = amp exp(j phi) over all four
    out/back combinations is sigma (e^{-j k L_1} / L_1 + Gamma e^{-j k L_2} / L_2)^2."""
    sc, p, pose, ssp, h = wm
    c = h["c_ref"]
    k = 2 * math.pi * p["f0"] / c
    R = _rot(pose["q"])
    for ip, x in enumerate(sc.points.astype(np.float64)):
        sel = (h["prim"] < 0) & (h["ray"] == ip)
        assert sel.sum() == 4
        xi = np.array([x[0], x[1], 2 * SEABED_Z - x[2]])
        L1, L2 = np.linalg.norm(x - pose["t"]), np.linalg.norm(xi - pose["t"])
        g = p["r_seabed"]
        want = sc.sigma[ip] * (np.exp(-1j * k * L1) / L1 + g * np.exp(-1j * k * L2) / L2) ** 2
        got = np.sum(h["amp"][sel] * np.exp(1j * h["phi"][sel]))
        assert abs(got - want) < 1e-9 * abs(sc.sigma[ip] / L1 ** 2), (got, want)
        # the cross pair (out direct, back via the seabed) arrives from the image point
        j = np.nonzero(sel & (h["sub"] == (0x10000 | (0 << 8) | 1)))[0]
        assert len(j) == 1
        u = R.T @ ((xi - pose["t"]) / L2)
        assert np.allclose([h["ux"][j[0]], h["uy"][j[0]], h["uz"][j[0]]], u, rtol=0, atol=1e-12)
        assert abs(h["tau"][j[0]] * c - (L1 + L2)) < 1e-12 * (L1 + L2)


def test_cross_needs_isovelocity():
    sc, p, ps, ssp = inputs.workload("c3")
    with pytest.raises(RuntimeError):
        oracle.trace(sc, dict(p, cross=1), ps[0], ssp)
