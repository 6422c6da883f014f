"""Pins of the oracle's rays in a range-dependent (2-D) sound-speed field (Sec. II.A:
rays bent by Snell's law through a range- and depth-dependent sound speed).

Independent routes to the same rays: a uniform field against the straight-ray route; a
field that varies with depth only against the exact circular arcs of the linear-profile
route; a field that varies with range only against the depth-only case turned by 90
degrees; and the convergence order of the step size.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_06130_gb300 import inputs
from tests import parity


def _field_from(fun, x0=-6.0, x1=16.0, z0=-7.0, z1=3.0, nx=12, nz=11, h=0.05):
    xs, zs = np.linspace(x0, x1, nx), np.linspace(z0, z1, nz)
    c = np.array([[fun(x, z) for x in xs] for z in zs])
    return {"x0": x0, "dx": xs[1] - xs[0], "z0": z0, "dz": zs[1] - zs[0], "c": c, "h": h}


def _wall():
    sc, p, ps, ssp = inputs.workload("wall_mirror")
    # no point scatterers: a 2-D field has no eigen-ray search
    sc = inputs.Scene(sc.verts, sc.tris, sc.mu, sc.flags)
    return sc, dict(p, c_ref=1500.0, max_bounces=1), ps[0]


def _match(a, b, n_sub):
    ka, kb = parity.oracle_keys(a, n_sub), parity.oracle_keys(b, n_sub)
    common, ia, ib = np.intersect1d(ka, kb, return_indices=True)
    return ia, ib, len(ka), len(kb)


def test_uniform_field_equals_straight_rays():
    sc, p, pose = _wall()
    iso = oracle.trace(sc, p, pose, {"z": np.array([0.0]), "c": np.array([1500.0])})
    fld = oracle.trace(sc, dict(p, field=_field_from(lambda x, z: 1500.0, h=0.25)), pose,
                       {"z": np.array([0.0]), "c": np.array([1500.0])})
    ia, ib, na, nb = _match(iso, fld, p["n_sub"])
    assert na == nb == len(ia) > 1000
    assert np.array_equal(iso["prim"][ia], fld["prim"][ib])
    assert np.max(np.abs(fld["tau"][ib] / iso["tau"][ia] - 1)) < 1e-12


@pytest.fixture(scope="module")
def depth_gradient():
    """Strong depth gradient (20 m/s per m: curvature radius ~75 m) so that the rays bend
    measurably over the 10 m of the scene."""
    sc, p, pose = _wall()
    g, zs = 20.0, pose["t"][2]
    prof = {"z": np.array([zs, zs + 1.0]), "c": np.array([1500.0, 1500.0 + g])}
    arcs = oracle.trace(sc, p, pose, prof)
    return sc, p, pose, g, zs, arcs


def test_depth_only_field_follows_the_exact_arcs(depth_gradient):
    sc, p, pose, g, zs, arcs = depth_gradient
    fld = oracle.trace(sc, dict(p, field=_field_from(lambda x, z: 1500.0 + g * (z - zs), h=0.05)), pose,
                       {"z": np.array([0.0]), "c": np.array([1500.0])})
    ia, ib, na, nb = _match(arcs, fld, p["n_sub"])
    assert len(ia) > 0.98 * max(na, nb) and len(ia) > 1000
    clear = (arcs["margin"][ia] > 1e-3) & (arcs["gap"][ia] > 1e-3)
    assert np.all(arcs["prim"][ia][clear] == fld["prim"][ib][clear])
    same = arcs["prim"][ia] == fld["prim"][ib]
    # the arc route places its hits on chords of up to 1e-4 m sagitta, with times linear
    # along each chord: the two agree to that (median 6e-6, at most 4e-5 here, whatever
    # the field step below 0.1 m), against 2.6e-2 for straight rays
    err = np.abs(fld["tau"][ib][same] / arcs["tau"][ia][same] - 1)
    assert err.max() < 1e-4 and np.median(err) < 1e-5, (err.max(), np.median(err))
    # the gradient matters: the straight-ray delays are far off
    iso = oracle.trace(sc, p, pose, {"z": np.array([0.0]), "c": np.array([1500.0])})
    i2, j2, _, _ = _match(arcs, iso, p["n_sub"])
    assert np.median(np.abs(iso["tau"][j2] / arcs["tau"][i2] - 1)) > 1e-4


def _rot_y(v, ang):
    c, s = math.cos(ang), math.sin(ang)
    v = np.asarray(v, np.float64)
    return np.stack([c * v[..., 0] + s * v[..., 2], v[..., 1], -s * v[..., 0] + c * v[..., 2]], -1)


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def test_range_only_field_equals_the_turned_depth_case(depth_gradient):
    """Turning scene, pose and field by 90 degrees about y maps c(z) onto c(x): the hits
    must be the same, up to rounding. Without a sea surface nothing else is tied to z."""
    sc, p, pose, g, zs, _ = depth_gradient
    p = dict(p, surface_z=None)
    f_z = _field_from(lambda x, z: 1500.0 + g * (z - zs), h=0.05)
    a = oracle.trace(sc, dict(p, field=f_z), pose, {"z": np.array([0.0]), "c": np.array([1500.0])})
    ang = math.pi / 2  # z -> x: (x, z) -> (x cos + z sin, -x sin + z cos) = (z, -x)
    sc2 = inputs.Scene(_rot_y(sc.verts, ang).astype(np.float32), sc.tris, sc.mu, sc.flags)
    t2 = _rot_y(pose["t"], ang)
    q2 = _qmul(np.array([math.cos(ang / 2), 0.0, math.sin(ang / 2), 0.0]), pose["q"])
    xs2 = t2[0]  # the old depth of the sonar is now its x
    f_x = _field_from(lambda x, z: 1500.0 + g * (x - xs2), x0=-8.0, x1=4.0, z0=-17.0, z1=7.0, nx=13, nz=12, h=0.05)
    b = oracle.trace(sc2, dict(p, field=f_x), {"t": t2, "q": q2}, {"z": np.array([0.0]), "c": np.array([1500.0])})
    ia, ib, na, nb = _match(a, b, p["n_sub"])
    assert len(ia) > 0.99 * max(na, nb) and len(ia) > 1000
    clear = (a["margin"][ia] > 1e-6) & (a["gap"][ia] > 1e-6)
    assert np.all(a["prim"][ia][clear] == b["prim"][ib][clear])
    same = a["prim"][ia] == b["prim"][ib]
    assert np.max(np.abs(b["tau"][ib][same] / a["tau"][ia][same] - 1)) < 1e-10


def test_step_convergence(depth_gradient):
    """Halving the step shrinks the delay error by about four or more (second order from
    the chords, fourth from the integrator; a first-order integrator would only halve
    it). Reference: the same route at a step of 1/64 of the largest."""
    sc, p, pose, g, zs, _ = depth_gradient
    prof = {"z": np.array([0.0]), "c": np.array([1500.0])}
    run = lambda h: oracle.trace(sc, dict(p, field=_field_from(lambda x, z: 1500.0 + g * (z - zs), h=h)), pose, prof)
    ref = run(0.8 / 64)
    errs = []
    for h in (0.8, 0.4, 0.2):
        fld = run(h)
        ia, ib, _, _ = _match(ref, fld, p["n_sub"])
        same = (ref["prim"][ia] == fld["prim"][ib]) & (ref["margin"][ia] > 1e-3) & (ref["gap"][ia] > 1e-3)
        errs.append(np.median(np.abs(fld["tau"][ib][same] / ref["tau"][ia][same] - 1)))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


def test_field_rejects_bad_grids_and_combinations():
    sc, p, pose = _wall()
    prof = {"z": np.array([0.0]), "c": np.array([1500.0])}
    bad = _field_from(lambda x, z: 1500.0)
    bad["c"] = bad["c"].copy()
    bad["c"][3, 4] = -1.0
    with pytest.raises(RuntimeError):
        oracle.trace(sc, dict(p, field=bad), pose, prof)
    with pytest.raises(RuntimeError):
        oracle.trace(sc, dict(p, field=_field_from(lambda x, z: 1500.0), cross=1), pose, prof)


def _arc_closed_form(c0, g, z0, o, d, s):
    """Exact ray in c = c0 + g (z - z0) after arc length s: a circular arc in the vertical
    plane of d with Snell invariant xi = cos(theta) / c; theta(s) = theta0 - xi g s;
    horizontal and vertical displacements (sin th0 - sin th) / (xi g) and
    (cos th - cos th0) / (xi g); time (atanh(sin th0) - atanh(sin th)) / g."""
    hz = math.hypot(d[0], d[1])
    e = np.array([d[0] / hz, d[1] / hz])
    th0 = math.atan2(d[2], hz)
    xi = math.cos(th0) / (c0 + g * (o[2] - z0))
    th = th0 - xi * g * s
    dh = (math.sin(th0) - math.sin(th)) / (xi * g)
    dz = (math.cos(th) - math.cos(th0)) / (xi * g)
    T = (math.atanh(math.sin(th0)) - math.atanh(math.sin(th))) / g
    return np.array([o[0] + dh * e[0], o[1] + dh * e[1], o[2] + dz]), T


@pytest.mark.parametrize("d", [(0.8, 0.3, -0.52), (0.6, -0.7, 0.38), (1.0, 0.0, 0.0)])
def test_integrator_is_fourth_order_against_the_exact_arc(d):
    c0, g, z0 = 1500.0, 40.0, -2.0
    p = dict(inputs.sensor_params("c1"), field=_field_from(lambda x, z: c0 + g * (z - z0), x0=-20, x1=20,
                                                            z0=-20, z1=20, nx=5, nz=5, h=0.1))
    o = np.array([0.3, -0.2, -2.5])
    d = np.asarray(d, np.float64) / np.linalg.norm(d)
    S = 8.0
    r_ex, T_ex = _arc_closed_form(c0, g, z0, o, d, S)
    errs = []
    for n in (8, 16, 32):
        y = oracle.field_ray(p, o, d, S / n, n)
        errs.append(np.linalg.norm(y[:3] - r_ex) + 1500.0 * abs(y[6] - T_ex))
    assert errs[2] < 1e-7, errs
    assert errs[0] / errs[1] > 10 and errs[1] / errs[2] > 10, errs
