"""Pins of the FP64 oracle against closed forms, brute force and invariants.

None of these tests re-types an oracle formula: each compares the oracle with an
independent route to the same quantity (numerical integration of a definition, the
Dirichlet-kernel closed form, a linear solve, an RK4 integration, exact symmetry), so
a dropped term, a wrong sign or index or a transposed operand in the oracle fails one.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_06130_gb300 import inputs

T_P = 100e-6
BW = 50e3


# ------------------------------------------------------------------ pulse autocorrelation
def _pulse(t):
    """Hann-windowed LFM pulse by its definition (Sec. II.B, reading A1/A2)."""
    inside = np.abs(t) <= T_P / 2
    w = 0.5 * (1.0 + np.cos(2 * np.pi * t / T_P))
    return np.where(inside, w * np.exp(1j * np.pi * (BW / T_P) * t * t), 0.0)


def numeric_acf(u, n=1 << 17):
    """R(u) = int p(v+u) p*(v) dv / int |p|^2 by the trapezoid rule on a fine grid."""
    v = np.linspace(-T_P / 2, T_P / 2, n + 1)
    h = v[1] - v[0]
    wts = np.full(v.shape, h)
    wts[0] = wts[-1] = h / 2
    p0 = _pulse(v)
    energy = np.sum(wts * np.abs(p0) ** 2)
    out = np.zeros(np.shape(u), np.complex128)
    for i, x in enumerate(np.ravel(u)):
        out.ravel()[i] = np.sum(wts * _pulse(v + x) * np.conj(p0)) / energy
    return out


def test_acf_equals_numeric_correlation():
    u = np.concatenate([np.linspace(-1.05 * T_P, 1.05 * T_P, 97), [0.0, 1e-9, -3.3e-5, 7.77e-5]])
    ref = numeric_acf(u)
    got = oracle.pulse_acf(u, T_P, BW)
    assert np.max(np.abs(got - ref)) < 1e-9
    assert abs(got[np.argmin(np.abs(u))] - 1.0) < 1e-12


def test_acf_hermitian_and_support():
    u = np.linspace(0, 1.2 * T_P, 61)
    a = oracle.pulse_acf(u, T_P, BW)
    b = oracle.pulse_acf(-u, T_P, BW)
    assert np.max(np.abs(a - np.conj(b))) < 1e-13
    assert np.all(np.abs(a[u >= T_P]) == 0.0)


# ------------------------------------------------------------------ array factor
def _dirichlet(psi, n):
    """Array factor of n centred isotropic elements: sin(n psi/2) / (n sin(psi/2))."""
    psi = np.asarray(psi, np.float64)
    s = np.sin(psi / 2)
    out = np.ones_like(psi)
    nz = np.abs(s) > 1e-12
    out[nz] = np.sin(n * psi[nz] / 2) / (n * s[nz])
    # exact limits at psi = 2 pi k
    k = np.round(psi[~nz] / (2 * np.pi)).astype(int)
    out[~nz] = np.where(k % 2 == 0, 1.0, (-1.0) ** (n - 1))
    return out


def _beam_dirs(p):
    i = np.arange(p["n_beam_az"])
    j = np.arange(p["n_beam_el"])
    az = -p["hfov"] / 2 + (i + 0.5) * p["hfov"] / p["n_beam_az"]
    el = -p["vfov"] / 2 + (j + 0.5) * p["vfov"] / p["n_beam_el"]
    EL, AZ = np.meshgrid(el, az, indexing="ij")
    return np.stack([np.cos(EL) * np.cos(AZ), np.cos(EL) * np.sin(AZ), np.sin(EL)], -1).reshape(-1, 3)


@pytest.mark.parametrize("nx,ny", [(8, 8), (5, 4)])
def test_beamformer_equals_array_factor(nx, ny):
    p = dict(inputs.sensor_params("c1"), nx=nx, ny=ny)
    c = 1500.0
    ka = 2 * np.pi * p["f0"] / c
    d = p["pitch"]
    rng = np.random.default_rng(3)
    # plane waves from random and from beam-centre directions
    us = list(rng.normal(size=(20, 3)))
    us += list(_beam_dirs(p)[rng.integers(0, 512, 6)])
    us = [u / np.linalg.norm(u) for u in us]
    mx, my = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    ym = ((mx - (nx - 1) / 2) * d).ravel()
    zm = ((my - (ny - 1) / 2) * d).ravel()
    s = np.array([np.exp(1j * ka * (u[1] * ym + u[2] * zm)) for u in us])
    B = oracle.beamform(p, c, s)                      # [Nb, n_waves]
    ub = _beam_dirs(p)
    for w, u in enumerate(us):
        af = _dirichlet(ka * d * (u[1] - ub[:, 1]), nx) * _dirichlet(ka * d * (u[2] - ub[:, 2]), ny)
        assert np.max(np.abs(B[:, w] - af)) < 1e-9


# ------------------------------------------------------------------ single point scatterer
def _empty_scene(points, sigma, planes=None):
    return inputs.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32),
                        np.zeros(0, np.float32), np.zeros(0, np.uint8),
                        np.asarray(points, np.float32).reshape(-1, 3), np.asarray(sigma, np.float32),
                        np.zeros((0, 4)) if planes is None else np.asarray(planes, np.float64))


def _rot(q):
    return inputs._rot(q)


def test_single_point_full_volume_closed_form():
    p = dict(inputs.sensor_params("c1"), surface_z=math.nan, max_bounces=0)
    ps = inputs.pose((1.0, -2.0, -3.0), yaw_deg=20.0, tilt_down_deg=12.0, roll_deg=5.0)
    x = np.array([3.2, -0.7, -3.6], np.float32)
    sc = _empty_scene([x], [0.8])
    h = oracle.trace(sc, p, ps, inputs.ssp("c1"))
    assert h["n"] == 1
    E, _, _ = oracle.volume(p, h)
    c = 1500.0
    dv = x.astype(np.float64) - ps["t"]
    L = np.linalg.norm(dv)
    u = _rot(ps["q"]).T @ (dv / L)
    tau = 2 * L / c
    dr = (p["r_max"] - p["r_min"]) / p["n_range"]
    rn = p["r_min"] + (np.arange(p["n_range"]) + 0.5) * dr
    tn = 2 * rn / c
    R = numeric_acf(tn - tau)
    ka = 2 * np.pi * p["f0"] / c
    ub = _beam_dirs(p)
    af = (_dirichlet(ka * p["pitch"] * (u[1] - ub[:, 1]), p["nx"])
          * _dirichlet(ka * p["pitch"] * (u[2] - ub[:, 2]), p["ny"]))
    ref = (float(np.float32(0.8)) / L ** 2) * np.abs(af)[:, None] * np.abs(R)[None, :] * rn[None, :]
    assert np.max(np.abs(E - ref)) < 1e-9 * ref.max()


def test_point_at_beam_and_bin_centre_peaks_exactly():
    p = dict(inputs.sensor_params("c1"), surface_z=math.nan, max_bounces=0, thr_mode=0, thr=0.0)
    ps = inputs.pose((0.0, 0.0, -2.0), yaw_deg=-30.0, tilt_down_deg=15.0)
    b, n = 7 * 32 + 21, 137
    dr = (p["r_max"] - p["r_min"]) / p["n_range"]
    rn = p["r_min"] + (n + 0.5) * dr
    u = _beam_dirs(p)[b]
    x = _rot(ps["q"]) @ (rn * u) + ps["t"]
    sc = _empty_scene([x], [1.0])
    h = oracle.trace(sc, p, ps, inputs.ssp("c1"))
    E, _, _ = oracle.volume(p, h)
    assert np.unravel_index(np.argmax(E), E.shape) == (b, n)
    # float32 storage of the point moves it by < 1e-6 m: value a r_n = r_n / L^2 ~ 1 / r_n
    assert abs(E[b, n] - 1.0 / rn) < 1e-5
    pk = oracle.peaks(p, ps, E)
    k = list(pk["beam"]).index(b)
    assert pk["bin"][k] == n
    assert np.allclose(pk["xyzi"][k, :3], x, atol=1e-5)


# ------------------------------------------------------------------ mirror image delay
def test_seabed_mirror_path_at_image_source_delay():
    p = dict(inputs.sensor_params("c1"), surface_z=math.nan, max_bounces=1, thr_mode=0, thr=0.0)
    ps = inputs.pose((0.0, 0.0, -2.0), tilt_down_deg=15.0)
    sea = np.array([[-10, -10, -4], [10, -10, -4], [10, 10, -4], [-10, 10, -4]], np.float32)
    x = np.array([2.6, 0.4, -3.0])
    sc = inputs.Scene(sea, np.array([[0, 1, 2], [0, 2, 3]], np.int32), np.zeros(2, np.float32),
                      np.ones(2, np.uint8), x[None].astype(np.float32), np.ones(1, np.float32),
                      np.array([[0.0, 0.0, 1.0, -4.0]]))
    h = oracle.trace(sc, p, ps, inputs.ssp("c1"))
    pts = h["prim"] < 0
    c = 1500.0
    xf = x.astype(np.float32).astype(np.float64)
    ximg = xf * np.array([1, 1, -1]) + np.array([0, 0, -8.0])
    t_direct = 2 * np.linalg.norm(xf - ps["t"]) / c
    t_image = 2 * np.linalg.norm(ximg - ps["t"]) / c
    taus = sorted(h["tau"][pts])
    assert len(taus) == 2
    assert abs(taus[0] - t_direct) < 1e-15 and abs(taus[1] - t_image) < 1e-15
    # the image route shows as a local peak in the beam of the image direction
    E, _, _ = oracle.volume(p, h)
    ub = _beam_dirs(p)
    uimg = _rot(ps["q"]).T @ ((ximg - ps["t"]) / np.linalg.norm(ximg - ps["t"]))
    b = int(np.argmax(ub @ uimg))
    dr = p["r_max"] / p["n_range"]
    n_img = int(round(t_image * c / 2 / dr - 0.5))
    win = E[b, n_img - 6:n_img + 7]
    assert abs(int(np.argmax(win)) - 6) <= 1 and win.max() > 0


def test_surface_image_route():
    p = dict(inputs.sensor_params("c1"), surface_z=0.0, max_bounces=1, r_max=5.0)
    ps = inputs.pose((0.0, 0.0, -1.0), tilt_down_deg=-10.0)
    x = np.array([3.0, 0.2, -0.6])
    sc = _empty_scene([x], [1.0])
    h = oracle.trace(sc, p, ps, inputs.ssp("c1"))
    xf = x.astype(np.float32).astype(np.float64)
    ximg = xf * np.array([1, 1, -1])
    got = sorted(h["tau"])
    want = sorted([2 * np.linalg.norm(xf - ps["t"]) / 1500, 2 * np.linalg.norm(ximg - ps["t"]) / 1500])
    assert np.allclose(got, want, rtol=0, atol=1e-15)
    # the surface route carries Gamma^2 = 1 and sigma / L^2
    amp_img = h["amp"][np.argmax(h["tau"])]
    assert abs(amp_img - 1.0 / np.linalg.norm(ximg - ps["t"]) ** 2) < 1e-12


# ------------------------------------------------------------------ curved rays
def _rk4_ray(c0, g, z0, o, d, ds, n):
    """RK4 on the eikonal ray equations dr/ds = c p, dp/ds = -grad(c)/c^2, dT/ds = 1/c."""
    def cz(z):
        return c0 + g * (z - z0)

    def f(y):
        r, pv = y[:3], y[3:6]
        c = cz(r[2])
        grad = np.array([0.0, 0.0, g])
        return np.concatenate([c * pv, -grad / c ** 2, [1.0 / c]])

    y = np.concatenate([o, np.asarray(d) / cz(o[2]), [0.0]])
    out = [y.copy()]
    for _ in range(n):
        k1 = f(y)
        k2 = f(y + ds / 2 * k1)
        k3 = f(y + ds / 2 * k2)
        k4 = f(y + ds * k3)
        y = y + ds / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        out.append(y.copy())
    return np.array(out)


@pytest.mark.parametrize("theta_deg", [-25.0, -3.0, 0.0, 8.0])
def test_arc_nodes_match_rk4(theta_deg):
    ssp = inputs.ssp("c3")
    g = (1490.0 - 1500.0) / (-10.0 - 0.0)
    o = np.array([0.3, -0.2, -2.0])
    th = math.radians(theta_deg)
    az = 0.4
    d = np.array([math.cos(th) * math.cos(az), math.cos(th) * math.sin(az), math.sin(th)])
    h = 0.5
    pos, tt, _ = oracle.arc_nodes(ssp, o, d, h, 41)
    steps_per_node = 100
    ref = _rk4_ray(1500.0, g, 0.0, o, d, h / steps_per_node, 40 * steps_per_node)[::steps_per_node]
    assert np.max(np.abs(pos - ref[:, :3])) < 1e-9
    assert np.max(np.abs(tt - ref[:, 6])) < 1e-12 * max(1.0, tt.max())


def test_eigen_arc_reaches_point():
    ssp = inputs.ssp("c3")
    g = 1.0
    o = np.array([0.0, 0.0, -2.0])
    for x in ([3.0, 1.0, -3.5], [1.0, -2.0, -0.5], [4.4, 0.0, -2.0]):
        x = np.array(x)
        d, T, s = oracle.eigen_arc(ssp, o, x)
        n = 2000
        ref = _rk4_ray(1500.0, g, 0.0, o, d, s / n, n)
        assert np.max(np.abs(ref[-1, :3] - x)) < 1e-9
        assert abs(ref[-1, 6] - T) < 1e-13


# ------------------------------------------------------------------ traversal
def _random_mesh(rng, n):
    c = rng.uniform(-2, 2, size=(n, 1, 3))
    v = (c + rng.normal(scale=0.3, size=(n, 3, 3))).reshape(-1, 3).astype(np.float32)
    t = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    return inputs.Scene(v, t, np.full(n, 0.3, np.float32), np.zeros(n, np.uint8))


def _solve_hit(sc, o, d):
    """Nearest hit by solving o + t d = a + u (b - a) + v (c - a) for every triangle."""
    best = (math.inf, -1)
    for k, (ia, ib, ic) in enumerate(sc.tris):
        a, b, c = (sc.verts[i].astype(np.float64) for i in (ia, ib, ic))
        A = np.stack([-d, b - a, c - a], 1)
        if abs(np.linalg.det(A)) < 1e-14:
            continue
        t, u, v = np.linalg.solve(A, o - a)
        if u >= 0 and v >= 0 and u + v <= 1 and t > 1e-7 and t < best[0]:
            best = (t, k)
    return best


@pytest.mark.parametrize("n_tris", [1, 37, 600])
def test_bvh_equals_brute_force(n_tris):
    rng = np.random.default_rng(n_tris)
    sc = _random_mesh(rng, n_tris)
    for _ in range(150):
        o = rng.uniform(-4, 4, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        a = oracle.closest_hit(sc, o, d, use_bvh=True)
        b = oracle.closest_hit(sc, o, d, use_bvh=False)
        assert a[0] == b[0] and (a[0] < 0 or a[1] == b[1])


def test_triangle_test_equals_linear_solve():
    rng = np.random.default_rng(11)
    sc = _random_mesh(rng, 40)
    hits = 0
    for _ in range(200):
        o = rng.uniform(-3, 3, 3)
        tgt = sc.verts[rng.integers(0, len(sc.verts))].astype(np.float64)
        d = tgt - o + rng.normal(scale=0.2, size=3)
        d /= np.linalg.norm(d)
        prim, t, margin, _ = oracle.closest_hit(sc, o, d, use_bvh=False)
        t_ref, k_ref = _solve_hit(sc, o, d)
        if k_ref < 0:
            assert prim < 0
            continue
        hits += 1
        if margin > 1e-9:
            assert prim == k_ref and abs(t - t_ref) < 1e-10
    assert hits > 25


# ------------------------------------------------------------------ invariants
def test_superposition_of_two_points():
    p = dict(inputs.sensor_params("c1"), surface_z=math.nan, max_bounces=0)
    ps = inputs.pose((0.0, 0.0, -2.0), tilt_down_deg=15.0)
    x1, x2 = [2.5, 0.3, -2.8], [3.1, -0.9, -2.2]
    ssp = inputs.ssp("c1")
    B = []
    for pts in ([x1], [x2], [x1, x2]):
        h = oracle.trace(_empty_scene(pts, [1.0] * len(pts)), p, ps, ssp)
        B.append(oracle.volume(p, h)[1])
    assert np.max(np.abs(B[2] - B[0] - B[1])) < 1e-12 * np.abs(B[2]).max()


def test_mirror_symmetric_scene_gives_mirror_symmetric_volume():
    p = dict(inputs.sensor_params("c1"), surface_z=math.nan, max_bounces=1)
    ps = inputs.pose((0.0, 0.0, -2.0), tilt_down_deg=15.0)
    sea = np.array([[-10, -10, -4], [10, -10, -4], [10, 10, -4], [-10, 10, -4]], np.float32)
    pts = [[2.5, 0.75, -3.0], [2.5, -0.75, -3.0], [3.5, 0.0, -2.5]]
    sc = inputs.Scene(sea, np.array([[0, 1, 2], [0, 2, 3]], np.int32), np.zeros(2, np.float32),
                      np.ones(2, np.uint8), np.array(pts, np.float32), np.ones(3, np.float32),
                      np.array([[0.0, 0.0, 1.0, -4.0]]))
    h = oracle.trace(sc, p, ps, inputs.ssp("c1"))
    E = oracle.volume(p, h)[0].reshape(p["n_beam_el"], p["n_beam_az"], p["n_range"])
    assert np.max(np.abs(E - E[:, ::-1, :])) < 1e-12 * E.max()


def test_peak_rules_first_index_blanking_and_threshold():
    p = dict(inputs.sensor_params("c1"), n_beam_az=2, n_beam_el=1, n_range=8, r_max=8.0,
             r_blank=2.0, thr_mode=1, thr=0.5)
    ps = inputs.pose((0.0, 0.0, 0.0))
    E = np.array([[9.0, 1.0, 3.0, 5.0, 5.0, 1.0, 0.0, 0.0],     # blanked bins 0, 1; tie -> bin 3
                  [0.0, 0.0, 1.0, 2.0, 2.0, 0.0, 0.0, 0.0]])    # 2 < 0.5 * 5 -> dropped
    pk = oracle.peaks(p, ps, E)
    assert list(pk["beam"]) == [0] and list(pk["bin"]) == [3]
    assert pk["xyzi"][0, 3] == 5.0


# ------------------------------------------------------------------ hash
def test_pcg4d_uniform_and_decorrelated():
    v = np.stack([np.arange(4096, dtype=np.uint32), np.zeros(4096, np.uint32),
                  np.ones(4096, np.uint32), np.full(4096, 7, np.uint32)], 1)
    out = np.array([oracle.pcg4d(r) for r in v])
    u = (out[:, 0] >> 8) / 2.0 ** 24
    hist = np.histogram(u, bins=16, range=(0, 1))[0]
    chi2 = np.sum((hist - 256.0) ** 2 / 256.0)
    assert chi2 < 40.0
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.05
    assert len(np.unique(out[:, 0])) == 4096


def test_lambertian_power_matches_quadrature():
    """Sum of a_k^2 over a wall facing the sonar approaches mu/D^2 int cos^3 dOmega
    (Lambertian intensity law over the footprint), evaluated by 2-D quadrature."""
    from scipy import integrate
    D, mu = 2.0, 0.4
    p = dict(inputs.sensor_params("c1"), surface_z=math.nan, max_bounces=0, n_ray_az=256,
             n_ray_el=128, r_max=6.0)
    ps = inputs.pose((0.0, 0.0, 0.0))
    wall = np.array([[D, -50, -50], [D, 50, -50], [D, 50, 50], [D, -50, 50]], np.float32)
    sc = inputs.Scene(wall, np.array([[0, 1, 2], [0, 2, 3]], np.int32), np.full(2, mu, np.float32),
                      np.zeros(2, np.uint8))
    h = oracle.trace(sc, p, ps, inputs.ssp("c1"))
    got = np.sum(h["amp"] ** 2)

    def f(el, az):
        cosk = math.cos(el) * math.cos(az)
        return mu * cosk ** 3 / D ** 2 * math.cos(el)

    ref, _ = integrate.dblquad(f, -p["hfov"] / 2, p["hfov"] / 2, -p["vfov"] / 2, p["vfov"] / 2,
                               epsabs=1e-12, epsrel=1e-10)
    assert abs(got - ref) < 2e-4 * ref


def test_acf_is_real_for_centred_chirp():
    """The Hann window is even and the chirp is centred on t = 0, so the window product
    w(s + u/2) w(s - u/2) is even in s and R(u) keeps only its cosine part: a real function
    (the tensor-core synthesis forms real taps |c_k| R and carries arg c_k in the element
    phase). A sign slip in any of the closed form's nine exponential integrals leaves an
    imaginary part."""
    for tp, bw in ((T_P, BW), (40e-6, 120e3), (250e-6, 10e3)):
        u = np.linspace(-1.1 * tp, 1.1 * tp, 801)
        r = oracle.pulse_acf(u, tp, bw)
        assert np.max(np.abs(r.imag)) < 1e-14
        assert np.max(np.abs(r.real)) == pytest.approx(1.0, abs=1e-12)
