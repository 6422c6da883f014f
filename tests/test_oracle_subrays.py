"""Oracle pins of the jittered sub-rays, the mesh speckle key and the carrier phase.

These fix the parts of the ray and hit definitions (Sec. III Eq. 2-3 sampling grid;
Sec. II.B speckle and delay-set carrier phase) that the headline configuration uses and
the other pins run only at one sub-ray per cell:
- the 2x2 stratified jitter: every sub-ray direction lies in its own quarter of its ray
  cell, uniformly and independently along azimuth and elevation, and the four quarters
  split the cell's solid angle (the Lambertian power of a facing wall still matches its
  quadrature at four sub-rays per cell);
- the speckle phase of mesh hits, 2 pi U with U the hash of (ray, sub-ray, 1 + bounce,
  seed), against an independent implementation of the published hash, on direct and
  mirror-route hits;
- the carrier phase of mesh hits: moving a facing wall away by half a wavelength
  lengthens the two-way path of a ray at angle theta from the wall normal by
  lambda / cos(theta), so its phase turns by -2 pi / cos(theta) (one whole carrier
  period on the normal ray), while the speckle phase stays and the amplitude scales by
  the inverse path length.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_06130_gb300 import inputs
from tests.test_oracle_volume import _pcg4d


def _wall(D, mu=0.4, half=50.0):
    v = np.array([[D, -half, -half], [D, half, -half], [D, half, half], [D, -half, half]], np.float32)
    return inputs.Scene(v, np.array([[0, 1, 2], [0, 2, 3]], np.int32), np.full(2, mu, np.float32),
                        np.zeros(2, np.uint8))


def _facing_params(**kw):
    p = dict(inputs.sensor_params("c1"), surface_z=math.nan, max_bounces=0, r_max=6.0, n_sub=4)
    p.update(kw)
    return p


def _u24(x):
    return (np.asarray(x, np.uint32) >> np.uint32(8)).astype(np.float64) / 2.0 ** 24


def test_subrays_lie_in_their_quarter_cells_uniformly():
    """Every sub-ray of a 4-sub-ray grid lies inside its quarter (s & 1 along azimuth,
    s >> 1 along elevation) of its ray cell; the position inside the quarter is uniform
    (mean 1/2 within 6 standard errors, chi-square of 16 bins) and uncorrelated between
    the two axes."""
    p = _facing_params(n_ray_az=128, n_ray_el=64)
    h = oracle.trace(_wall(2.0), p, inputs.pose((0.0, 0.0, 0.0)), inputs.ssp("c1"))
    assert h["n"] == p["n_ray_az"] * p["n_ray_el"] * 4
    nra = p["n_ray_az"]
    i, j, s = h["ray"] % nra, h["ray"] // nra, h["sub"]
    az = np.arctan2(h["uy"], h["ux"])
    el = np.arcsin(np.clip(h["uz"], -1.0, 1.0))
    daz, dele = p["hfov"] / nra, p["vfov"] / p["n_ray_el"]
    # position inside the quarter cell, in units of a quarter cell
    fa = ((az + p["hfov"] / 2) / daz - i) * 2.0 - (s & 1)
    fe = ((el + p["vfov"] / 2) / dele - j) * 2.0 - (s >> 1)
    tol = 1e-9
    assert fa.min() > -tol and fa.max() < 1 + tol
    assert fe.min() > -tol and fe.max() < 1 + tol
    n = len(fa)
    for f in (fa, fe):
        for q in range(4):
            sel = f[s == q]
            assert abs(sel.mean() - 0.5) < 6 * math.sqrt(1 / 12 / len(sel))
        hist = np.histogram(f, bins=16, range=(0, 1))[0]
        chi2 = np.sum((hist - n / 16) ** 2 / (n / 16))
        assert chi2 < 45.0  # 15 degrees of freedom: p < 1e-4
    assert abs(np.corrcoef(fa, fe)[0, 1]) < 6 / math.sqrt(n)


def test_lambertian_power_matches_quadrature_with_four_subrays():
    """The quadrature pin of the Lambertian law at four jittered sub-rays per cell: the
    sub-ray solid angle is the cell's divided by four, so the summed power of a facing
    wall still approaches mu / D^2 times the integral of cos^3 over the field of view."""
    from scipy import integrate
    D, mu = 2.0, 0.4
    p = _facing_params(n_ray_az=128, n_ray_el=64)
    h = oracle.trace(_wall(D, mu), p, inputs.pose((0.0, 0.0, 0.0)), inputs.ssp("c1"))
    got = np.sum(h["amp"] ** 2)

    def f(el, az):
        return mu * (math.cos(el) * math.cos(az)) ** 3 / D ** 2 * math.cos(el)

    ref, _ = integrate.dblquad(f, -p["hfov"] / 2, p["hfov"] / 2, -p["vfov"] / 2, p["vfov"] / 2,
                               epsabs=1e-12, epsrel=1e-10)
    assert abs(got - ref) < 5e-4 * ref


@pytest.mark.parametrize("n_sub", [1, 4])
def test_mesh_speckle_phase_follows_the_hash_key(n_sub):
    """psi of every mesh hit is 2 pi U(pcg4d(ray, sub-ray, 1 + bounce, seed)), on direct
    and seabed-mirror routes (the harbour wall over its mirror seabed, coarse ray grid)."""
    scene, params, poses, ssp = inputs.workload("c2")
    params = dict(params, n_sub=n_sub, n_ray_az=64, n_ray_el=32, seed=0x123456789)
    h = oracle.trace(scene, params, poses[0], ssp)
    mesh = h["prim"] >= 0
    assert np.count_nonzero(mesh & (h["seg"] == 1)) > 20  # mirror routes present
    seed = params["seed"]
    s32 = np.uint32((seed ^ (seed >> 32)) & 0xFFFFFFFF)
    m = int(np.count_nonzero(mesh))
    x, _, _, _ = _pcg4d(h["ray"][mesh].astype(np.uint32), h["sub"][mesh].astype(np.uint32),
                        (1 + h["seg"][mesh]).astype(np.uint32), np.full(m, s32, np.uint32))
    psi = 2 * math.pi * _u24(x)
    assert np.max(np.abs(psi - h["psi"][mesh])) < 1e-12


def test_mesh_carrier_phase_turns_with_half_wavelength_shift():
    """A facing wall moved away by lambda / 2: each ray at angle theta to the wall normal
    gains lambda / cos(theta) of two-way path, so its carrier phase turns by
    -2 pi / cos(theta) (a whole period on the normal), psi is unchanged and the amplitude
    falls as 1 / L."""
    # a carrier of 384 kHz at 1500 m/s puts lambda / 2 at exactly 2^-9 m, so the moved
    # wall's FP32 vertices sit exactly half a wavelength further away
    p = _facing_params(n_ray_az=32, n_ray_el=16, c_ref=1500.0, f0=384e3)
    lam = p["c_ref"] / p["f0"]
    assert lam / 2 == 2.0 ** -9
    D = 2.0
    ps = inputs.pose((0.0, 0.0, 0.0))
    ssp = {"z": np.array([0.0]), "c": np.array([1500.0])}
    a = oracle.trace(_wall(D), p, ps, ssp)
    b = oracle.trace(_wall(D + lam / 2), p, ps, ssp)
    # the wall is two triangles: keys (ray, sub) identify the same sub-ray in both runs
    ka = a["ray"] * 4 + a["sub"]
    kb = b["ray"] * 4 + b["sub"]
    assert np.array_equal(ka, kb)
    cos_t = a["ux"]
    assert np.allclose(a["ux"], b["ux"], rtol=0, atol=1e-15)
    assert np.max(np.abs(a["psi"] - b["psi"])) == 0.0
    dphi = np.angle(np.exp(1j * (b["phi"] - a["phi"])) * np.exp(1j * 2 * math.pi / cos_t))
    assert np.max(np.abs(dphi)) < 1e-9
    assert np.max(np.abs(b["tau"] - a["tau"] - 2 * (lam / 2) / cos_t / 1500.0)) < 1e-15
    assert np.max(np.abs(b["amp"] / a["amp"] - D / (D + lam / 2))) < 1e-12
