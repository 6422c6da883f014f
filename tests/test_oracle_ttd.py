"""Oracle pins of the wideband element echoes and true-time-delay beamforming (Sec. II.A
range- and depth-dependent propagation asks for per-element delays over a wide aperture;
the reading: plane-wave delays across the array kept in the envelope, beams formed by
reading each element at its steering delay).

- Hits arriving broadside (u . p_m = 0 for every element) give the same wideband and
  phase-only echoes.
- A single hit exactly in a beam's direction: the true-time-delay beam is c R(t_n - tau)
  at every sample (the steering delays cancel the arrival delays exactly), whereas the
  phase-shift beam of the same wideband echoes is smeared across the aperture's delays.
- At the broadside beam the steering delays vanish: the true-time-delay beam equals the
  phase-shift beam of the wideband echoes for any hits.
- The fractional-delay form (4-point Lagrange interpolation on a grid U times finer than
  the range samples) converges to the exact beam with the interpolation's fourth order;
  the kernel reproduces cubics exactly and is 1 and 0 on the nodes.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_06130_gb300 import inputs

C = 1500.0


def _hits(tau, c, uy, uz):
    """A hand-made hit list (mesh-free): delays, complex coefficients, arrival (uy, uz)."""
    n = len(tau)
    uy, uz = np.asarray(uy, float), np.asarray(uz, float)
    h = {k: np.zeros(n, np.int32) for k in ("ray", "sub", "seg")}
    h["prim"] = -np.ones(n, np.int32)
    c = np.asarray(c, np.complex128)
    h.update(tau=np.asarray(tau, float), len=np.asarray(tau, float) * C / 2, amp=np.abs(c), psi=np.zeros(n),
             phi=np.angle(c), ux=np.sqrt(1 - uy ** 2 - uz ** 2), uy=uy, uz=uz, cr=c.real, ci=c.imag,
             margin=np.ones(n), gap=np.ones(n), n=n, c_ref=C)
    return h


def _params(**kw):
    p = dict(inputs.sensor_params("c2"), n_beam_az=9, n_beam_el=5, n_range=64, r_max=4.0, c_ref=C)
    p.update(kw)
    return p


def _beam_dir(p, b):
    i, j = b % p["n_beam_az"], b // p["n_beam_az"]
    az = -p["hfov"] / 2 + (i + 0.5) * p["hfov"] / p["n_beam_az"]
    el = -p["vfov"] / 2 + (j + 0.5) * p["vfov"] / p["n_beam_el"]
    return math.cos(el) * math.sin(az), math.sin(el)


def test_broadside_hits_wideband_equals_phase_only():
    p = _params()
    rng = np.random.default_rng(1)
    h = _hits(rng.uniform(1e-3, 4e-3, 6), rng.normal(size=6) + 1j * rng.normal(size=6), np.zeros(6), np.zeros(6))
    ns = np.arange(p["n_range"])
    a = oracle.synth_wideband(p, h, ns)
    b = oracle.synth(p, h, ns)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(b))


def test_ttd_matched_beam_recovers_the_pulse():
    """One hit in beam b's own direction at tau: B_ttd[b][n] = c R(t_n - tau) exactly; the
    phase-shift beam of the same wideband echoes misses its peak by more than 1% of |c|
    (the 32 x 32 aperture spans +-15 us of delay at a corner beam, and R falls to 0.96 at
    5 us)."""
    p = _params(n_range=256)  # 20.8 us samples, as fine as the headline grid's 19.5 us
    b = 0 + 4 * p["n_beam_az"]  # a corner beam: the aperture's delays span +-15 us
    uy, uz = _beam_dir(p, b)
    dr = (p["r_max"] - p["r_min"]) / p["n_range"]
    tau = 2 * (p["r_min"] + 100.5 * dr) / C  # on a sample: the peak of R lands there
    c = 0.7 * np.exp(0.4j)
    h = _hits([tau], [c], [uy], [uz])
    ns = np.arange(p["n_range"])
    got = oracle.ttd_exact(p, h, ns, [b])[0]
    t = 2 * (p["r_min"] + (ns + 0.5) * dr) / C
    want = c * oracle.pulse_acf(t - tau, p["pulse"], p["bw"])
    assert np.max(np.abs(got - want)) < 1e-12
    ps = oracle.beamform(p, C, oracle.synth_wideband(p, h, ns), [b])[0]
    assert np.max(np.abs(ps - want)) > 1e-2 * abs(c)


def test_ttd_broadside_beam_equals_phase_shift_beam():
    p = _params()
    b = (p["n_beam_el"] // 2) * p["n_beam_az"] + p["n_beam_az"] // 2  # the centre beam: u_y = u_z = 0
    assert max(abs(v) for v in _beam_dir(p, b)) < 1e-15
    rng = np.random.default_rng(2)
    n = 12
    h = _hits(rng.uniform(1e-3, 4.5e-3, n), rng.normal(size=n) + 1j * rng.normal(size=n),
              rng.uniform(-0.6, 0.6, n), rng.uniform(-0.3, 0.3, n))
    ns = np.arange(p["n_range"])
    got = oracle.ttd_exact(p, h, ns, [b])[0]
    ps = oracle.beamform(p, C, oracle.synth_wideband(p, h, ns), [b])[0]
    assert np.max(np.abs(got - ps)) < 1e-12 * np.max(np.abs(ps))


def test_lagrange_kernel_reproduces_cubics():
    rng = np.random.default_rng(4)
    coef = rng.normal(size=4)
    for x in rng.uniform(-3, 3, 20):
        q = np.arange(int(np.floor(x)) - 3, int(np.floor(x)) + 5)
        f = np.polyval(coef, q)
        assert abs(np.sum(oracle.lagrange4(x - q) * f) - np.polyval(coef, x)) < 1e-12
    assert list(oracle.lagrange4([0.0, 1.0, -1.0, 2.0, 2.5])) == [1.0, 0.0, 0.0, 0.0, 0.0]


def test_fractional_delay_form_converges_to_exact():
    """On a 20.8 us range grid the Lagrange form's error against the exact beams falls by
    more than eight per doubling of U (fourth order) and is below 1e-3 of the beam energy
    at U = 4."""
    p = _params(n_beam_az=5, n_beam_el=3, n_range=192, r_max=3.0)
    rng = np.random.default_rng(3)
    n = 8
    h = _hits(rng.uniform(0.6e-3, 3.4e-3, n), rng.normal(size=n) + 1j * rng.normal(size=n),
              rng.uniform(-0.6, 0.6, n), rng.uniform(-0.3, 0.3, n))
    ns = np.arange(p["n_range"])
    beams = np.arange(p["n_beam_az"] * p["n_beam_el"])
    exact = oracle.ttd_exact(p, h, ns, beams)
    err = {}
    for U in (2, 4, 8):
        got = oracle.ttd_interpolated(p, h, ns, U, beams)
        err[U] = np.linalg.norm(got - exact) / np.linalg.norm(exact)
    assert err[4] < 1e-3 and err[2] / err[4] > 8.0 and err[4] / err[8] > 8.0, err
