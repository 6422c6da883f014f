"""Pins of the oracle's raw-echo path (Sec. II.B time series and matched filtering).

The raw element series is the echo before pulse compression, r_m(t) = sum_k c_k
p(t - tau_k) exp(j k_a u_k . p_m), p the Hann-windowed chirp; the matched filter
correlates it with p. Pinned here: the pulse's energy and its autocorrelation against the
closed-form R (itself pinned to brute force in test_oracle_pins), the raw series of a
single hit, time-shift invariance and superposition of the raw series, and the
convergence of the matched-filter output to the compressed echoes as the raw sampling
rate grows (the quadrature error of the correlation integral).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_06130_gb300 import inputs

T, BW = 100e-6, 50e3


def test_pulse_energy_is_three_eighths_of_its_length():
    t = np.linspace(-T / 2, T / 2, 20001)
    p = oracle.pulse(t, T, BW)
    e = np.trapezoid(np.abs(p) ** 2, t)
    assert abs(e - 3 * T / 8) < 1e-9 * T
    assert not oracle.pulse(np.array([-T / 2 - 1e-9, T / 2 + 1e-9]), T, BW).any()


@pytest.mark.parametrize("u", [0.0, 7e-6, -23e-6, 51e-6, -88e-6])
def test_pulse_autocorrelation_matches_the_closed_form(u):
    """(1/E) int p(v + u) conj(p(v)) dv by a fine trapezoid rule against orc_pulse_acf."""
    v = np.linspace(-T / 2, T / 2, 40001)
    r = np.trapezoid(oracle.pulse(v + u, T, BW) * np.conj(oracle.pulse(v, T, BW)), v) / (3 * T / 8)
    assert abs(r - oracle.pulse_acf(u, T, BW)[0]) < 2e-8


def one_hit(tau, c=1.0 + 0.0j, uy=0.0, uz=0.0, c_ref=1500.0):
    h = {k: np.zeros(1, np.int32) for k in ("ray", "sub", "seg", "prim")}
    h.update({k: np.zeros(1, np.float64) for k in ("tau", "len", "amp", "psi", "phi", "ux", "uy", "uz", "cr", "ci",
                                                    "margin", "gap")})
    h["tau"][0], h["cr"][0], h["ci"][0], h["uy"][0], h["uz"][0] = tau, c.real, c.imag, uy, uz
    h["n"], h["c_ref"] = 1, c_ref
    return h


def grid(params, c_ref=1500.0):
    dr = (params["r_max"] - params["r_min"]) / params["n_range"]
    return 2 * dr / c_ref, lambda n: 2 * (params["r_min"] + (n + 0.5) * dr) / c_ref


def test_raw_series_of_one_hit_is_the_delayed_pulse_at_every_phase():
    _, params, _, _ = inputs.workload("c1")
    dt, tn = grid(params)
    tau = tn(100) + 0.37 * dt
    c = 0.3 - 0.4j
    ns = np.arange(90, 112)
    U = 3
    raw = oracle.raw_echoes(params, one_hit(tau, c), U, ns)
    for s in range(U):
        want = c * oracle.pulse(tn(ns) + s * dt / U - tau, T, BW)
        # the element phasor is 1 for a broadside arrival (u_y = u_z = 0)
        assert np.abs(raw[s] - want[:, None]).max() < 1e-15


def test_raw_phase_equals_phase_zero_of_an_earlier_echo():
    _, params, _, _ = inputs.workload("c1")
    dt, tn = grid(params)
    tau, U, s = tn(60) + 0.1 * dt, 4, 3
    ns = np.arange(50, 75)
    a = oracle.raw_echoes(params, one_hit(tau, 1j, 0.2, -0.1), U, ns)[s]
    b = oracle.raw_echoes(params, one_hit(tau - s * dt / U, 1j, 0.2, -0.1), U, ns)[0]
    assert np.abs(a - b).max() < 1e-12


def test_raw_series_is_linear_in_the_hits():
    scene, params, poses, ssp = inputs.workload("c1")
    h = oracle.trace(scene, params, poses[0], ssp)
    half = {k: (v[: h["n"] // 2] if isinstance(v, np.ndarray) else v) for k, v in h.items()}
    rest = {k: (v[h["n"] // 2:] if isinstance(v, np.ndarray) else v) for k, v in h.items()}
    half["n"], rest["n"] = h["n"] // 2, h["n"] - h["n"] // 2
    ns = np.arange(0, params["n_range"], 7)
    r = oracle.raw_echoes(params, h, 2, ns)
    r2 = oracle.raw_echoes(params, half, 2, ns) + oracle.raw_echoes(params, rest, 2, ns)
    assert np.abs(r - r2).max() <= 1e-12 * np.abs(r).max()


def test_matched_filter_tends_to_the_compressed_echoes():
    """Sec. II.B: compressing the raw series reproduces the echo defined through the
    pulse autocorrelation; the gap is the rectangle-rule quadrature error, which falls
    with the raw sampling rate U / dt (U = 1 already samples at fs >= B)."""
    scene, params, poses, ssp = inputs.workload("c1")
    h = oracle.trace(scene, params, poses[0], ssp)
    ns = np.arange(params["n_range"])
    s_ref = oracle.synth(params, h, ns)
    err = [np.linalg.norm(oracle.matched_filter(params, h, U, ns) - s_ref) / np.linalg.norm(s_ref)
           for U in (1, 2, 3, 4, 6)]
    assert all(b < a for a, b in zip(err, err[1:])), err
    assert err[3] < 4e-4 and err[4] < 1e-4, err
