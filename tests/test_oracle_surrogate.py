"""Pins of the learned-surrogate oracle (oracle/surrogate.py): the convolution against a
library routine, its impulse response and a hand-computed layer; the backward pass
against central finite differences and the adjoint identities; Adam's first step in
closed form; BF16 rounding on values the format fixes; the geometric rendering against
the closed-form routes of a flat mirror seabed and a wall; rasterisation, the
geometric envelope and the evaluation metrics on hand-worked cases."""
import math

import numpy as np
import pytest

import oracle
from oracle import surrogate as sg
from paper_2606_06130_gb300 import inputs


def _net(channels, seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    W = [rng.normal(0, scale, (channels[i + 1], channels[i], sg.KERNEL)) for i in range(len(channels) - 1)]
    b = [rng.normal(0, 0.1, channels[i + 1]) for i in range(len(channels) - 1)]
    return {"W": W, "b": b}


# ------------------------------------------------------------------ convolution
def test_single_channel_conv_is_library_convolution():
    rng = np.random.default_rng(1)
    x = rng.normal(size=50)
    w = rng.normal(size=sg.KERNEL)
    z = sg.conv(x[None, :, None], w[None, None, :], [0.0])[0, :, 0]
    ref = np.convolve(x, w[::-1], mode="same")
    assert np.max(np.abs(z - ref)) < 1e-13


def test_impulse_response_is_the_kernel():
    """A unit impulse at bin q of channel c gives z[n, o] = b[o] + W[o, c, q - n + 4]
    for |q - n| <= 4 and b[o] elsewhere."""
    net = _net((3, 5))
    W, b = net["W"][0], net["b"][0]
    x = np.zeros((1, 30, 3))
    q, c = 13, 1
    x[0, q, c] = 1.0
    z = sg.conv(x, W, b)[0]
    for n in range(30):
        k = q - n + 4
        want = b + (W[:, c, k] if 0 <= k < sg.KERNEL else 0.0)
        assert np.max(np.abs(z[n] - want)) < 1e-15


def test_hand_computed_layer():
    """W taps 3..5 = (1, 2, 3), bias 0.5 on x = (1, 2, 0, ...): z[n] = 0.5 + x[n-1] + 2 x[n]
    + 3 x[n+1], worked out by hand: 8.5, 5.5, 2.5, then 0.5."""
    W = np.zeros((1, 1, 9))
    W[0, 0, 3:6] = (1.0, 2.0, 3.0)
    x = np.zeros((1, 8, 1))
    x[0, :2, 0] = (1.0, 2.0)
    z = sg.conv(x, W, [0.5])[0, :, 0]
    assert list(z) == [8.5, 5.5, 2.5, 0.5, 0.5, 0.5, 0.5, 0.5]


def test_adjoint_identities():
    """<conv(x, W), z> = <x, input_grad(z, W)> = <W, weight_grad(z, x)>."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 37, 5))
    W = rng.normal(size=(4, 5, 9))
    z = rng.normal(size=(2, 37, 4))
    lhs = np.sum(sg.conv(x, W, None) * z)
    assert abs(lhs - np.sum(x * sg.conv_input_grad(z, W))) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(W * sg.conv_weight_grad(z, x))) < 1e-10 * abs(lhs)


@pytest.mark.parametrize("channels", [(4, 6, 1), (4, 8, 8, 8, 8, 8, 1)])
def test_backward_matches_central_differences(channels):
    rng = np.random.default_rng(3)
    net = _net(channels, seed=4)
    x0 = np.abs(rng.normal(size=(2, 40, channels[0])))
    y = rng.normal(size=(2, 40))
    acts, yhat = sg.forward(net, x0)
    dW, db = sg.backward(net, acts, yhat, y)
    h = 1e-6

    def f():
        return sg.loss(sg.forward(net, x0)[1], y)

    for l in range(len(net["W"])):
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in net["W"][l].shape)
            w0 = net["W"][l][idx]
            net["W"][l][idx] = w0 + h
            fp = f()
            net["W"][l][idx] = w0 - h
            fm = f()
            net["W"][l][idx] = w0
            num = (fp - fm) / (2 * h)
            assert abs(num - dW[l][idx]) < 1e-6 * max(1.0, abs(num)), (l, idx, num, dW[l][idx])
        o = int(rng.integers(0, len(net["b"][l])))
        b0 = net["b"][l][o]
        net["b"][l][o] = b0 + h
        fp = f()
        net["b"][l][o] = b0 - h
        fm = f()
        net["b"][l][o] = b0
        assert abs((fp - fm) / (2 * h) - db[l][o]) < 1e-6 * max(1.0, abs(db[l][o]))


def test_adam_first_step_closed_form():
    """At t = 1 the bias corrections undo (1 - beta): the step is -lr g / (|g| + eps)."""
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    th, m, v = sg.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.max(np.abs(th - (-0.01 * g / (np.abs(g) + 1e-8)))) < 1e-15
    assert np.allclose(m, (1 - 0.9) * g, rtol=1e-15, atol=0)
    assert np.allclose(v, (1 - 0.999) * g * g, rtol=1e-15, atol=0)


def test_bf16_rounding_values():
    """BF16 keeps 8 significant bits: 1 + 2^-8 is a tie that rounds to even (1), 1 + 3 2^-8
    rounds up to 1 + 2^-6, 1 + 2^-7 is exact, and -0.1 rounds to -0.10009765625."""
    x = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 1 + 2.0 ** -7, -0.1])
    assert list(sg.bf16(x)) == [1.0, 1 + 2.0 ** -6, 1 + 2.0 ** -7, -0.10009765625]


# ------------------------------------------------------------------ rendering
def _seabed_wall_scene(h=3.0, D=6.0):
    """Mirror seabed at z = -h (20 x 20 m) and a non-mirror wall at x = D."""
    sea = np.array([[-10, -10, -h], [10, -10, -h], [10, 10, -h], [-10, 10, -h]], np.float32)
    wall = np.array([[D, -10, -h - 1], [D, 10, -h - 1], [D, 10, 2], [D, -10, 2]], np.float32)
    v = np.concatenate([sea, wall])
    t = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]], np.int32)
    return inputs.Scene(v, t, np.array([0.3, 0.3, 0.5, 0.5], np.float32), np.array([1, 1, 0, 0], np.uint8))


def test_render_matches_closed_form_routes():
    """Flat mirror seabed h below the sonar and a wall at x = D: a beam with world
    direction u that meets the wall first has L1 = D / u_x, kappa1 = u_x; one that meets
    the seabed first has L1 = h / -u_z, kappa1 = -u_z, and its reflected ray (u_x, u_y,
    -u_z) meets the wall at L2 = D / u_x, kappa2 = u_x, Gamma2 = r_seabed."""
    h, D = 3.0, 6.0
    sc = _seabed_wall_scene(h, D)
    p = dict(inputs.sensor_params("c1"), surface_z=math.nan, r_max=10.0, n_range=512, r_seabed=0.5)
    ps = inputs.pose((0.0, 0.0, 0.0), tilt_down_deg=10.0)
    feat = sg.render(sc, p, ps, inputs.ssp("c1"))
    R = inputs._rot(ps["q"])
    nba, nbe = p["n_beam_az"], p["n_beam_el"]
    L_stop = p["r_max"] + 1500.0 * p["pulse"] / 2
    checked = [0, 0]
    for j in range(nbe):
        for i in range(nba):
            az = -p["hfov"] / 2 + (i + 0.5) * p["hfov"] / nba
            el = -p["vfov"] / 2 + (j + 0.5) * p["vfov"] / nbe
            u = R @ np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
            f = feat[j * nba + i]
            t_wall = D / u[0]
            t_sea = h / -u[2] if u[2] < 0 else math.inf
            if t_wall < t_sea and t_wall < L_stop:
                assert abs(f[0] - t_wall) < 1e-12 and abs(f[1] - u[0]) < 1e-12
                assert f[2] == np.float32(0.5) and f[3] == 1.0 and f[4] == 0.0
                checked[0] += 1
            elif t_sea < t_wall and D / u[0] < L_stop:
                assert abs(f[0] - t_sea) < 1e-12 and abs(f[1] + u[2]) < 1e-12
                assert f[2] == np.float32(0.3) and f[3] == 1.0
                assert abs(f[4] - D / u[0]) < 1e-12 and abs(f[5] - u[0]) < 1e-12
                assert f[6] == np.float32(0.5) and f[7] == 0.5
                checked[1] += 1
    assert min(checked) > 50


def test_rasterize_hand_example():
    """dr = 1 m: a first hit at L = 2.75 sits at x = 2.25 -> bins 2, 3 with 0.75, 0.25;
    a second hit at L = 5.5 sits exactly on bin 5."""
    p = {"n_range": 8, "r_min": 0.0, "r_max": 8.0}
    feat = np.array([[2.75, 0.8, 0.4, 1.0, 5.5, 0.5, 0.2, 0.5]])
    X = sg.rasterize(feat, p)[0]
    want = np.zeros((8, 4))
    want[2] = (0.75, 0, 0.75 * 0.8, 0.75 * 0.4)
    want[3] = (0.25, 0, 0.25 * 0.8, 0.25 * 0.4)
    want[5] = (0, 1.0, 0.5, 0.2)
    assert np.max(np.abs(X - want)) < 1e-15


def test_geometric_envelope_single_hit():
    """One beam, one hit on a bin centre after a reflection of coefficient 0.5: E at that
    bin is Gamma^2 sqrt(mu kappa dOmega)/L |R(0)| r with R(0) = 1 (Gamma^2 = 1/4); one
    pulse length away it vanishes."""
    p = dict(inputs.sensor_params("c1"), n_beam_az=1, n_beam_el=1, hfov=0.1, vfov=0.05, n_range=64,
             r_max=6.4, alpha=0.0)
    L = 3.05  # bin 30's centre
    feat = np.array([[L, 0.6, 0.3, 0.5, 0, 0, 0, 0]])
    E = sg.geometric_envelope(feat, p, 1500.0)[0]
    domega = 0.1 * 2 * math.sin(0.025)
    assert abs(E[30] - 0.25 * math.sqrt(0.3 * 0.6 * domega) / L * L) < 1e-12
    assert E[30] == E.max() and E[0] == 0.0


def test_beam_metrics_cases():
    rng = np.random.default_rng(5)
    E_ref = np.abs(rng.normal(size=(40, 64)) + 1j * rng.normal(size=(40, 64)))
    m = sg.beam_metrics(E_ref, E_ref, 2, 0.0)
    assert m["nl2"] == 0 and np.all(m["peak_bins"] == 0) and m["si"] == m["si_ref"]
    # fully developed speckle: complex Gaussian amplitudes have exponential intensity, SI -> 1
    big = np.abs(rng.normal(size=(400, 512)) + 1j * rng.normal(size=(400, 512)))
    assert abs(sg.beam_metrics(big, big, 0, 0.0)["si"] - 1.0) < 0.02
    shifted = np.roll(E_ref, 2, axis=1)
    d = sg.beam_metrics(shifted, E_ref, 0, 0.0)["peak_bins"]
    am = np.argmax(E_ref, axis=1)
    assert np.all(d[am < 62] == 2)
