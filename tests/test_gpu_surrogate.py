"""GPU parity of the learned surrogate (the CUDA kernels through the C ABI) against the
FP64 oracle in oracle/surrogate.py.

Tolerances. The rendering stores lengths, cosines and reflection products in FP32: L to
2e-6 relative, the incidence cosine to 2e-6, reflectivity and reflection products exactly.
The network's forward and backward passes are compared with the oracle in two ways:
- against the oracle with BF16 rounding at the same storage points (activations a1..a5,
  gradients dz1..dz5): the two differ by FP32 against FP64 accumulation only, so a stored
  BF16 value differs by one BF16 step where the FP32 and FP64 sums straddle a rounding
  boundary (a few in 10^5 of the values). Output to 1e-3 normalised L2, weight gradients
  to 5e-3 per layer;
- against the plain FP64 oracle: BF16 storage adds a relative error of about 2^-9 per
  stored value, which six layers compound to a few 1e-3: output to 2e-2, gradients to
  5e-2 per layer.
Adam's step against the oracle's on the GPU's own gradient: to 1e-3 of the learning rate.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import surrogate as sg
from paper_2606_06130_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sonar():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06130_gb300.sonar import Sonar
    s = Sonar(0)
    yield s
    s.close()


def _c1_sur():
    """The C1 sensor with its range axis kept at 256 bins (a multiple of 256) and a wall
    over the mirror seabed, so that beams carry first and second hits."""
    scene, params, poses, ssp = inputs.workload("wall_mirror")
    params = dict(params, n_range=256, r_max=10.0, surface_z=0.0)
    return scene, params, poses[0], ssp


def _feat_np(feat_gpu):
    return np.asarray(feat_gpu, np.float64)


# ------------------------------------------------------------------ rendering
@pytest.mark.parametrize("name", ["wall_mirror", "c2", "train"])
def test_render_parity(sonar, name):
    if name == "wall_mirror":
        scene, params, pose, ssp = _c1_sur()
    elif name == "c2":
        scene, params, poses, ssp = inputs.workload("c2")
        pose = poses[0]
    else:
        scene = inputs.training_scene(101)
        params, ssp = inputs.sensor_params("c2"), inputs.ssp("c2")
        pose = inputs.training_poses(102, 4, scene)[2]  # far enough from the wall to see the seabed
    sonar.upload(scene)
    got = _feat_np(sonar.sur_render([pose], params, ssp)[0])
    want, clear = sg.render(scene, params, pose, ssp, with_ties=True)
    n_hits_g = (got[:, 0] > 0).astype(int) + (got[:, 4] > 0)
    n_hits_w = (want[:, 0] > 0).astype(int) + (want[:, 4] > 0)
    same = clear & (n_hits_g == n_hits_w)
    # beams whose route passes within the FP32 slack of an edge may end differently
    assert np.count_nonzero(clear & (n_hits_g != n_hits_w)) <= 2
    assert np.count_nonzero(same & (n_hits_w > 0)) > 0.5 * len(got)
    g, w = got[same], want[same]
    for h in range(2):
        has = w[:, 4 * h] > 0
        assert np.max(np.abs(g[has, 4 * h] - w[has, 4 * h]) / w[has, 4 * h], initial=0) < 2e-6
        assert np.max(np.abs(g[has, 4 * h + 1] - w[has, 4 * h + 1]), initial=0) < 2e-6
        assert np.array_equal(g[has, 4 * h + 2], np.float32(w[has, 4 * h + 2]).astype(np.float64))
        assert np.array_equal(g[has, 4 * h + 3], w[has, 4 * h + 3])
    if name != "c2":
        assert np.count_nonzero(w[:, 4] > 0) > 20  # second hits present


# ------------------------------------------------------------------ network
def _oracle_forward(theta, feat_rows, params, bf16):
    """Oracle output yhat [beams, n_range] for rendering rows (the GPU's, so that only the
    network is compared), with the network's BF16 weights."""
    net = inputs.surrogate_unpack(theta)
    net["W"] = [sg.bf16(W) for W in net["W"]]
    x0 = sg.rasterize(feat_rows, params)
    acts, yhat = sg.forward(net, x0, bf16_storage=bf16)
    return net, acts, yhat


@pytest.mark.parametrize("name", ["wall_mirror", "c2"])
def test_forward_parity(sonar, name):
    """sonar_sur_ping against the oracle network on the GPU's own rendering, on 96 sampled
    beams (wall_mirror) or 24 sampled beams of the full C2 ping, half of them with second
    hits."""
    if name == "wall_mirror":
        scene, params, pose, ssp = _c1_sur()
    else:
        scene, params, poses, ssp = inputs.workload("c2")
        pose = poses[0]
    sonar.upload(scene)
    theta = inputs.surrogate_init(5)
    theta[inputs.SUR_CHANNELS[0] * 64 * 9:][:64] = 0.05  # non-zero first-layer biases
    e_scale = 0.02
    sonar.sur_set_weights(theta, e_scale)
    env = sonar.sur_ping([pose], params, ssp)
    torch.cuda.synchronize()
    E = env.reshape(-1, params["n_range"]).double().cpu().numpy()
    feat = _feat_np(sonar.sur_render([pose], params, ssp)[0])
    rng = np.random.default_rng(3)
    k = 48 if name == "wall_mirror" else 12
    beams = np.sort(np.concatenate([rng.choice(np.nonzero(feat[:, 4] > 0)[0], k, replace=False),
                                    rng.choice(np.nonzero(feat[:, 4] == 0)[0], k, replace=False)]))
    for bf16, tol in ((True, 1e-3), (False, 2e-2)):
        _, _, yhat = _oracle_forward(theta, feat[beams], params, bf16)
        err = parity.nl2(E[beams], e_scale * yhat)
        assert err < tol, (bf16, err)


def test_gradient_and_adam_parity(sonar):
    """sonar_sur_train_step on 40 selected beams (device indices): the gradient of every
    layer's weights and biases against the oracle's backward pass, then one Adam step
    against the oracle's Adam on the GPU's gradient."""
    scene, params, pose, ssp = _c1_sur()
    sonar.upload(scene)
    env_ref, _, _ = sonar.ping_batch([pose], params, ssp)
    torch.cuda.synchronize()
    theta = inputs.surrogate_init(7)
    e_scale = float(env_ref.double().pow(2).mean().sqrt().item()) * 3
    sonar.sur_set_weights(theta, e_scale)
    feat = _feat_np(sonar.sur_render([pose], params, ssp)[0])
    rng = np.random.default_rng(9)
    lit = np.nonzero(feat[:, 0] > 0)[0]
    sel = np.sort(rng.choice(lit, 40, replace=False)).astype(np.int32)
    beams = torch.from_numpy(sel).to("cuda:0")
    loss, grad = sonar.sur_train_step([pose], params, ssp, env_ref, beams, update=False, want_grad=True)
    y = env_ref.reshape(-1, params["n_range"]).double().cpu().numpy()[sel] / e_scale
    for bf16, tol in ((True, 5e-3), (False, 5e-2)):
        net, acts, yhat = _oracle_forward(theta, feat[sel], params, bf16)
        assert abs(loss - sg.loss(yhat, y)) < (1e-3 if bf16 else 2e-2) * sg.loss(yhat, y)
        dW, db = sg.backward(net, acts, yhat, y, bf16_storage=bf16)
        g = inputs.surrogate_unpack(grad)
        for l in range(6):
            e_w = parity.nl2(g["W"][l], dW[l])
            e_b = parity.nl2(g["b"][l], db[l])
            assert e_w < tol and e_b < tol, (bf16, l, e_w, e_b)
    # one Adam step on the same batch: theta - lr m^ / (sqrt(v^) + eps) with the GPU's gradient
    lr = 1e-3
    sonar.sur_train_step([pose], params, ssp, env_ref, beams, lr=lr, update=True)
    new = sonar.sur_get_weights().astype(np.float64)
    want, _, _ = sg.adam(theta.astype(np.float64), grad.astype(np.float64), np.zeros(len(theta)),
                         np.zeros(len(theta)), 1, lr)
    assert np.max(np.abs(new - want)) < 1e-3 * lr


def test_train_step_rejects_bad_inputs(sonar):
    from paper_2606_06130_gb300.sonar import SonarError, SONAR_E_ARG, SONAR_E_UNSUPPORTED
    scene, params, pose, ssp = _c1_sur()
    sonar.upload(scene)
    sonar.sur_set_weights(inputs.surrogate_init(1), 1.0)
    env_ref, _, _ = sonar.ping_batch([pose], params, ssp)
    nb = params["n_beam_az"] * params["n_beam_el"]
    bad = torch.tensor([0, nb], dtype=torch.int32, device="cuda:0")  # nb is one past the last beam
    with pytest.raises(SonarError) as e:
        sonar.sur_train_step([pose], params, ssp, env_ref, bad, update=False)
    assert e.value.code == SONAR_E_ARG
    with pytest.raises(SonarError) as e:
        sonar.sur_train_step([pose], params, ssp, env_ref.cpu(), None, update=False)
    assert e.value.code == SONAR_E_ARG
    with pytest.raises(SonarError) as e:
        sonar.sur_ping([pose], dict(params, n_range=200), ssp)
    assert e.value.code == SONAR_E_UNSUPPORTED
    with pytest.raises(SonarError) as e:
        sonar.sur_ping([pose], params, inputs.ssp("c3"))
    assert e.value.code == SONAR_E_UNSUPPORTED


def test_compare_metrics_match_oracle(sonar):
    """sonar_sur_compare against the oracle's metric definitions on two volumes."""
    scene, params, pose, ssp = _c1_sur()
    sonar.upload(scene)
    env_ref, _, _ = sonar.ping_batch([pose], params, ssp)
    sonar.sur_set_weights(inputs.surrogate_init(2), float(env_ref.max().item()))
    env = sonar.sur_ping([pose], params, ssp)
    torch.cuda.synchronize()
    m = sonar.sur_compare(env, env_ref, params, 0.1)
    E = env.reshape(-1, params["n_range"]).double().cpu().numpy()
    R = env_ref.reshape(-1, params["n_range"]).double().cpu().numpy()
    ref = sg.beam_metrics(E, R, parity.n_blank(params), 0.1)
    assert abs(m["nl2"] - ref["nl2"]) < 1e-6 * ref["nl2"]
    assert m["lit_beams"] == len(ref["peak_bins"])
    assert abs(m["peak_bin_mean"] - ref["peak_bins"].mean()) < 1e-9
    assert abs(m["si_ref"] - ref["si_ref"]) < 1e-6 * abs(ref["si_ref"])
    assert abs(m["si"] - ref["si"]) < 1e-6 * abs(ref["si"])
