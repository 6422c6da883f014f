"""GPU parity of the separable phase-shift beamformer against the FP64 oracle, through
the C ABI.

With a separable taper w_m = wy[my] wx[mx], the steering phase of element (mx, my) is
u_y y_mx + u_z z_my and u_z = sin(el) depends only on the beam's elevation row, so the
library forms the beams in two stages (a sum over the array's rows per elevation, then
the tensor-core contraction over its columns). The oracle sums over all elements in one
step. Checked: the two-stage beams against the oracle's dense beamformer (uniform and
Hann x Hann tapers, FP32 and BF16 forms), against the library's own dense contraction on
the same ping (C1 scene on a wide beam grid, and the full C2 ping), and that every case
outside the separable form's conditions falls back to the dense contraction.
"""
import numpy as np
import pytest

import oracle
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


def wide(**over):
    """The C1 scene seen by a 16 x 16 array on a 64 x 8 beam grid (rows of 64 beams, so
    the contraction's N tile of 128 columns lies in one elevation row)."""
    scene, params, poses, ssp = inputs.workload("c1")
    params = dict(params, nx=16, ny=16, n_beam_az=64, n_beam_el=8)
    params.update(over)
    return scene, params, poses[0], ssp


def hann(n):
    return 0.5 - 0.5 * np.cos(2 * np.pi * (np.arange(n) + 0.5) / n)


def ping(s, scene, params, pose, ssp, dense=False, precision="fp32", taper=None):
    from paper_2606_06130_gb300.sonar import SONAR_OPT_BEAMFORM
    s.set_option(SONAR_OPT_BEAMFORM, 1 if dense else 0)
    try:
        s.upload(scene)
        env, cloud, n = s.ping(pose, params, ssp, precision=precision, taper=taper)
        torch.cuda.synchronize()
        st = s.stats()
    finally:
        s.set_option(SONAR_OPT_BEAMFORM, 0)
    return env.reshape(-1, params["n_range"]).double().cpu().numpy(), st


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("bf16", 1e-2)])
@pytest.mark.parametrize("tapered", [False, True])
def test_separable_beams_match_oracle(sonar, precision, tol, tapered):
    scene, params, pose, ssp = wide()
    taper = np.outer(hann(params["ny"]), hann(params["nx"])).astype(np.float32).ravel() if tapered else None
    E, st = ping(sonar, scene, params, pose, ssp, precision=precision, taper=taper)
    assert st["beam_sep"] == 1
    ref = oracle.trace(scene, params, pose, ssp)
    E_ref, _, _ = oracle.volume(params, ref, taper=taper)
    assert parity.nl2(E, E_ref) <= tol, parity.nl2(E, E_ref)


def test_separable_equals_dense_contraction(sonar):
    scene, params, pose, ssp = wide()
    E_sep, st_sep = ping(sonar, scene, params, pose, ssp)
    E_den, st_den = ping(sonar, scene, params, pose, ssp, dense=True)
    assert st_sep["beam_sep"] == 1 and st_den["beam_sep"] == 0
    # both carry the FP32 form's ~1e-5 representation error against the oracle
    assert parity.nl2(E_sep, E_den) <= 3e-5, parity.nl2(E_sep, E_den)


def test_c2_separable_equals_dense(sonar):
    """The full harbour-wall ping: 8192 beams x 1024 bins from a 32 x 32 array."""
    scene, params, poses, ssp = inputs.workload("c2")
    E_sep, st_sep = ping(sonar, scene, params, poses[0], ssp)
    E_den, st_den = ping(sonar, scene, params, poses[0], ssp, dense=True)
    assert st_sep["beam_sep"] == 1 and st_den["beam_sep"] == 0
    assert parity.nl2(E_sep, E_den) <= 3e-5, parity.nl2(E_sep, E_den)
    # per-beam peak bins agree wherever the peak clears its runner-up by 1e-3
    nb = parity.n_blank(params)
    top2 = np.sort(E_den[:, nb:], axis=1)[:, -2:]
    clear = top2[:, 1] > (1 + 1e-3) * top2[:, 0]
    assert np.count_nonzero(clear) > 0.5 * E_den.shape[0]
    assert np.array_equal(np.argmax(E_sep[clear, nb:], axis=1), np.argmax(E_den[clear, nb:], axis=1))


def test_outside_the_conditions_the_dense_contraction_runs(sonar):
    from paper_2606_06130_gb300.sonar import SONAR_OPT_TILE_N
    scene, params, pose, ssp = wide()
    rng = np.random.default_rng(5)
    # a taper no row x column product reproduces
    taper = rng.uniform(0.2, 1.0, params["nx"] * params["ny"]).astype(np.float32)
    E, st = ping(sonar, scene, params, pose, ssp, taper=taper)
    assert st["beam_sep"] == 0
    ref = oracle.trace(scene, params, pose, ssp)
    E_ref, _, _ = oracle.volume(params, ref, taper=taper)
    assert parity.nl2(E, E_ref) <= 1e-4
    # FP16 operands, rows of 32 beams, and a caller's N tile that crosses elevation rows
    assert ping(sonar, scene, params, pose, ssp, precision="fp16")[1]["beam_sep"] == 0
    s2, p2, pose2, ssp2 = wide(n_beam_az=32, n_beam_el=16)
    assert ping(sonar, s2, p2, pose2, ssp2)[1]["beam_sep"] == 0
    sonar.set_option(SONAR_OPT_TILE_N, 224)
    try:
        assert ping(sonar, scene, params, pose, ssp)[1]["beam_sep"] == 0
    finally:
        sonar.set_option(SONAR_OPT_TILE_N, 0)


def test_beamform_option_arguments(sonar):
    from paper_2606_06130_gb300.sonar import SONAR_OPT_BEAMFORM, SonarError
    with pytest.raises(SonarError):
        sonar.set_option(SONAR_OPT_BEAMFORM, 2)


def test_ragged_range_and_batch_mirrored_rows(sonar):
    """64 elevation rows (the mirrored-row first stage), an odd number of range bins (each
    ping's last two-sample unit holds one sample), and six pings in one call, so that
    every first-stage CTA takes several units and refills both halves of its S buffer."""
    scene, params, pose, ssp = wide(n_beam_el=64, n_range=333)
    from paper_2606_06130_gb300.sonar import SONAR_OPT_BEAMFORM
    sonar.set_option(SONAR_OPT_BEAMFORM, 0)
    sonar.upload(scene)
    P = 6
    env, _, n = sonar.ping_batch([pose] * P, params, ssp, precision="fp32")
    torch.cuda.synchronize()
    assert sonar.stats()["beam_sep"] == 1
    ref = oracle.trace(scene, params, pose, ssp)
    E_ref, _, _ = oracle.volume(params, ref)
    E = env.reshape(P, -1, params["n_range"]).double().cpu().numpy()
    for i in range(P):
        assert parity.nl2(E[i], E_ref) <= 1e-4, (i, parity.nl2(E[i], E_ref))
    assert np.all(n == n[0])
