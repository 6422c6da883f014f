"""GPU raw element series and matched filter (Sec. II.B time series) against the FP64
oracle, through the C ABI.

With SONAR_OPT_RAW = U the library synthesises the raw echo of the transmitted chirp at U
samples per range cell and compresses it with an explicit matched filter before
beamforming. Checked: every phase of the raw series against the oracle's raw series
(FP32 form, S_TOL), the matched-filter output against the oracle's matched filter
(S_TOL) and against the compressed echoes (the quadrature error), the envelope of the
raw path against the oracle's, and the option's argument checks.
"""
import numpy as np
import pytest

import oracle
from paper_2606_06130_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

S_TOL = 5e-5


@pytest.fixture(scope="module")
def sonar():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06130_gb300.sonar import Sonar, SONAR_OPT_DEBUG
    s = Sonar(0)
    s.set_option(SONAR_OPT_DEBUG, 1)
    yield s
    s.close()


def run(s, scene, params, pose, ssp, U, precision="fp32"):
    from paper_2606_06130_gb300.sonar import SONAR_OPT_RAW
    s.set_option(SONAR_OPT_RAW, U)
    try:
        s.upload(scene)
        env, cloud, n = s.ping(pose, params, ssp, precision=precision)
        torch.cuda.synchronize()
        out = (env.reshape(-1, params["n_range"]).double().cpu().numpy(), s.echoes(params)[0],
               [s.raw(params, k)[0] for k in range(U)] if U else [])
    finally:
        s.set_option(SONAR_OPT_RAW, 0)
    return out


def c1(**over):
    scene, params, poses, ssp = inputs.workload("c1")
    return scene, dict(params, **over), poses[0], ssp


@pytest.mark.parametrize("U,nx,ny", [(1, 8, 8), (4, 8, 8), (3, 16, 16), (4, 12, 12)])
def test_raw_phases_match_oracle(sonar, U, nx, ny):
    """8x8 and 16x16 arrays take the two tensor-core kernels, 12x12 the FP32 SIMT kernel."""
    scene, params, pose, ssp = c1(nx=nx, ny=ny, n_beam_az=24, n_beam_el=12)
    _, _, raw = run(sonar, scene, params, pose, ssp, U)
    h = oracle.trace(scene, params, pose, ssp)
    ref = oracle.raw_echoes(params, h, U, np.arange(params["n_range"]))
    for s in range(U):
        assert parity.nl2(raw[s], ref[s]) < S_TOL, (s, parity.nl2(raw[s], ref[s]))


def test_matched_filter_matches_oracle_and_the_compressed_echoes(sonar):
    scene, params, pose, ssp = c1()
    U = 4
    E, y, _ = run(sonar, scene, params, pose, ssp, U)
    h = oracle.trace(scene, params, pose, ssp)
    ns = np.arange(params["n_range"])
    y_ref = oracle.matched_filter(params, h, U, ns)
    assert parity.nl2(y, y_ref) < S_TOL
    # the compressed path of the same scene: equal to the quadrature error at U = 4
    E0, s0, _ = run(sonar, scene, params, pose, ssp, 0)
    assert parity.nl2(y, s0) < 4e-4
    # envelope of the raw path against the oracle's envelope of its matched filter
    B = oracle.beamform(params, h["c_ref"], y_ref)
    E_ref = oracle.envelope(params, B, ns)
    assert parity.nl2(E, E_ref) < 1e-4
    assert parity.nl2(E, E0) < 4e-4


def test_raw_path_batch_equals_single_pings(sonar):
    from paper_2606_06130_gb300.sonar import SONAR_OPT_RAW
    scene, params, pose0, ssp = c1()
    poses = [inputs.pose(pose0["t"] + np.array([0.1 * k, 0.0, 0.0]), yaw_deg=-5.0 + 6.0 * k,
                         tilt_down_deg=15.0, roll_deg=0.0) for k in range(3)]
    sonar.set_option(SONAR_OPT_RAW, 2)
    try:
        sonar.upload(scene)
        env_b, _, _ = sonar.ping_batch(poses, params, ssp)
        torch.cuda.synchronize()
        env_b = env_b.reshape(len(poses), -1, params["n_range"]).double().cpu().numpy()
        for k, ps in enumerate(poses):
            env, _, _ = sonar.ping(ps, params, ssp)
            torch.cuda.synchronize()
            assert parity.nl2(env_b[k], env.reshape(-1, params["n_range"]).double().cpu().numpy()) < 1e-6
    finally:
        sonar.set_option(SONAR_OPT_RAW, 0)


def test_raw_option_arguments(sonar):
    from paper_2606_06130_gb300.sonar import SONAR_OPT_RAW, SonarError
    with pytest.raises(SonarError) as e:
        sonar.set_option(SONAR_OPT_RAW, 9)
    assert e.value.code == -1  # SONAR_E_ARG
    scene, params, pose, ssp = c1()
    run(sonar, scene, params, pose, ssp, 2)
    with pytest.raises(SonarError):
        sonar.raw(params, 2)  # phases 0 and 1 only


def test_c2_raw_path_equals_compressed_to_quadrature_error(sonar):
    """Full-size harbour ping (534k hits, 32x32 array): the raw path at U = 4 against the
    compressed path, envelope and element echoes, all beams and bins."""
    scene, params, poses, ssp = inputs.workload("c2")
    E4, y4, _ = run(sonar, scene, params, poses[0], ssp, 4)
    E0, s0, _ = run(sonar, scene, params, poses[0], ssp, 0)
    assert parity.nl2(y4, s0) < 4e-4
    assert parity.nl2(E4, E0) < 4e-4
