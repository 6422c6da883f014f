"""GPU parity of water-column (volume) reverberation (sonar_set_volume) against the FP64
oracle: hit lists (keys bit-exact, delays 1e-12, amplitudes and phases 2e-6), element
echoes within 5e-5 and envelopes within 1e-4 normalised L2 (FP32 form)."""
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
    s.set_volume(0)
    s.close()


def _vol(params, n, lo, hi, sv):
    return dict(params, vol_n=n, vol_lo=lo, vol_hi=hi, vol_sv=sv)


def _volume_keys(keys):
    k = keys.astype(np.uint64)
    return int(np.count_nonzero((k & np.uint64(0xF0000000)) == np.uint64(0xA0000000)))


def test_volume_only_parity(sonar):
    scene = inputs.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.float32),
                         np.zeros(0, np.uint8))
    params = dict(inputs.sensor_params("c1"), surface_z=None, max_bounces=0, n_ray_az=4, n_ray_el=2, r_max=4.0)
    pose = inputs.pose((0.0, 0.0, -10.0), tilt_down_deg=10.0)
    lo, hi = (-4.0, -4.0, -14.0), (4.0, 4.0, -6.0)
    sonar.upload(scene)
    sonar.set_volume(100_000, lo, hi, 1e-3)
    try:
        env, _, _ = sonar.ping(pose, params, inputs.ssp("c1"))
        torch.cuda.synchronize()
        hits = sonar.hits()
        s_gpu = sonar.echoes(params)[0]
    finally:
        sonar.set_volume(0)
    E = env.reshape(-1, params["n_range"]).double().cpu().numpy()
    ref = oracle.trace(scene, _vol(params, 100_000, lo, hi, 1e-3), pose, inputs.ssp("c1"))
    assert ref["n"] > 20000 and _volume_keys(hits["key"]) == ref["n"]
    parity.check_hits(hits, ref, params["n_sub"], per_tie=0)
    E_ref, _, s_ref = oracle.volume(params, ref)
    assert parity.nl2(s_gpu, s_ref) < S_TOL
    assert parity.nl2(E, E_ref) <= 1e-4


def test_volume_with_mesh_cross_terms_and_shadowing(sonar):
    from paper_2606_06130_gb300.sonar import SONAR_OPT_CROSS
    scene, params, poses, ssp = inputs.workload("wall_mirror")
    lo, hi = (-1.0, -4.0, -4.0), (8.0, 4.0, 0.0)
    sonar.upload(scene)
    sonar.set_volume(50_000, lo, hi, 2e-3)
    sonar.set_option(SONAR_OPT_CROSS, 1)
    try:
        env, _, _ = sonar.ping(poses[0], params, ssp)
        torch.cuda.synchronize()
        hits = sonar.hits()
    finally:
        sonar.set_volume(0)
        sonar.set_option(SONAR_OPT_CROSS, 0)
    E = env.reshape(-1, params["n_range"]).double().cpu().numpy()
    ref = oracle.trace(scene, _vol(dict(params, cross=1), 50_000, lo, hi, 2e-3), poses[0], ssp)
    n_vol_ref = int(np.count_nonzero(ref["sub"] == 0x20000))
    assert _volume_keys(hits["key"]) == n_vol_ref
    # the wall hides the scatterers behind it and the plate a cone of them
    assert n_vol_ref < 0.8 * 50_000
    parity.check_hits(hits, ref, params["n_sub"], per_tie=6)
    E_ref, _, _ = oracle.volume(params, ref)
    assert parity.nl2(E, E_ref) <= 1e-4


def test_volume_c2_sampled_parity_and_batch(sonar):
    scene, params, poses, ssp = inputs.workload("c2")
    lo, hi = (-2.0, -12.0, -10.5), (14.0, 12.0, -4.0)
    n, sv = 1_000_000, 1e-4
    ps = [poses[0], inputs.pose((0.3, -0.2, -8.1), yaw_deg=4.0, tilt_down_deg=11.0)]
    sonar.upload(scene)
    sonar.set_volume(n, lo, hi, sv)
    try:
        env, _, _ = sonar.ping_batch(ps, params, ssp)
        torch.cuda.synchronize()
    finally:
        sonar.set_volume(0)
    env = env.reshape(len(ps), -1, params["n_range"]).double().cpu().numpy()
    rng = np.random.default_rng(17)
    ns = np.unique(rng.integers(0, params["n_range"], 20)).astype(np.int32)
    for i, pose in enumerate(ps):
        ref = oracle.trace(scene, _vol(params, n, lo, hi, sv), pose, ssp)
        assert np.count_nonzero(ref["sub"] == 0x20000) > 100_000
        E_ref, _, _ = oracle.volume(params, ref, ns=ns)
        assert parity.nl2(env[i][:, ns], E_ref) <= 1e-4, i


def test_set_volume_rejects_bad_arguments(sonar):
    from paper_2606_06130_gb300.sonar import SonarError, SONAR_E_ARG, SONAR_E_UNSUPPORTED
    for args in [(10, (0, 0, 0), (1, 0, 1), 1e-3), (-1, (0, 0, 0), (1, 1, 1), 1e-3),
                 (10, (0, 0, 0), (1, 1, 1), -1.0), ((1 << 28) + 1, (0, 0, 0), (1, 1, 1), 1e-3)]:
        with pytest.raises(SonarError) as e:
            sonar.set_volume(*args)
        assert e.value.code == SONAR_E_ARG
    scene, params, poses, ssp = inputs.workload("c3")
    sonar.upload(scene)
    sonar.set_volume(10, (-1, -1, -3), (1, 1, -1), 1e-3)
    try:
        with pytest.raises(SonarError) as e:
            sonar.ping(poses[0], params, ssp)
        assert e.value.code == SONAR_E_UNSUPPORTED
    finally:
        sonar.set_volume(0)


def test_volume_degenerate_cases(sonar):
    """One scatterer; a box beyond the range (no echoes); a zero s_v (echoes of zero
    amplitude): each against the oracle."""
    scene = inputs.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.float32),
                         np.zeros(0, np.uint8))
    params = dict(inputs.sensor_params("c1"), surface_z=None, max_bounces=0, n_ray_az=4, n_ray_el=2, r_max=4.0)
    pose = inputs.pose((0.0, 0.0, -10.0))
    sonar.upload(scene)
    for n, lo, hi, sv in [(1, (1.0, -0.5, -10.5), (2.0, 0.5, -9.5), 1e-2),
                          (500, (50.0, 50.0, 0.0), (60.0, 60.0, 10.0), 1e-3),
                          (200, (-2.0, -2.0, -12.0), (2.0, 2.0, -8.0), 0.0)]:
        sonar.set_volume(n, lo, hi, sv)
        try:
            env, _, _ = sonar.ping(pose, params, inputs.ssp("c1"))
            torch.cuda.synchronize()
            hits = sonar.hits()
        finally:
            sonar.set_volume(0)
        ref = oracle.trace(scene, _vol(params, n, lo, hi, sv), pose, inputs.ssp("c1"))
        assert _volume_keys(hits["key"]) == ref["n"]
        if ref["n"] and sv > 0:  # zero amplitudes have no relative error to compare
            parity.check_hits(hits, ref, params["n_sub"], per_tie=0)
        E = env.reshape(-1, params["n_range"]).double().cpu().numpy()
        E_ref, _, _ = oracle.volume(params, ref)
        if np.linalg.norm(E_ref) > 0:
            assert parity.nl2(E, E_ref) <= 1e-4
        else:
            assert np.all(E == 0.0)
