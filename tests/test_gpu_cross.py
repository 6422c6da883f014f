"""GPU parity of out/back cross-term multipath (SONAR_OPT_CROSS) against the FP64 oracle.

Same bars as the plain path: prim ids bit-exact outside the near-tie margins, delays to
1e-12 relative, amplitudes and phases to 2e-6, arrival directions to 1e-6; element
echoes within 5e-5 and the envelope within 1e-4 normalised L2 (FP32 form).
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
    from paper_2606_06130_gb300.sonar import Sonar, SONAR_OPT_DEBUG, SONAR_OPT_CROSS
    s = Sonar(0)
    s.set_option(SONAR_OPT_DEBUG, 1)
    s.set_option(SONAR_OPT_CROSS, 1)
    yield s
    s.close()


def _ping(s, scene, params, pose, ssp, precision="fp32"):
    s.upload(scene)
    env, cloud, n = s.ping(pose, params, ssp, precision=precision)
    torch.cuda.synchronize()
    return env.reshape(-1, params["n_range"]).double().cpu().numpy()


def _cross_counts(keys):
    k = keys.astype(np.uint64)
    mesh = (k & np.uint64(0x80000000)) == 0
    return (int(np.count_nonzero(mesh & ((k & np.uint64(0x40000000)) != 0))),
            int(np.count_nonzero(mesh & ((k & np.uint64(0x20000000)) != 0))),
            int(np.count_nonzero((k & np.uint64(0xC0000000)) == np.uint64(0xC0000000))))


def test_wall_mirror_cross_parity(sonar):
    scene, params, poses, ssp = inputs.workload("wall_mirror")
    E = _ping(sonar, scene, params, poses[0], ssp)
    ref = oracle.trace(scene, dict(params, cross=1), poses[0], ssp)
    hits = sonar.hits()
    excluded, matched = parity.check_hits(hits, ref, params["n_sub"], per_tie=6)
    assert matched == ref["n"]
    d, r, pairs = _cross_counts(hits["key"])
    assert d == r == int(np.count_nonzero(ref["seg"] == 17)) > 300
    assert pairs == 6  # three points, two routes each: two ordered pairs per point
    E_ref, _, s_ref = oracle.volume(params, ref)
    assert parity.nl2(sonar.echoes(params)[0], s_ref) < S_TOL
    assert parity.nl2(E, E_ref) <= 1e-4
    # the cross terms change the volume: the plain oracle is far from it
    E_mono, _, _ = oracle.volume(params, oracle.trace(scene, params, poses[0], ssp))
    assert parity.nl2(E_mono, E_ref) > 1e-2


def test_c2_cross_sampled_parity(sonar):
    scene, params, poses, ssp = inputs.workload("c2")
    E = _ping(sonar, scene, params, poses[0], ssp)
    ref = oracle.trace(scene, dict(params, cross=1), poses[0], ssp)
    excluded, matched = parity.check_hits(sonar.hits(), ref, params["n_sub"], per_tie=6)
    assert matched >= ref["n"] - 6 * (excluded + 1)
    assert np.count_nonzero(ref["seg"] >= 16) > 10000
    dr = params["r_max"] / params["n_range"]
    n_hit = np.floor(ref["tau"] * ref["c_ref"] / 2 / dr).astype(int)
    dense = np.argsort(np.bincount(n_hit, minlength=params["n_range"]))[-12:]
    rng = np.random.default_rng(11)
    ns = np.unique(np.concatenate([dense, rng.integers(0, params["n_range"], 8)])).astype(np.int32)
    E_ref, _, s_ref = oracle.volume(params, ref, ns=ns)
    assert parity.nl2(sonar.echoes(params)[0][ns], s_ref) < S_TOL
    assert parity.nl2(E[:, ns], E_ref) <= 1e-4


def test_cross_batch_equals_oracle_per_ping(sonar):
    scene, params, poses, ssp = inputs.workload("wall_mirror")
    rng = np.random.default_rng(3)
    ps = [inputs.pose((0.2 * rng.uniform(-1, 1), 0.3 * rng.uniform(-1, 1), -2.0 + 0.2 * rng.uniform(-1, 1)),
                      yaw_deg=5 * rng.uniform(-1, 1), tilt_down_deg=15 + 3 * rng.uniform(-1, 1)) for _ in range(3)]
    sonar.upload(scene)
    env, _, _ = sonar.ping_batch(ps, params, ssp)
    torch.cuda.synchronize()
    env = env.reshape(len(ps), -1, params["n_range"]).double().cpu().numpy()
    for i, pose in enumerate(ps):
        E_ref, _, _ = oracle.volume(params, oracle.trace(scene, dict(params, cross=1), pose, ssp))
        assert parity.nl2(env[i], E_ref) <= 1e-4, i


def test_cross_off_is_monostatic(sonar):
    from paper_2606_06130_gb300.sonar import SONAR_OPT_CROSS
    scene, params, poses, ssp = inputs.workload("wall_mirror")
    sonar.set_option(SONAR_OPT_CROSS, 0)
    try:
        E = _ping(sonar, scene, params, poses[0], ssp)
        hits = sonar.hits()
    finally:
        sonar.set_option(SONAR_OPT_CROSS, 1)
    assert _cross_counts(hits["key"]) == (0, 0, 0)
    ref = oracle.trace(scene, params, poses[0], ssp)
    parity.check_hits(hits, ref, params["n_sub"])
    E_ref, _, _ = oracle.volume(params, ref)
    assert parity.nl2(E, E_ref) <= 1e-4


def test_cross_rejects_refraction_and_bad_values(sonar):
    from paper_2606_06130_gb300.sonar import SONAR_OPT_CROSS, SonarError, SONAR_E_UNSUPPORTED, SONAR_E_ARG
    scene, params, poses, ssp = inputs.workload("c3")
    sonar.upload(scene)
    with pytest.raises(SonarError) as e:
        sonar.ping(poses[0], params, ssp)
    assert e.value.code == SONAR_E_UNSUPPORTED
    with pytest.raises(SonarError) as e:
        sonar.set_option(SONAR_OPT_CROSS, 2)
    assert e.value.code == SONAR_E_ARG


def test_cross_without_reflections_is_monostatic(sonar):
    """max_bounces 0 leaves no reflected route, so cross terms add nothing but the point
    scatterers' pairs of image routes (none either: only the direct route remains)."""
    scene, params, poses, ssp = inputs.workload("wall_mirror")
    params = dict(params, max_bounces=0)
    E = _ping(sonar, scene, params, poses[0], ssp)
    hits = sonar.hits()
    assert _cross_counts(hits["key"]) == (0, 0, 0)
    ref = oracle.trace(scene, dict(params, cross=1), poses[0], ssp)
    parity.check_hits(hits, ref, params["n_sub"])
    E_ref, _, _ = oracle.volume(params, ref)
    assert parity.nl2(E, E_ref) <= 1e-4
