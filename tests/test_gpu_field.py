"""GPU parity of rays in a range-dependent sound-speed field (sonar_set_field) against
the FP64 oracle: prim ids bit-exact outside the near-tie margins, delays to 1e-12,
amplitudes and phases to 2e-6, envelopes within 1e-4 normalised L2 (FP32 form)."""
import math

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
    from paper_2606_06130_gb300.sonar import Sonar, SONAR_OPT_DEBUG
    s = Sonar(0)
    s.set_option(SONAR_OPT_DEBUG, 1)
    yield s
    s.set_field(None)
    s.close()


def _field(fun, x0, x1, z0, z1, nx, nz, h):
    xs, zs = np.linspace(x0, x1, nx), np.linspace(z0, z1, nz)
    return {"x0": x0, "dx": xs[1] - xs[0], "z0": z0, "dz": zs[1] - zs[0],
            "c": np.array([[fun(x, z) for x in xs] for z in zs]), "h": h}


ISO = {"z": np.array([0.0]), "c": np.array([1500.0])}


def _run(s, scene, params, pose, field):
    s.upload(scene)
    s.set_field(field)
    try:
        env, _, _ = s.ping(pose, params, ISO)
        torch.cuda.synchronize()
        hits = s.hits()
        echoes = s.echoes(params)[0]
    finally:
        s.set_field(None)
    return env.reshape(-1, params["n_range"]).double().cpu().numpy(), hits, echoes


def _wall():
    sc, p, ps, _ = inputs.workload("wall_mirror")
    return inputs.Scene(sc.verts, sc.tris, sc.mu, sc.flags), dict(p, max_bounces=1), ps[0]


@pytest.mark.parametrize("kind", ["depth", "range_and_depth"])
def test_wall_mirror_field_parity(sonar, kind):
    scene, params, pose = _wall()
    zs = pose["t"][2]
    if kind == "depth":
        fun = lambda x, z: 1500.0 + 20.0 * (z - zs)
    else:
        fun = lambda x, z: 1500.0 + 12.0 * math.sin(x / 2.5) + 8.0 * (z - zs) + 0.6 * x * (z - zs)
    fld = _field(fun, -6.0, 16.0, -7.0, 3.0, 23, 21, 0.05)
    E, hits, s_gpu = _run(sonar, scene, params, pose, fld)
    ref = oracle.trace(scene, dict(params, field=fld), pose, ISO)
    excluded, matched = parity.check_hits(hits, ref, params["n_sub"])
    assert matched >= ref["n"] - 2 * (excluded + 1) and ref["n"] > 1000
    E_ref, _, s_ref = oracle.volume(params, ref)
    assert parity.nl2(s_gpu, s_ref) < 5e-5
    assert parity.nl2(E, E_ref) <= 1e-4


def test_c2_thermocline_field_parity(sonar):
    """The harbour wall through a thermocline that deepens with range (reduced ray grid:
    the oracle integrates every ray in FP64)."""
    scene, params, poses, _ = inputs.workload("c2")
    params = dict(params, n_ray_az=128, n_ray_el=64, n_sub=1, c_ref=1500.0)
    fun = lambda x, z: 1500.0 - 6.0 * math.tanh((z + 6.0 + 0.15 * x) / 1.5)
    fld = _field(fun, -4.0, 16.0, -12.0, 1.0, 21, 27, 0.25)
    E, hits, _ = _run(sonar, scene, params, poses[0], fld)
    ref = oracle.trace(scene, dict(params, field=fld), poses[0], ISO)
    excluded, matched = parity.check_hits(hits, ref, params["n_sub"])
    assert matched >= ref["n"] - 2 * (excluded + 1) and ref["n"] > 5000
    rng = np.random.default_rng(23)
    ns = np.unique(rng.integers(0, params["n_range"], 16)).astype(np.int32)
    E_ref, _, _ = oracle.volume(params, ref, ns=ns)
    assert parity.nl2(E[:, ns], E_ref) <= 1e-4


def test_field_arguments_and_combinations(sonar):
    from paper_2606_06130_gb300.sonar import SonarError, SONAR_E_ARG, SONAR_E_UNSUPPORTED, SONAR_OPT_CROSS
    scene, params, pose = _wall()
    good = _field(lambda x, z: 1500.0, -6.0, 16.0, -7.0, 3.0, 3, 3, 0.1)
    for bad in (dict(good, h=0.0), dict(good, dx=-1.0), dict(good, c=-good["c"]), dict(good, c=good["c"][:1])):
        with pytest.raises(SonarError) as e:
            sonar.set_field(bad)
        assert e.value.code == SONAR_E_ARG
    sonar.upload(scene)
    sonar.set_field(good)
    sonar.set_option(SONAR_OPT_CROSS, 1)
    try:
        with pytest.raises(SonarError) as e:
            sonar.ping(pose, params, ISO)
        assert e.value.code == SONAR_E_UNSUPPORTED
    finally:
        sonar.set_option(SONAR_OPT_CROSS, 0)
        sonar.set_field(None)
    # a uniform field gives the straight-ray volume
    E_f, _, _ = _run(sonar, scene, dict(params, c_ref=1500.0), pose, good)
    sonar.upload(scene)
    env, _, _ = sonar.ping(pose, dict(params, c_ref=1500.0), ISO)
    torch.cuda.synchronize()
    assert parity.nl2(E_f, env.reshape(-1, params["n_range"]).double().cpu().numpy()) < 1e-5


def test_smallest_field_grid(sonar):
    """A 2 x 2 grid (one bilinear cell covering nothing: every position is clamped onto
    it) with a depth gradient: against the oracle."""
    scene, params, pose = _wall()
    zs = pose["t"][2]
    fld = {"x0": 0.0, "dx": 1.0, "z0": zs - 0.5, "dz": 1.0,
           "c": np.array([[1495.0, 1496.0], [1505.0, 1504.0]]), "h": 0.1}
    E, hits, _ = _run(sonar, scene, params, pose, fld)
    ref = oracle.trace(scene, dict(params, field=fld), pose, ISO)
    excluded, matched = parity.check_hits(hits, ref, params["n_sub"])
    assert matched >= ref["n"] - 2 * (excluded + 1) and ref["n"] > 1000
    E_ref, _, _ = oracle.volume(params, ref)
    assert parity.nl2(E, E_ref) <= 1e-4
