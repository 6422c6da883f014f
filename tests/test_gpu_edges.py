"""GPU edge cases against the FP64 oracle, through the C ABI.

Empty and point-only scenes; sizes that are multiples of no tile (bins, beams, rays);
array shapes that select each synthesis kernel (z-split tensor-core kernel at L2 = 2
and 4, per-tile tensor-core kernel, FP32 SIMT kernel); the 16-tap limit and the
rejection of 17 taps; a batch of pings against the same pings one at a time; a single
ray without bounces. Tolerances as in test_gpu_parity: envelope normalised L2 <= 1e-4
for the FP32 form, hit primitive ids exact outside the near-tie margins.
"""
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
    s.close()


def ping(s, scene, params, pose, ssp, precision="fp32"):
    s.upload(scene)
    env, cloud, n = s.ping(pose, params, ssp, precision=precision)
    torch.cuda.synchronize()
    return env.reshape(-1, params["n_range"]).double().cpu().numpy(), cloud, n


def full_parity(s, scene, params, pose, ssp, env_tol=1e-4):
    """Hits, envelope and peaks against the oracle; returns the oracle hit count."""
    from paper_2606_06130_gb300.sonar import cloud_records
    E, cloud, n = ping(s, scene, params, pose, ssp)
    ref = oracle.trace(scene, params, pose, ssp)
    parity.check_hits(s.hits(), ref, params["n_sub"])
    E_ref, _, _ = oracle.volume(params, ref)
    err = parity.nl2(E, E_ref) if np.linalg.norm(E_ref) > 0 else float(np.abs(E).max())
    assert err <= env_tol, err
    pk = oracle.peaks(params, pose, E_ref)
    pts = cloud_records(cloud, n)
    nb = parity.n_blank(params)
    vmax = E_ref[:, nb:].max()
    thr = params["thr"] * vmax if params["thr_mode"] == 1 else params["thr"]
    ok = parity.peak_margin_mask(E_ref, nb, thr, 1e-3)
    gpu = {int(b): int(k) for b, k in zip(pts["beam"], pts["bin"])}
    want = {int(b): int(k) for b, k in zip(pk["beam"], pk["bin"])}
    for b in np.nonzero(ok)[0]:
        assert gpu.get(int(b)) == want.get(int(b)), (b, gpu.get(int(b)), want.get(int(b)))
    return ref["n"]


def c1(**over):
    scene, params, poses, ssp = inputs.workload("c1")
    return scene, dict(params, **over), poses[0], ssp


def test_empty_scene_gives_zero_volume_and_blank_peaks(sonar):
    _, params, pose, ssp = c1()
    empty = inputs.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.float32),
                         np.zeros(0, np.uint8))
    E, cloud, n = ping(sonar, empty, params, pose, ssp)
    assert sonar.stats()["n_hits"] == 0
    assert not E.any()
    ref = oracle.trace(empty, params, pose, ssp)
    assert ref["n"] == 0
    # a zero volume meets the relative threshold everywhere: every beam peaks at the
    # first unblanked bin with intensity 0, on both sides
    from paper_2606_06130_gb300.sonar import cloud_records
    pk = oracle.peaks(params, pose, np.zeros_like(E))
    pts = cloud_records(cloud, n)
    assert list(pts["beam"]) == list(pk["beam"])
    assert list(pts["bin"]) == list(pk["bin"]) and set(pts["bin"]) == {parity.n_blank(params)}


def test_points_only_scene(sonar):
    scene, params, pose, ssp = c1()
    pts_only = inputs.Scene(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), np.zeros(0, np.float32),
                            np.zeros(0, np.uint8), scene.points, scene.sigma, scene.planes)
    n = full_parity(sonar, pts_only, params, pose, ssp)
    assert n > 0


def test_ragged_bins_beams_and_rays(sonar):
    scene, params, pose, ssp = c1(n_range=200, n_beam_az=30, n_beam_el=10, n_ray_az=50, n_ray_el=20)
    assert full_parity(sonar, scene, params, pose, ssp) > 0


@pytest.mark.parametrize("nx,ny", [(16, 16), (64, 8), (12, 12)])
def test_array_shapes_select_each_synthesis_kernel(sonar, nx, ny):
    """(16, 16) and (64, 8): z-split tensor-core kernel with L2 = 2 and 4; (12, 12):
    no tensor-core layout applies, the FP32 SIMT kernel runs."""
    scene, params, pose, ssp = c1(nx=nx, ny=ny, n_beam_az=24, n_beam_el=12)
    assert full_parity(sonar, scene, params, pose, ssp) > 0


@pytest.mark.parametrize("nx", [8, 32])
def test_sixteen_taps(sonar, nx):
    """The longest supported pulse: floor(2 T_p / dt) + 1 = 16 taps, in the per-tile
    (8x8) and z-split (32x32, four rows per tile) kernels."""
    scene, params, pose, ssp = c1(nx=nx, ny=nx, pulse=2.0e-4)
    dt = 2 * (params["r_max"] - params["r_min"]) / params["n_range"] / inputs.C_WATER
    assert math.floor(2 * params["pulse"] / dt) + 1 == 16
    assert full_parity(sonar, scene, params, pose, ssp) > 0


def test_seventeen_taps_are_rejected(sonar):
    from paper_2606_06130_gb300.sonar import SonarError
    scene, params, pose, ssp = c1(pulse=2.2e-4)
    sonar.upload(scene)
    with pytest.raises(SonarError) as e:
        sonar.ping(pose, params, ssp)
    assert e.value.code == -7  # SONAR_E_UNSUPPORTED


def test_batch_equals_single_pings_and_oracle(sonar):
    scene, params, pose0, ssp = c1()
    poses = [inputs.pose(pose0["t"] + np.array([0.1 * k, -0.05 * k, 0.0]), yaw_deg=-10.0 + 8.0 * k,
                         tilt_down_deg=15.0 - k, roll_deg=2.0 * k) for k in range(4)]
    sonar.upload(scene)
    env_b, cloud_b, n_b = sonar.ping_batch(poses, params, ssp)
    torch.cuda.synchronize()
    env_b = env_b.reshape(len(poses), -1, params["n_range"]).double().cpu().numpy()
    for k, ps in enumerate(poses):
        E1, _, n1 = ping(sonar, scene, params, ps, ssp)
        assert parity.nl2(env_b[k], E1) <= 1e-6
        assert int(n_b[k]) == n1
        ref = oracle.trace(scene, params, ps, ssp)
        E_ref, _, _ = oracle.volume(params, ref)
        assert parity.nl2(env_b[k], E_ref) <= 1e-4


def test_single_ray_without_bounces(sonar):
    scene, params, pose, ssp = c1(n_ray_az=1, n_ray_el=1, max_bounces=0, hfov=math.radians(10.0),
                                  vfov=math.radians(10.0))
    full_parity(sonar, scene, params, pose, ssp)


def test_outputs_in_device_pinned_and_pageable_memory_agree(sonar):
    """Device outputs are written in place, pinned host outputs through the device's
    mapping of them, pageable ones through staging: all three give the same ping."""
    from paper_2606_06130_gb300.sonar import cloud_records
    scene, params, pose, ssp = c1()
    sonar.upload(scene)
    nb = params["n_beam_az"] * params["n_beam_el"]
    shape = (1, params["n_beam_el"], params["n_beam_az"], params["n_range"])
    env_d, cloud_d, n_d = sonar.ping_batch([pose], params, ssp)
    env_p = torch.zeros(shape, dtype=torch.float32, pin_memory=True)
    cloud_p = torch.zeros((1, nb, 6), dtype=torch.int32, pin_memory=True)
    _, _, n_p = sonar.ping_batch([pose], params, ssp, env=env_p, cloud=cloud_p, cloud_cap=nb)
    env_h = np.zeros(shape, np.float32)
    cloud_h = np.zeros((1, nb, 6), np.int32)
    _, _, n_h = sonar.ping_batch([pose], params, ssp, env=env_h, cloud=cloud_h, cloud_cap=nb)
    torch.cuda.synchronize()
    E_d = env_d.cpu().numpy()
    assert parity.nl2(env_p.numpy(), E_d) <= 1e-6 and parity.nl2(env_h, E_d) <= 1e-6
    assert int(n_d[0]) == int(n_p[0]) == int(n_h[0])
    c_d = cloud_records(cloud_d[0], int(n_d[0]))
    for c in (cloud_records(cloud_p[0], int(n_p[0])), cloud_records(cloud_h[0], int(n_h[0]))):
        assert list(c["beam"]) == list(c_d["beam"]) and list(c["bin"]) == list(c_d["bin"])
