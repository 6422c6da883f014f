"""The allocation-free cloud entry point (sonar_cloud_noalloc) against sonar_ping.

sonar_cloud_noalloc serves callers that cannot call cudaMalloc; it keeps its scratch in
a fixed file-scope device array. Here it runs through the C ABI on envelopes written by
sonar_ping / sonar_ping_batch, twice in a row (the array keeps the previous call's
contents), and must give the same cloud as those calls: beams, bins and intensities
exactly, positions to 1e-5 m. This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2606_06130_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sonar_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06130_gb300 import sonar
    return sonar


def _call(sonar, env_ptr, params, poses, cloud_ptr, cap):
    P = len(poses)
    n = (C.c_int64 * P)()
    arr = (sonar.sonar_pose * P)(*[sonar.make_pose(p) for p in poses])
    sp = sonar.make_params(params)
    rc = sonar.lib().sonar_cloud_noalloc(env_ptr, P, C.byref(sp), arr, cloud_ptr, cap, n,
                                         C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, list(n)


def _noalloc(sonar, env, params, poses, cap):
    cloud = torch.zeros((len(poses), cap, 6), dtype=torch.int32, device="cuda:0")
    rc, n = _call(sonar, env.data_ptr(), params, poses, cloud.data_ptr(), cap)
    assert rc == sonar.SONAR_OK, rc
    return cloud, n


def _same_cloud(sonar, a, na, b, nb):
    assert na == nb
    pa = sonar.cloud_records(a, na)
    pb = sonar.cloud_records(b, nb)
    assert np.array_equal(pa["beam"], pb["beam"]) and np.array_equal(pa["bin"], pb["bin"])
    assert np.array_equal(pa["intensity"], pb["intensity"])
    for k in ("x", "y", "z"):
        assert np.max(np.abs(pa[k] - pb[k]), initial=0.0) <= 1e-5


def test_noalloc_cloud_matches_ping_twice(sonar_mod):
    sonar = sonar_mod
    scene, params, poses, ssp = inputs.workload("c1")
    s = sonar.Sonar(0)
    s.upload(scene)
    nb = params["n_beam_az"] * params["n_beam_el"]
    env, cloud, n = s.ping(poses[0], params, ssp)
    torch.cuda.synchronize()
    assert n > 0
    for _ in range(2):
        c2, n2 = _noalloc(sonar, env, params, poses[:1], nb)
        _same_cloud(sonar, cloud, n, c2[0], n2[0])

    # a two-ping batch with a different threshold mode
    p2 = dict(params, thr_mode=0, thr=0.05)
    poses2 = [poses[0], inputs.pose((0.3, -0.2, -2.1), yaw_deg=12.0, tilt_down_deg=18.0)]
    envb, cloudb, nbat = s.ping_batch(poses2, p2, ssp)
    torch.cuda.synchronize()
    for _ in range(2):
        c3, n3 = _noalloc(sonar, envb, p2, poses2, nb)
        for i in range(2):
            _same_cloud(sonar, cloudb[i], int(nbat[i]), c3[i], n3[i])
    s.close()


def test_noalloc_rejects_sizes_beyond_its_maximum(sonar_mod):
    sonar = sonar_mod
    params = inputs.sensor_params("c2")
    env = torch.zeros(1, dtype=torch.float32, device="cuda:0")
    poses = [inputs.pose((0.0, 0.0, -8.0))] * 65
    arr = (sonar.sonar_pose * 65)(*[sonar.make_pose(p) for p in poses])
    sp = sonar.make_params(params)
    n = (C.c_int64 * 65)()
    rc = sonar.lib().sonar_cloud_noalloc(env.data_ptr(), 65, C.byref(sp), arr, None, 0, n, None)
    assert rc == sonar.SONAR_E_CAPACITY


def test_noalloc_warm_call_allocates_nothing_and_truncates(sonar_mod):
    """A warm call leaves the device's free memory unchanged; a cloud buffer smaller
    than a ping's points gives SONAR_E_CAPACITY, the full count, and the first cap
    points of sonar_ping's cloud; a count-only call (no cloud) succeeds."""
    sonar = sonar_mod
    scene, params, poses, ssp = inputs.workload("c1")
    s = sonar.Sonar(0)
    s.upload(scene)
    nb = params["n_beam_az"] * params["n_beam_el"]
    env, cloud, n = s.ping(poses[0], params, ssp)
    torch.cuda.synchronize()
    assert n > 8
    out = torch.zeros((1, nb, 6), dtype=torch.int32, device="cuda:0")
    rc, _ = _call(sonar, env.data_ptr(), params, poses[:1], out.data_ptr(), nb)  # warm
    assert rc == sonar.SONAR_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    rc, n1 = _call(sonar, env.data_ptr(), params, poses[:1], out.data_ptr(), nb)
    torch.cuda.synchronize()
    assert rc == sonar.SONAR_OK and n1[0] == n
    assert torch.cuda.mem_get_info(0)[0] == free0

    cap = n // 2
    small = torch.zeros((1, cap, 6), dtype=torch.int32, device="cuda:0")
    rc, n2 = _call(sonar, env.data_ptr(), params, poses[:1], small.data_ptr(), cap)
    assert rc == sonar.SONAR_E_CAPACITY and n2[0] == n
    _same_cloud(sonar, cloud[:cap], cap, small[0], cap)

    rc, n3 = _call(sonar, env.data_ptr(), params, poses[:1], None, 0)
    assert rc == sonar.SONAR_OK and n3[0] == n
    s.close()


def test_noalloc_rejects_host_buffers(sonar_mod):
    """Host buffers are refused with SONAR_E_ARG before any kernel runs."""
    sonar = sonar_mod
    params = inputs.sensor_params("c1")
    nb = params["n_beam_az"] * params["n_beam_el"]
    poses = [inputs.pose((0.0, 0.0, -2.0))]
    env_host = np.zeros((nb, params["n_range"]), np.float32)
    env_dev = torch.zeros((nb, params["n_range"]), dtype=torch.float32, device="cuda:0")
    cloud_host = np.zeros((nb, 6), np.int32)
    cloud_dev = torch.zeros((nb, 6), dtype=torch.int32, device="cuda:0")
    rc, _ = _call(sonar, env_host.ctypes.data, params, poses, cloud_dev.data_ptr(), nb)
    assert rc == sonar.SONAR_E_ARG
    rc, _ = _call(sonar, env_dev.data_ptr(), params, poses, cloud_host.ctypes.data, nb)
    assert rc == sonar.SONAR_E_ARG
    rc, _ = _call(sonar, env_dev.data_ptr(), params, poses, cloud_dev.data_ptr(), nb)
    assert rc == sonar.SONAR_OK
