"""Asynchronous pings (sonar_ping_async / sonar_wait): the same results as the
synchronous calls, with at most two calls in flight and outputs in pinned host or device
memory. Hits are emitted through atomics, so their order, the tensor-core synthesis'
K-block grouping and with it the rounding of the BF16 hi/lo operands change from run to
run: every run lies about 1e-5 (normalised L2) from the oracle, and two runs agree to
within 5e-5, the bound used here; the C1 stream is held to the FP32 bar (1e-4) against
the oracle itself."""
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


def _poses(base, k, seed):
    rng = np.random.default_rng(seed)
    t = base["t"]
    return [inputs.pose((t[0] + 0.2 * rng.uniform(-1, 1), t[1] + 0.2 * rng.uniform(-1, 1), t[2] + 0.1 * rng.uniform(-1, 1)),
                        yaw_deg=4 * rng.uniform(-1, 1), tilt_down_deg=12 + 3 * rng.uniform(-1, 1)) for _ in range(k)]


def test_async_stream_matches_oracle_c1(sonar):
    scene, params, poses, ssp = inputs.workload("c1")
    sonar.upload(scene)
    ps = _poses(poses[0], 5, 1)
    shape = (1, params["n_beam_el"], params["n_beam_az"], params["n_range"])
    nb = params["n_beam_az"] * params["n_beam_el"]
    envs = [torch.empty(shape, dtype=torch.float32, pin_memory=True) for _ in ps]
    clouds = [torch.empty((1, nb, 6), dtype=torch.int32, pin_memory=True) for _ in ps]
    counts = []
    for i, p in enumerate(ps):
        _, _, n = sonar.ping_async([p], params, ssp, env=envs[i], cloud=clouds[i], cloud_cap=nb)
        counts.append(n)
    sonar.wait()
    for i, p in enumerate(ps):
        E_ref, _, _ = oracle.volume(params, oracle.trace(scene, params, p, ssp))
        E = envs[i].reshape(-1, params["n_range"]).double().numpy()
        assert parity.nl2(E, E_ref) <= 1e-4, i
        assert counts[i][0] > 0


def test_async_equals_sync_c2_pinned_and_device(sonar):
    scene, params, poses, ssp = inputs.workload("c2")
    sonar.upload(scene)
    ps = _poses(poses[0], 6, 2)
    nb = params["n_beam_az"] * params["n_beam_el"]
    shape = (1, params["n_beam_el"], params["n_beam_az"], params["n_range"])
    ref = []
    for p in ps:
        env, cloud, n = sonar.ping(p, params, ssp)
        torch.cuda.synchronize()
        ref.append((env.double().cpu().numpy(), n))
    # alternate pinned-host and device outputs
    outs = []
    for i, p in enumerate(ps):
        if i % 2 == 0:
            env = torch.empty(shape, dtype=torch.float32, pin_memory=True)
            cloud = torch.empty((1, nb, 6), dtype=torch.int32, pin_memory=True)
        else:
            env = torch.empty(shape, dtype=torch.float32, device="cuda")
            cloud = torch.empty((1, nb, 6), dtype=torch.int32, device="cuda")
        _, _, n = sonar.ping_async([p], params, ssp, env=env, cloud=cloud, cloud_cap=nb)
        outs.append((env, n))
    sonar.wait()
    torch.cuda.synchronize()
    for i, ((env, n), (E_ref, n_ref)) in enumerate(zip(outs, ref)):
        E = env[0].double().cpu().numpy()
        assert parity.nl2(E, E_ref) < 5e-5, i
        assert abs(int(n[0]) - n_ref) <= 2, (i, int(n[0]), n_ref)


def test_async_then_sync_and_debug_reads(sonar):
    from paper_2606_06130_gb300.sonar import SONAR_OPT_DEBUG
    scene, params, poses, ssp = inputs.workload("c1")
    sonar.upload(scene)
    sonar.set_option(SONAR_OPT_DEBUG, 1)
    try:
        p = _poses(poses[0], 2, 3)
        sonar.ping_async([p[0]], params, ssp)
        sonar.ping_async([p[1]], params, ssp)
        hits = sonar.hits()  # retires both, then reads the last call's hits
        ref = oracle.trace(scene, params, p[1], ssp)
        parity.check_hits(hits, ref, params["n_sub"])
        env, _, _ = sonar.ping(p[0], params, ssp)  # a synchronous call after the stream
        torch.cuda.synchronize()
        E_ref, _, _ = oracle.volume(params, oracle.trace(scene, params, p[0], ssp))
        assert parity.nl2(env.reshape(-1, params["n_range"]).double().cpu().numpy(), E_ref) <= 1e-4
    finally:
        sonar.set_option(SONAR_OPT_DEBUG, 0)


def test_async_rejects_pageable_outputs(sonar):
    from paper_2606_06130_gb300.sonar import SonarError, SONAR_E_ARG
    scene, params, poses, ssp = inputs.workload("c1")
    sonar.upload(scene)
    env = torch.empty((1, params["n_beam_el"], params["n_beam_az"], params["n_range"]), dtype=torch.float32)
    with pytest.raises(SonarError) as e:
        sonar.ping_async([poses[0]], params, ssp, env=env)
    assert e.value.code == SONAR_E_ARG
    sonar.wait()


def test_async_batches(sonar):
    """Asynchronous calls of three pings each, alternating between two pinned buffers:
    every ping within the FP32 bar of the oracle."""
    scene, params, poses, ssp = inputs.workload("c1")
    sonar.upload(scene)
    ps = _poses(poses[0], 9, 4)
    nb = params["n_beam_az"] * params["n_beam_el"]
    shape = (3, params["n_beam_el"], params["n_beam_az"], params["n_range"])
    bufs = [torch.empty(shape, dtype=torch.float32, pin_memory=True) for _ in range(3)]
    counts = []
    for c in range(3):
        _, _, n = sonar.ping_async(ps[3 * c:3 * c + 3], params, ssp, env=bufs[c], cloud_cap=nb)
        counts.append(n)
    sonar.wait()
    for c in range(3):
        assert np.all(counts[c] > 0)
        for i in range(3):
            E_ref, _, _ = oracle.volume(params, oracle.trace(scene, params, ps[3 * c + i], ssp))
            E = bufs[c][i].reshape(-1, params["n_range"]).double().numpy()
            assert parity.nl2(E, E_ref) <= 1e-4, (c, i)
