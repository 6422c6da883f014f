"""Failure detection without a GPU fault, through the C ABI: a device-side bounded wait
that nothing completes (an mbarrier no thread arrives at) gives up at its limit, the
call returns SONAR_E_TIMEOUT with its message, and the context keeps working: a ping
made after it matches the FP64 oracle."""
import time

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


def test_bounded_wait_times_out_and_the_context_survives(sonar):
    from paper_2606_06130_gb300.sonar import SONAR_E_ARG, SONAR_E_TIMEOUT, lib
    t0 = time.perf_counter()
    rc = sonar.probe_wait_limit(1 << 22)  # a few milliseconds of SM clock
    dt = time.perf_counter() - t0
    assert rc == SONAR_E_TIMEOUT, rc
    assert "wait" in lib().sonar_last_error(sonar.h).decode()
    assert dt < 5.0
    # the limit must lie in 1 .. 2^31
    assert sonar.probe_wait_limit(0) == SONAR_E_ARG
    assert sonar.probe_wait_limit((1 << 31) + 1) == SONAR_E_ARG
    # a second timeout in a row, then a ping on the same context
    assert sonar.probe_wait_limit(1 << 20) == SONAR_E_TIMEOUT
    scene, params, poses, ssp = inputs.workload("c1")
    sonar.upload(scene)
    env, _, n = sonar.ping(poses[0], params, ssp, precision="fp32")
    torch.cuda.synchronize()
    E = env.reshape(-1, params["n_range"]).double().cpu().numpy()
    ref = oracle.trace(scene, params, poses[0], ssp)
    E_ref, _, _ = oracle.volume(params, ref)
    assert parity.nl2(E, E_ref) <= 1e-4
    assert n > 0


def test_host_side_failures_leave_the_context_usable(sonar):
    """Failures made on the host: a ping before any scene, a pose with a zero quaternion
    or a non-finite position, and a context that is used again afterwards."""
    import numpy as np
    from paper_2606_06130_gb300.sonar import SONAR_E_ARG, SONAR_E_NOSCENE, Sonar, SonarError
    scene, params, poses, ssp = inputs.workload("c1")
    fresh = Sonar(0)
    try:
        with pytest.raises(SonarError) as e:
            fresh.ping(poses[0], params, ssp, precision="fp32")
        assert e.value.code == SONAR_E_NOSCENE
        fresh.upload(scene)
        bad_q = dict(poses[0], q=np.zeros(4))
        bad_t = dict(poses[0], t=np.array([np.nan, 0.0, 0.0]))
        for bad in (bad_q, bad_t):
            with pytest.raises(SonarError) as e:
                fresh.ping(bad, params, ssp, precision="fp32")
            assert e.value.code == SONAR_E_ARG
        env, _, n = fresh.ping(poses[0], params, ssp, precision="fp32")
        torch.cuda.synchronize()
        E = env.reshape(-1, params["n_range"]).double().cpu().numpy()
        E_ref, _, _ = oracle.volume(params, oracle.trace(scene, params, poses[0], ssp))
        assert parity.nl2(E, E_ref) <= 1e-4
    finally:
        fresh.close()
