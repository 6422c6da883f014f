"""GPU true-time-delay beamforming (wide apertures, Sec. II.A range- and depth-dependent
settings) against the FP64 oracle, through the C ABI.

With SONAR_OPT_TTD = U the library synthesises wideband element echoes (the plane-wave
delay of each hit across the aperture kept in the envelope) at U phases per range cell
and forms each beam by reading every element at its steering delay through 4-point
Lagrange interpolation on that grid. Checked: every wideband phase against the oracle's
wideband echoes (WB_TOL: the synthesis table is linear on a grid of about dt / 128), the
envelope against the oracle's fractional-delay beamformer (FP32 form E_TOL, BF16 form
1e-2), its convergence to the exact true-time-delay beams as U grows, a full-size
harbour ping on sampled beams and range samples, batches, and the option's checks.
"""
import numpy as np
import pytest

import oracle
from paper_2606_06130_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WB_TOL = 1e-4
E_TOL = 2e-4


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


def run(s, scene, params, pose, ssp, U, precision="fp32", phases=False):
    from paper_2606_06130_gb300.sonar import SONAR_OPT_TTD
    s.set_option(SONAR_OPT_TTD, U)
    try:
        s.upload(scene)
        env, _, _ = s.ping(pose, params, ssp, precision=precision)
        torch.cuda.synchronize()
        E = env.reshape(-1, params["n_range"]).double().cpu().numpy()
        wb = [s.raw(params, k)[0] for k in range(U)] if phases else []
    finally:
        s.set_option(SONAR_OPT_TTD, 0)
    return E, wb


def c1(**over):
    scene, params, poses, ssp = inputs.workload("c1")
    return scene, dict(params, **over), poses[0], ssp


def dt_of(params, c_ref):
    return 2.0 * (params["r_max"] - params["r_min"]) / params["n_range"] / c_ref


def subset(h: dict, keep) -> dict:
    """The hits of h selected by a boolean mask."""
    out = {k: (v[keep] if isinstance(v, np.ndarray) and v.shape[:1] == (h["n"],) else v) for k, v in h.items()}
    out["n"] = int(np.count_nonzero(keep))
    return out


@pytest.mark.parametrize("U,nx,ny", [(1, 8, 8), (4, 32, 32), (3, 12, 12)])
def test_wideband_phases_match_oracle(sonar, U, nx, ny):
    scene, params, pose, ssp = c1(nx=nx, ny=ny, n_beam_az=24, n_beam_el=12)
    _, wb = run(sonar, scene, params, pose, ssp, U, phases=True)
    h = oracle.trace(scene, params, pose, ssp)
    ns = np.arange(params["n_range"])
    dt = dt_of(params, h["c_ref"])
    for s in range(U):
        ref = oracle.synth_wideband(params, h, ns, shift=s * dt / U)
        assert parity.nl2(wb[s], ref) < WB_TOL, (s, parity.nl2(wb[s], ref))


def test_ttd_beams_match_oracle_fractional_delay_beamformer(sonar):
    """32 x 32 array on the C1 scene, U = 4, all beams and bins: the envelope against the
    oracle's fractional-delay beamformer, FP32 and BF16 forms. The true-time-delay beams
    differ from the phase-shift beams of the same scene by far more than the tolerance."""
    scene, params, pose, ssp = c1(nx=32, ny=32, n_beam_az=24, n_beam_el=12)
    U = 4
    h = oracle.trace(scene, params, pose, ssp)
    ns = np.arange(params["n_range"])
    E_ref = oracle.envelope(params, oracle.ttd_interpolated(params, h, ns, U), ns)
    E, _ = run(sonar, scene, params, pose, ssp, U)
    assert parity.nl2(E, E_ref) < E_TOL, parity.nl2(E, E_ref)
    E16, _ = run(sonar, scene, params, pose, ssp, U, precision="bf16")
    assert parity.nl2(E16, E_ref) < 1e-2
    E_ps, _ = run(sonar, scene, params, pose, ssp, 0)
    assert parity.nl2(E_ps, E_ref) > 20 * E_TOL, parity.nl2(E_ps, E_ref)


def test_ttd_converges_to_exact_beams(sonar):
    """16 x 16 array, 24 sampled beams, all bins: the GPU's beams against the exact
    true-time-delay beams (no interpolation) improve as the grid refines (fourth order:
    at least four times smaller from U = 2 to U = 4) and sit below 1e-3 at U = 4."""
    scene, params, pose, ssp = c1(nx=16, ny=16, n_beam_az=24, n_beam_el=12)
    h = oracle.trace(scene, params, pose, ssp)
    ns = np.arange(params["n_range"])
    rng = np.random.default_rng(11)
    beams = np.sort(rng.choice(params["n_beam_az"] * params["n_beam_el"], 24, replace=False))
    E_exact = oracle.envelope(params, oracle.ttd_exact(params, h, ns, beams), ns)
    err = {}
    for U in (2, 4):
        E, _ = run(sonar, scene, params, pose, ssp, U)
        err[U] = parity.nl2(E[beams], E_exact)
    assert err[4] < 1e-3 and err[4] < err[2] / 4, err


def test_c2_ttd_sampled_parity(sonar):
    """Full-size harbour ping (32 x 32 array, 8192 beams, 1024 bins, 11 delay levels) at
    U = 4, in the launch configuration the bench times: the envelope on 64 sampled beams
    at two range samples against the oracle's fractional-delay beamformer over the hits
    that reach them. The rows are drawn among rows of moderate echo density (between the
    25th and 50th percentile of the rows with hits): the oracle evaluates the pulse
    autocorrelation for every (element, hit, sample, level), about 10^9 times here."""
    scene, params, poses, ssp = inputs.workload("c2")
    U = 4
    E, _ = run(sonar, scene, params, poses[0], ssp, U)
    h = oracle.trace(scene, params, poses[0], ssp)
    dr = (params["r_max"] - params["r_min"]) / params["n_range"]
    n_hit = np.floor((h["tau"] * h["c_ref"] / 2 - params["r_min"]) / dr).astype(int)
    counts = np.bincount(np.clip(n_hit, 0, params["n_range"] - 1), minlength=params["n_range"])
    lo, hi = np.percentile(counts[counts > 0], [25, 50])
    cand = np.nonzero((counts >= lo) & (counts <= hi))[0]
    ns = np.sort(np.random.default_rng(14).choice(cand, 2, replace=False)).astype(np.int32)
    # hits whose pulse can reach a sampled row at any element, phase and level
    dt = dt_of(params, h["c_ref"])
    t = 2 * (params["r_min"] + (ns + 0.5) * dr) / h["c_ref"]
    reach = params["pulse"] + 4 * dt
    keep = np.any(np.abs(t[None, :] - h["tau"][:, None]) < reach, axis=1)
    rng = np.random.default_rng(12)
    beams = np.sort(rng.choice(params["n_beam_az"] * params["n_beam_el"], 64, replace=False))
    B = oracle.ttd_interpolated(params, subset(h, keep), ns, U, beams)
    E_ref = oracle.envelope(params, B, ns)
    assert parity.nl2(E[beams][:, ns], E_ref) < E_TOL, parity.nl2(E[beams][:, ns], E_ref)


def test_ttd_batch_equals_single_pings(sonar):
    from paper_2606_06130_gb300.sonar import SONAR_OPT_TTD
    scene, params, pose0, ssp = c1(nx=16, ny=16, n_beam_az=24, n_beam_el=12)
    poses = [inputs.pose(pose0["t"] + np.array([0.1 * k, 0.0, 0.0]), yaw_deg=-5.0 + 6.0 * k,
                         tilt_down_deg=15.0, roll_deg=0.0) for k in range(3)]
    sonar.set_option(SONAR_OPT_TTD, 2)
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
        sonar.set_option(SONAR_OPT_TTD, 0)


def test_ttd_option_arguments(sonar):
    from paper_2606_06130_gb300.sonar import (SONAR_OPT_RAW, SONAR_OPT_TTD, SonarError, SONAR_E_ARG,
                                              SONAR_E_UNSUPPORTED)
    with pytest.raises(SonarError) as e:
        sonar.set_option(SONAR_OPT_TTD, 9)
    assert e.value.code == SONAR_E_ARG
    scene, params, pose, ssp = c1()
    sonar.upload(scene)
    sonar.set_option(SONAR_OPT_TTD, 2)
    try:
        with pytest.raises(SonarError) as e:
            sonar.ping(pose, params, ssp, precision="fp16")
        assert e.value.code == SONAR_E_UNSUPPORTED
        sonar.set_option(SONAR_OPT_RAW, 2)
        with pytest.raises(SonarError) as e:
            sonar.ping(pose, params, ssp)
        assert e.value.code == SONAR_E_UNSUPPORTED
        sonar.set_option(SONAR_OPT_RAW, 0)
        sonar.ping(pose, params, ssp)
        torch.cuda.synchronize()
        with pytest.raises(SonarError):
            sonar.raw(params, 2)  # phases 0 and 1 only
    finally:
        sonar.set_option(SONAR_OPT_TTD, 0)
        sonar.set_option(SONAR_OPT_RAW, 0)
