"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances: hit prim ids bit-exact outside the near-tie margins (barycentric 1e-5,
runner-up gap 1e-6 m); delays to 1e-12 relative; envelope normalised L2 <= 1e-4 for the
FP32 form and <= 1e-2 for BF16/FP16; peak (beam, bin) bit-exact where the oracle's peak
beats its runner-up and the threshold by 1e-3 (FP32) or 2e-2 (BF16/FP16).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_06130_gb300 import inputs
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# Element echoes (FP32 form): the tensor-core synthesis forms BF16 hi/lo operands
# (representation error ~2^-17 per operand, ~2^-16 per product), so S agrees with the
# FP64 oracle to a few 1e-5; 5e-5 keeps the envelope inside its 1e-4 bound.
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


def run(s, scene, params, pose, ssp, precision="fp32"):
    s.upload(scene)
    env, cloud, n = s.ping(pose, params, ssp, precision=precision)
    torch.cuda.synchronize()
    return env.reshape(-1, params["n_range"]).double().cpu().numpy(), cloud, n


def cloud_check(cloud, n, params, pose, E_ref, rel):
    from paper_2606_06130_gb300.sonar import cloud_records
    pk = oracle.peaks(params, pose, E_ref)
    pts = cloud_records(cloud, n)
    nb = parity.n_blank(params)
    vmax = E_ref[:, nb:].max()
    thr = params["thr"] * vmax if params["thr_mode"] == 1 else params["thr"]
    ok = parity.peak_margin_mask(E_ref, nb, thr, rel)
    gpu = {int(b): int(k) for b, k in zip(pts["beam"], pts["bin"])}
    ref = {int(b): int(k) for b, k in zip(pk["beam"], pk["bin"])}
    checked = 0
    for b in np.nonzero(ok)[0]:
        assert gpu.get(int(b)) == ref.get(int(b)), (b, gpu.get(int(b)), ref.get(int(b)))
        checked += 1
    assert list(pts["beam"]) == sorted(pts["beam"])
    return checked, int(np.count_nonzero(~ok))


# ------------------------------------------------------------------ C1: tiny plain ping
def test_c1_fp32_full_parity(sonar):
    scene, params, poses, ssp = inputs.workload("c1")
    E, cloud, n = run(sonar, scene, params, poses[0], ssp)
    ref = oracle.trace(scene, params, poses[0], ssp)
    excluded, matched = parity.check_hits(sonar.hits(), ref, params["n_sub"])
    assert matched == ref["n"]
    E_ref, _, s_ref = oracle.volume(params, ref)
    s_gpu = sonar.echoes(params)[0]
    assert parity.nl2(s_gpu, s_ref) < S_TOL
    assert parity.nl2(E, E_ref) <= 1e-4
    checked, _ = cloud_check(cloud, n, params, poses[0], E_ref, 1e-3)
    assert checked > 0.8 * params["n_beam_az"] * params["n_beam_el"]


@pytest.mark.parametrize("precision,tol", [("bf16", 1e-2), ("fp16", 1e-2)])
def test_c1_reduced_precision(sonar, precision, tol):
    scene, params, poses, ssp = inputs.workload("c1")
    E, cloud, n = run(sonar, scene, params, poses[0], ssp, precision)
    ref = oracle.trace(scene, params, poses[0], ssp)
    E_ref, _, _ = oracle.volume(params, ref)
    assert parity.nl2(E, E_ref) <= tol
    cloud_check(cloud, n, params, poses[0], E_ref, 2e-2)


# ------------------------------------------------------------------ C3: curved rays, 2 bounces
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("bf16", 1e-2), ("fp16", 1e-2)])
def test_c3_refraction_precision_forms(sonar, precision, tol):
    scene, params, poses, ssp = inputs.workload("c3")
    E, cloud, n = run(sonar, scene, params, poses[0], ssp, precision)
    ref = oracle.trace(scene, params, poses[0], ssp)
    assert ref["c_ref"] != 1500.0
    parity.check_hits(sonar.hits(), ref, params["n_sub"])
    E_ref, _, _ = oracle.volume(params, ref)
    err = parity.nl2(E, E_ref)
    assert err <= tol, err
    cloud_check(cloud, n, params, poses[0], E_ref, 1e-3 if precision == "fp32" else 2e-2)


# ------------------------------------------------------------------ C2: harbour wall, full size
def test_c2_fp32_sampled_parity(sonar):
    scene, params, poses, ssp = inputs.workload("c2")
    E, cloud, n = run(sonar, scene, params, poses[0], ssp)
    ref = oracle.trace(scene, params, poses[0], ssp)
    excluded, matched = parity.check_hits(sonar.hits(), ref, params["n_sub"])
    assert matched >= ref["n"] - 2 * (excluded + 1)
    # sampled range samples: the densest echo region plus random ones
    dr = params["r_max"] / params["n_range"]
    n_hit = np.floor(ref["tau"] * ref["c_ref"] / 2 / dr).astype(int)
    dense = np.argsort(np.bincount(n_hit, minlength=params["n_range"]))[-12:]
    rng = np.random.default_rng(5)
    ns = np.unique(np.concatenate([dense, rng.integers(0, params["n_range"], 8)])).astype(np.int32)
    E_ref, _, s_ref = oracle.volume(params, ref, ns=ns)
    s_gpu = sonar.echoes(params)[0][ns]
    assert parity.nl2(s_gpu, s_ref) < S_TOL
    assert parity.nl2(E[:, ns], E_ref) <= 1e-4


# ------------------------------------------------------------------ synthesis kernels agree
@pytest.mark.parametrize("name,precision", [("c1", "fp32"), ("c2", "fp32"), ("c2", "bf16")])
def test_tensor_core_synthesis_matches_simt(sonar, name, precision):
    """Element echoes from the tensor-core synthesis against the FP32 SIMT kernel (both
    checked against the oracle elsewhere): FP32 form to S_TOL, BF16 form to 1e-2."""
    from paper_2606_06130_gb300.sonar import SONAR_OPT_SYNTH
    scene, params, poses, ssp = inputs.workload(name)
    out = {}
    for mode in (1, 0):
        sonar.set_option(SONAR_OPT_SYNTH, mode)
        E, _, _ = run(sonar, scene, params, poses[0], ssp, precision)
        out[mode] = (E, sonar.echoes(params)[0])
    sonar.set_option(SONAR_OPT_SYNTH, 0)
    tol = S_TOL if precision == "fp32" else 1e-2
    assert parity.nl2(out[0][1], out[1][1]) < tol
    assert parity.nl2(out[0][0], out[1][0]) < (1e-4 if precision == "fp32" else 1e-2)


@pytest.mark.parametrize("shape", [2, 3, 4])
@pytest.mark.parametrize("nx,ny,precision", [(32, 32, "fp32"), (16, 16, "fp32"), (8, 16, "fp32"), (32, 32, "bf16")])
def test_z_split_tile_shapes_match_simt(sonar, shape, nx, ny, precision):
    """The z-split kernel at each tile width (32, 64, 96 complex columns: synthesis
    option 2, 3, 4) with L2 = 8, 2 and 1 fine z elements per tile row, against the FP32
    SIMT kernel: FP32 form to S_TOL, BF16 form to 1e-2."""
    from paper_2606_06130_gb300.sonar import SONAR_OPT_SYNTH
    scene, params, poses, ssp = inputs.workload("c1")
    params = dict(params, nx=nx, ny=ny, n_beam_az=24, n_beam_el=12)
    out = {}
    for mode in (1, shape):
        sonar.set_option(SONAR_OPT_SYNTH, mode)
        E, _, _ = run(sonar, scene, params, poses[0], ssp, precision)
        out[mode] = (E, sonar.echoes(params)[0])
    sonar.set_option(SONAR_OPT_SYNTH, 0)
    tol = S_TOL if precision == "fp32" else 1e-2
    assert parity.nl2(out[shape][1], out[1][1]) < tol
    assert parity.nl2(out[shape][0], out[1][0]) < (1e-4 if precision == "fp32" else 1e-2)


# ------------------------------------------------------------------ C4: 64-ping trajectory
def test_c4_trajectory_batch_sampled_parity(sonar):
    """The full 64-ping batch in one call (the batch form the bench times), checked on
    four of its pings against the oracle's full volumes (every beam and range bin): the
    envelope to 1e-4, and the peak (beam, bin) of every beam whose oracle peak beats its
    runner-up and the threshold by the FP32 margin."""
    from paper_2606_06130_gb300.sonar import cloud_records
    scene, params, poses, ssp = inputs.workload("c4")
    sonar.upload(scene)
    env, cloud, n = sonar.ping_batch(poses, params, ssp)
    torch.cuda.synchronize()
    env = env.reshape(len(poses), -1, params["n_range"])
    total = 0
    for i in (0, 17, 40, 63):
        ref = oracle.trace(scene, params, poses[i], ssp)
        E_ref, _, _ = oracle.volume(params, ref)
        E = env[i].double().cpu().numpy()
        assert parity.nl2(E, E_ref) <= 1e-4, i
        assert int(n[i]) > 0
        checked, _ = cloud_check(cloud[i], int(n[i]), params, poses[i], E_ref, 1e-3)
        assert checked > 0.5 * len(cloud_records(cloud[i], int(n[i]))), i
        total += checked
    assert total > 1000


def test_c2_fp32_full_volume_peaks(sonar):
    """The headline ping at full size against the oracle's full volume (8192 beams x 1024
    bins): envelope normalised L2 <= 1e-4 and every peak (beam, bin) outside the FP32
    margin bit-exact."""
    scene, params, poses, ssp = inputs.workload("c2")
    E, cloud, n = run(sonar, scene, params, poses[0], ssp)
    ref = oracle.trace(scene, params, poses[0], ssp)
    E_ref, _, _ = oracle.volume(params, ref)
    assert parity.nl2(E, E_ref) <= 1e-4
    checked, excluded = cloud_check(cloud, n, params, poses[0], E_ref, 1e-3)
    assert checked > 0.9 * params["n_beam_az"] * params["n_beam_el"] - excluded
    assert checked > 4000


@pytest.mark.parametrize("name", ["c1", "c2", "c4"])
def test_device_lbvh_hit_parity(sonar, name):
    """The Morton-order LBVH built on the device (SONAR_OPT_BVH 1) gives the oracle's hits:
    prim ids bit-exact outside the near-tie margins, delays to 1e-12; and the envelope on
    sampled range bins to 1e-4 (c4: its first pose)."""
    from paper_2606_06130_gb300.sonar import SONAR_OPT_BVH
    scene, params, poses, ssp = inputs.workload(name)
    sonar.set_option(SONAR_OPT_BVH, 1)
    try:
        E, _, _ = run(sonar, scene, params, poses[0], ssp)
        hits = sonar.hits()
    finally:
        sonar.set_option(SONAR_OPT_BVH, 0)
    ref = oracle.trace(scene, params, poses[0], ssp)
    excluded, matched = parity.check_hits(hits, ref, params["n_sub"])
    assert matched >= ref["n"] - 2 * (excluded + 1)
    ns = np.arange(7, params["n_range"], max(1, params["n_range"] // 24), dtype=np.int32)
    E_ref, _, _ = oracle.volume(params, ref, ns=ns)
    assert parity.nl2(E[:, ns], E_ref) <= 1e-4


# ------------------------------------------------------------------ autotuner
def test_autotuned_batch_parity_and_choice(sonar):
    """The C4 64-ping batch with the autotuner on (the default): the first call of the
    shape tunes, the stats report a tuned N tile and synthesis width from the candidate
    sets, a second call reuses them, and the envelope matches the untuned heuristic's to
    the FP32 bound and the oracle on a sampled ping."""
    from paper_2606_06130_gb300.sonar import SONAR_OPT_AUTOTUNE
    scene, params, poses, ssp = inputs.workload("c4")
    sonar.upload(scene)
    sonar.set_option(SONAR_OPT_AUTOTUNE, 0)
    env0, _, _ = sonar.ping_batch(poses, params, ssp)
    torch.cuda.synchronize()
    st0 = sonar.stats()
    assert st0["autotuned"] == 0
    sonar.set_option(SONAR_OPT_AUTOTUNE, 1)
    env1, _, n1 = sonar.ping_batch(poses, params, ssp)
    torch.cuda.synchronize()
    st1 = sonar.stats()
    assert st1["autotuned"] == 1
    assert st1["tile_n"] in (128, 192, 224, 256) and st1["synth_cols"] in (32, 64, 96)
    env2, _, _ = sonar.ping_batch(poses, params, ssp)
    torch.cuda.synchronize()
    assert sonar.stats()["tile_n"] == st1["tile_n"] and sonar.stats()["synth_cols"] == st1["synth_cols"]
    a = env1.reshape(len(poses), -1, params["n_range"]).double().cpu().numpy()
    b = env0.reshape(len(poses), -1, params["n_range"]).double().cpu().numpy()
    assert parity.nl2(a, b) < 1e-4
    ns = np.arange(3, params["n_range"], 48, dtype=np.int32)
    ref = oracle.trace(scene, params, poses[21], ssp)
    E_ref, _, _ = oracle.volume(params, ref, ns=ns)
    assert parity.nl2(a[21][:, ns], E_ref) <= 1e-4


@pytest.mark.parametrize("name", ["c1", "c2", "c4"])
def test_warp_traversal_hit_parity(sonar, name):
    """The warp-cooperative traversal (SONAR_OPT_TRAVERSAL 1) gives the oracle's hits: prim
    ids bit-exact outside the near-tie margins, delays to 1e-12, and the same hit keys as
    the per-thread traversal; the envelope on sampled bins to 1e-4 (c4: its first pose)."""
    from paper_2606_06130_gb300.sonar import SONAR_OPT_TRAVERSAL
    scene, params, poses, ssp = inputs.workload(name)
    E0, _, _ = run(sonar, scene, params, poses[0], ssp)
    keys0 = np.sort(sonar.hits()["key"])
    sonar.set_option(SONAR_OPT_TRAVERSAL, 1)
    try:
        E, _, _ = run(sonar, scene, params, poses[0], ssp)
        hits = sonar.hits()
    finally:
        sonar.set_option(SONAR_OPT_TRAVERSAL, 0)
    assert np.array_equal(np.sort(hits["key"]), keys0)
    ref = oracle.trace(scene, params, poses[0], ssp)
    excluded, matched = parity.check_hits(hits, ref, params["n_sub"])
    assert matched >= ref["n"] - 2 * (excluded + 1)
    ns = np.arange(5, params["n_range"], max(1, params["n_range"] // 24), dtype=np.int32)
    E_ref, _, _ = oracle.volume(params, ref, ns=ns)
    assert parity.nl2(E[:, ns], E_ref) <= 1e-4
    assert parity.nl2(E, E0) < 1e-4  # the same hits, emitted in another order (FP32 atomics)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("tile_n", [128, 224, 256])
def test_cluster_gemm_equals_single_cta_gemm(sonar, precision, tile_n):
    """The beamforming GEMM in clusters of 2 and 4 CTAs sharing each steering tile by
    multicast against one CTA per tile (SONAR_OPT_GEMM_CLUSTER), on a batch of four pings
    of 128 range bins (four row tiles). Each form accumulates every tile in the same
    order; the element echoes they read may differ in the last bit between calls (the
    synthesis adds its tiles with FP32 atomics in any order), so the envelopes agree to
    1e-6 in the FP32 form and to 1e-4 in the BF16 form (where such a bit can move an
    echo's BF16 rounding by one step, 2^-9 relative), and the peaks on all but near-tied
    beams. The automatic choice is a cluster of two for the FP32 form, one CTA per tile
    for the BF16 form."""
    from paper_2606_06130_gb300.sonar import SONAR_OPT_GEMM_CLUSTER, SONAR_OPT_TILE_N, cloud_records
    scene, params, poses, ssp = inputs.workload("c1")
    params = dict(params, n_range=128, nx=32, ny=32, n_beam_az=48, n_beam_el=24)
    pp = [inputs.pose(poses[0]["t"] + np.array([0.1 * k, 0.0, 0.0]), yaw_deg=-6.0 + 4.0 * k, tilt_down_deg=15.0)
          for k in range(4)]
    sonar.upload(scene)
    sonar.set_option(SONAR_OPT_TILE_N, tile_n)
    out = {}
    try:
        for cs in (1, 2, 4, 0):
            sonar.set_option(SONAR_OPT_GEMM_CLUSTER, cs)
            env, cloud, n = sonar.ping_batch(pp, params, ssp, precision=precision)
            torch.cuda.synchronize()
            out[cs] = (env.reshape(len(pp), -1, params["n_range"]).cpu().numpy(),
                       [cloud_records(cloud[k], int(n[k])) for k in range(len(pp))], sonar.stats()["gemm_cluster"])
    finally:
        sonar.set_option(SONAR_OPT_TILE_N, 0)
        sonar.set_option(SONAR_OPT_GEMM_CLUSTER, 0)
    assert [out[cs][2] for cs in (1, 2, 4)] == [1, 2, 4]
    assert out[0][2] == (2 if precision == "fp32" else 1)
    tol = 1e-6 if precision == "fp32" else 1e-4
    ref_env, ref_pts, _ = out[1]
    for cs in (2, 4):
        env, pts, _ = out[cs]
        assert parity.nl2(env, ref_env) < tol, (cs, parity.nl2(env, ref_env))
        for got, want in zip(pts, ref_pts):
            assert abs(len(got) - len(want)) <= 2
            g = dict(zip(got["beam"].tolist(), got["bin"].tolist()))
            w = dict(zip(want["beam"].tolist(), want["bin"].tolist()))
            same = sum(1 for b in w if g.get(b) == w[b])
            assert same >= 0.99 * len(w), (cs, same, len(w))
