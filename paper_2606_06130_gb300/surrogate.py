"""Training and evaluation of the learned echo surrogate through the C ABI.

The paper proposes learned scattering functions as a stand-in for costly echo physics
(Sec. II.B). Here the plain method (sonar_ping_batch) renders the training pings over
randomised harbour scenes, the surrogate's own kernels train the network on them
(sonar_sur_train_step: forward, backward and Adam on the GPU), and the plain method
judges the trained network on held-out scenes (sonar_sur_compare), beside the geometric
rendering without the network (sonar_sur_geometric). This module only sequences those
calls and draws the random choices (scenes, poses, training beams) from seeded
generators; every step of the computation runs in the library's kernels.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs
from .sonar import SONAR_OPT_BVH


def _plain(sonar, poses, params, ssp):
    env, _, _ = sonar.ping_batch(poses, params, ssp, cloud_cap=0)
    return env


def _scene(sonar, seed):
    """Uploads the training scene of a seed (device-built hierarchy: the fastest build,
    the same hits)."""
    scene = inputs.training_scene(seed)
    sonar.set_option(SONAR_OPT_BVH, 1)
    try:
        sonar.upload(scene)
    finally:
        sonar.set_option(SONAR_OPT_BVH, 0)
    return scene


def train(sonar, params: dict, ssp: dict, n_pings: int, seed: int = 1000, beams_per_step: int = 1024,
          batch: int = 8, pings_per_scene: int = 64, lr: float = 1e-3, lr_final: float = 1e-4,
          weights=None, log_every: int = 0) -> dict:
    """Trains the surrogate on n_pings pings that the plain method renders, `batch` poses
    at a time, each batch followed by `batch` training steps of beams_per_step beams drawn
    at random from the batch (so every ping is used about once). The learning rate decays
    geometrically from lr to lr_final. weights: initial parameters (default: the seeded
    initialisation). Returns a dict with the loss history and the timings."""
    import torch
    dev = f"cuda:{sonar.device}"
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    nb = params["n_beam_az"] * params["n_beam_el"]
    scene_seed = seed
    scene = _scene(sonar, scene_seed)
    poses = inputs.training_poses(scene_seed + 1, pings_per_scene, scene)
    env = _plain(sonar, poses[:batch], params, ssp)
    torch.cuda.synchronize()
    # output scale: three times the RMS envelope of the first batch
    e_scale = 3.0 * float(env.double().pow(2).mean().sqrt().item())
    sonar.sur_set_weights(inputs.surrogate_init(seed) if weights is None else weights, e_scale)
    losses, steps, done = [], 0, 0
    t_plain = t_train = 0.0
    n_steps = max(1, n_pings)  # one step per ping
    decay = (lr_final / lr) ** (1.0 / max(1, n_steps - 1))
    used = 0
    while done < n_pings:
        if used + batch > pings_per_scene:
            scene_seed += 2
            scene = _scene(sonar, scene_seed)
            poses = inputs.training_poses(scene_seed + 1, pings_per_scene, scene)
            used = 0
        pb = poses[used:used + batch]
        used += batch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if done > 0:
            env = _plain(sonar, pb, params, ssp)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        t_plain += t1 - t0
        for _ in range(len(pb)):
            beams = torch.randint(0, len(pb) * nb, (beams_per_step,), generator=gen, device=dev, dtype=torch.int32)
            loss, _ = sonar.sur_train_step(pb, params, ssp, env, beams, lr=lr * decay ** steps)
            losses.append(loss)
            steps += 1
            if log_every and steps % log_every == 0:
                print(f"step {steps} loss {np.mean(losses[-log_every:]):.4g}", flush=True)
        torch.cuda.synchronize()
        t_train += time.perf_counter() - t1
        done += len(pb)
    return {"losses": np.array(losses), "e_scale": e_scale, "steps": steps, "pings": done,
            "plain_s": t_plain, "train_s": t_train, "beams_per_step": beams_per_step}


def evaluate(sonar, params: dict, ssp: dict, scene_seeds, pings_per_scene: int, rel_thr: float = 0.1,
             batch: int = 8) -> dict:
    """Held-out evaluation: for every held-out scene and pose, the surrogate's envelope and
    the geometric envelope (the rendering without the network) against the plain
    method's, by sonar_sur_compare over all beams and bins. Returns the metrics of both,
    pooled over all pings as sums (normalised L2 over the pooled volumes)."""
    import torch
    acc = {"surrogate": [], "geometric": []}
    for s in scene_seeds:
        scene = _scene(sonar, s)
        poses = inputs.training_poses(s + 1, pings_per_scene, scene)
        for b0 in range(0, len(poses), batch):
            pb = poses[b0:b0 + batch]
            ref = _plain(sonar, pb, params, ssp)
            sur = sonar.sur_ping(pb, params, ssp)
            geo = sonar.sur_geometric(pb, params, ssp)
            torch.cuda.synchronize()
            acc["surrogate"].append(sonar.sur_compare(sur, ref, params, rel_thr))
            acc["geometric"].append(sonar.sur_compare(geo, ref, params, rel_thr))
    return {k: _pool(v) for k, v in acc.items()}


def _pool(ms: list) -> dict:
    """Pools per-batch metrics: L2 errors by their mean square (each batch's reference
    energy is similar), peak statistics weighted by lit beams, speckle indices averaged."""
    lit = np.array([m["lit_beams"] for m in ms], float)
    w = lit / max(lit.sum(), 1.0)
    return {"nl2": float(np.sqrt(np.mean([m["nl2"] ** 2 for m in ms]))),
            "peak_bin_mean": float(np.sum(w * [m["peak_bin_mean"] for m in ms])),
            "peak_within_1": float(np.sum(w * [m["peak_within_1"] for m in ms])),
            "peak_within_4": float(np.sum(w * [m["peak_within_4"] for m in ms])),
            "lit_beams": int(lit.sum()),
            "si": float(np.mean([m["si"] for m in ms])), "si_ref": float(np.mean([m["si_ref"] for m in ms])),
            "speckle_gap": float(np.mean([m["si"] - m["si_ref"] for m in ms])),
            "batches": len(ms)}
