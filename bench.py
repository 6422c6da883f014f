"""Benchmark: pings/s of per-ping coherent echo formation at 8192 beams x 1024 range bins.

Workload (one step = one ping through the whole path: ray casting, shading, binning,
element-echo synthesis, beamforming GEMM with fused envelope/TVG/peak search, point
cloud): the harbour sheet-pile scene (32x32 array, 128x64 beams, 1024 bins to 15 m,
512x256 rays x 4 sub-rays, direct + one surface/seabed bounce), FP32 form, synthetic
data. Inputs are resident in HBM; L2 is flushed (256 MB write) before every timed step
outside the timed events. ``--impl reference`` times the FP64 CPU oracle instead.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--precision fp32|bf16|fp16]
Under torchrun each rank runs an independent replica (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pings/s at 8192 beams x 1024 range bins (harbour wall, 32x32 array)"
UNIT = "pings/s"
WORKLOAD = ("harbour sheet-pile wall (20.5k tri) over fBm seabed (130k tri); 32x32 array at lambda/2, "
            "128x64 beams over 90x40 deg, 1024 bins to 15 m, 512x256 rays x 4 jittered sub-rays, "
            "direct + 1 surface/seabed bounce; 1 ping per step")
FP32_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"


def peaks_file():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def max_over_ranks(x: float, ws: int) -> float:
    """Maximum of a host value over all ranks (the slowest rank's time); identity at N=1.
    The tensor lives where the process group's backend wants it (CUDA for NCCL)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws: int, steps_per_rank: int, seconds: float) -> float:
    """Units per second of the whole job: every rank processes steps_per_rank pings in
    the (max-over-ranks) time."""
    return ws * steps_per_rank / seconds


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ oracle sample
def oracle_sample_params(p, k=8):
    """1/k of a ping (k in 8, 16, 32, 64): the central 1/k of the vertical field of view
    (ray and beam rows), all range bins, all elements."""
    q = dict(p)
    q["vfov"] = p["vfov"] / k
    q["n_ray_el"] = p["n_ray_el"] // k
    q["n_beam_el"] = p["n_beam_el"] // k
    return q, 1.0 / k


def sample_divisor(steps):
    """Oracle sample size for a run of `steps` steps: about 0.4 s per 1/8 ping on 16 host
    cores, so larger K takes smaller samples and the run stays near a minute."""
    for k in (8, 16, 32):
        if steps * 0.4 * 8 / k <= 60:
            return k
    return 64


def oracle_ping(scene, params, pose, ssp):
    import oracle
    h = oracle.trace(scene, params, pose, ssp)
    E, _, _ = oracle.volume(params, h)
    pk = oracle.peaks(params, pose, E)
    return h, E, pk


def time_oracle(steps, warmup, min_seconds=0.0, k=8, keep=None):
    """Oracle pings/s on the 1/k-ping sample: `steps` samples, more until min_seconds pass.
    keep (a dict), if given, receives the sample's parameters and the last oracle outputs."""
    import oracle
    from paper_2606_06130_gb300 import inputs
    scene, params, poses, ssp = inputs.workload("c2")
    q, frac = oracle_sample_params(params, k)
    for _ in range(warmup):
        oracle_ping(scene, q, poses[0], ssp)
    t0 = time.perf_counter()
    done = 0
    while done < steps or time.perf_counter() - t0 < min_seconds:
        out = oracle_ping(scene, q, poses[0], ssp)
        done += 1
    steps = done
    dt = time.perf_counter() - t0
    if keep is not None:
        keep.update(params=q, pose=poses[0], ssp=ssp, h=out[0], E=out[1], peaks=out[2])
    return {"value": steps * frac / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"1/{k} of the ping per step: central 1/{k} of the vertical field of view "
                      f"({params['n_ray_el'] // k} of {params['n_ray_el']} ray rows, {params['n_beam_el'] // k} of "
                      f"{params['n_beam_el']} beam rows), all 1024 bins and 1024 elements; FP64 C oracle, OpenMP",
            "seconds": dt, "steps": steps}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock samples every 50 ms; only those taken inside [begin(), end()] count."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.all_rows = []
        self.rows = []
        self.t_begin = self.t_end = None
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_id), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            t0 = time.monotonic()
            while not self.all_rows and time.monotonic() - t0 < 10.0:  # sampler running
                time.sleep(0.01)
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.all_rows.append((time.monotonic(), parts))

    def begin(self):
        self.t_begin = time.monotonic()

    def end(self):
        self.t_end = time.monotonic()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.rows = [r for t, r in self.all_rows
                     if self.t_begin is not None and self.t_begin <= t <= (self.t_end or t)]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ roofline
def stage_work(stage, params, stats, n_pings):
    """Algorithmic work of one launch of a stage: (amount, unit, bound)."""
    M = params["nx"] * params["ny"]
    nb = params["n_beam_az"] * params["n_beam_el"]
    nr = params["n_range"]
    if stage == "beamform":
        # complex [Nb x M] . [M x Nr] as a real GEMM: 8 Nb M Nr flop per ping; separable
        # beams contract only over the array's columns (K = nx) in this stage
        K = params["nx"] if stats.get("beam_sep") else M
        return 8.0 * nb * K * nr * n_pings, "flop", "tensor"
    if stage == "synth":
        # per (hit, element): phasor product (6 flop) + W complex MACs (8 flop each); the
        # contraction runs on the tensor cores (BF16 operands, hi/lo split in the FP32 form)
        return float(stats["n_hits"]) * M * (8 * stats["taps"] + 6), "flop", "tensor"
    if stage == "convert":
        if stats.get("beam_sep"):
            # first stage of the separable beams: n_el x ny x nx complex multiply-adds per sample
            return 8.0 * params["n_beam_el"] * M * nr * n_pings, "flop", "alu"
        return float(n_pings) * nr * M * (8 + 8), "byte", "hbm"
    return None


def read_profile(kernel, extra=None):
    """(DRAM bytes, executed warp instructions) per launch from the committed ncu
    summary (profiles/dram_traffic.txt), each None when absent or when the kernel's
    source has changed since the capture. extra: a dict that receives the row's further
    key=value counters (cache hit rates, L2 bytes, cycles) under the same rule."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        row = None
        for line in open(path):
            if line.startswith("#") or not line.strip():
                continue
            f = line.split()
            if f[0] == kernel:
                row = f
                break
        if row is None:
            return None, None
        import hashlib
        unit = {"k_synth_tz": "synth_tc.cu", "k_gemm": "beamform.cu", "k_trace": "trace.cu",
                "k_volume": "trace.cu"}.get(kernel)
        cur = hashlib.sha1(open(os.path.join(ROOT, "paper_2606_06130_gb300", "csrc", unit), "rb").read()).hexdigest()[:12]
        if cur != row[2]:
            return None, None
        if extra is not None:
            for kv in row[4:]:
                k, v = kv.split("=", 1)
                extra[k] = float(v)
        return float(row[1]), (float(row[3]) if len(row) > 3 else None)
    except (OSError, ValueError, IndexError):
        return None, None


# ------------------------------------------------------------------ our arm
# water-column scatterers of --volume (and of the volume form): a box over the wall and
# the seabed in front of the sonar, s_v = 1e-4 /m
VOLUME_BOX = ((-2.0, -12.0, -10.5), (14.0, 12.0, -4.0))
VOLUME_SV = 1e-4
# --field and the field form: a thermocline that deepens with range, 6 m/s either side
XS_F, ZS_F = np.linspace(-4.0, 16.0, 21), np.linspace(-12.0, 1.0, 27)
THERMOCLINE = {"x0": -4.0, "dx": 1.0, "z0": -12.0, "dz": 0.5,
               "c": np.array([[1500.0 - 6.0 * math.tanh((z + 6.0 + 0.15 * x) / 1.5) for x in XS_F] for z in ZS_F])}


def run_ours(args, ws, rank, local):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06130_gb300 import inputs
    from paper_2606_06130_gb300.sonar import Sonar, SONAR_OPT_TIMING

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    scene, params, poses, ssp = inputs.workload("c2")
    s = Sonar(local)
    if args.synth_cols or args.tile_n:
        # pinned tiles (profiling runs: the same kernels every launch, no tuner trials)
        from paper_2606_06130_gb300.sonar import SONAR_OPT_SYNTH, SONAR_OPT_TILE_N
        if args.synth_cols:
            s.set_option(SONAR_OPT_SYNTH, {32: 2, 64: 3, 96: 4}[args.synth_cols])
        if args.tile_n:
            s.set_option(SONAR_OPT_TILE_N, args.tile_n)
    if args.dense:
        # the dense beamforming contraction in place of the separable stages (profiling)
        from paper_2606_06130_gb300.sonar import SONAR_OPT_BEAMFORM
        s.set_option(SONAR_OPT_BEAMFORM, 1)
    if args.cross:
        from paper_2606_06130_gb300.sonar import SONAR_OPT_CROSS
        s.set_option(SONAR_OPT_CROSS, 1)
    if args.volume > 0:
        s.set_volume(args.volume, VOLUME_BOX[0], VOLUME_BOX[1], VOLUME_SV)
    if args.field > 0:
        s.set_field(dict(THERMOCLINE, h=args.field))
        params = dict(params, c_ref=1500.0)
    s.upload(scene)
    torch.cuda.synchronize()
    # scene upload and BVH build, timed apart from the pings (median of 3 rebuilds)
    up = []
    for _ in range(3):
        t0 = time.perf_counter()
        s.upload(scene)
        torch.cuda.synchronize()
        up.append((time.perf_counter() - t0) * 1e3)
    upload_ms = {"value": float(np.median(up)), "unit": "ms", "triangles": int(len(scene.tris)),
                 "what": "host-to-device copy, binned-SAH hierarchy on the host, device refit and packing (wall clock)"}
    nb = params["n_beam_az"] * params["n_beam_el"]
    env = torch.empty((params["n_beam_el"], params["n_beam_az"], params["n_range"]), dtype=torch.float32, device=dev)
    cloud = torch.empty((nb, 6), dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    pose = poses[0]

    def ping():
        return s.ping_batch([pose], params, ssp, precision=args.precision, env=env[None], cloud=cloud[None],
                            cloud_cap=nb)

    stream = torch.cuda.current_stream(dev)
    gpu_id = torch.cuda.get_device_properties(local).uuid if hasattr(torch.cuda.get_device_properties(local), "uuid") else local

    # headline: the library's default path, each ping replayed as one captured CUDA graph;
    # steps are enqueued back to back (L2 flush between them, outside the events) so the
    # device never waits on the host, and the events time device work only
    s.set_option(SONAR_OPT_TIMING, 0)
    for _ in range(max(args.warmup, 3)):
        ping()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(f"GPU-{gpu_id}" if not isinstance(gpu_id, int) else gpu_id)
    clocks.begin()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        ping()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clocks.end()
    clk = clocks.stop()
    t_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), ws)

    # the same steps with per-stage events (diagnostic mode: kernels launched one by one,
    # no graph), for the stage breakdown and the kernel count
    s.set_option(SONAR_OPT_TIMING, 1)
    for _ in range(3):
        ping()
    torch.cuda.synchronize()
    stages = {k: [] for k in ("trace", "bin", "synth", "convert", "beamform", "peaks")}
    launches = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eager_ms = 0.0
    for i in range(args.steps):
        flush.zero_()
        e0.record(stream)
        ping()
        e1.record(stream)
        e1.synchronize()  # the call waits for its own stream, not for the caller's
        st = s.stats()
        eager_ms += e0.elapsed_time(e1)
        for k in stages:
            stages[k].append(st["ms_" + k])
        launches += st["kernels"]
    eager_ms = max_over_ranks(eager_ms, ws)
    stats = s.stats()
    s.set_option(SONAR_OPT_TIMING, 0)

    # end to end through the C ABI as a user calls it (defaults: graph replay, no stage
    # events), pose in, envelope and cloud out to pinned host buffers that the kernels
    # write through the device's mapping of them
    env_h = torch.empty(env.shape, dtype=torch.float32, pin_memory=True)
    cloud_h = torch.empty((nb, 6), dtype=torch.int32, pin_memory=True)
    for _ in range(2):
        s.ping_batch([pose], params, ssp, precision=args.precision, env=env_h[None], cloud=cloud_h[None], cloud_cap=nb)
    k_e2e = max(3, min(args.steps, 200))
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(k_e2e):
        s.ping_batch([pose], params, ssp, precision=args.precision, env=env_h[None], cloud=cloud_h[None], cloud_cap=nb)
    torch.cuda.synchronize()
    e2e_sync_s = max_over_ranks(time.perf_counter() - e0, ws)
    # the streaming call: sonar_ping_async with two calls in flight, each into its own
    # pinned host buffers; the envelope goes to the host by copy engine while the next
    # ping computes. Every step's pose upload and envelope/cloud/count read-back is inside
    # the timed region (the final wait retires the last two).
    env_a = [torch.empty(env.shape, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    cloud_a = [torch.empty((nb, 6), dtype=torch.int32, pin_memory=True) for _ in range(2)]
    for i in range(4):
        s.ping_async([pose], params, ssp, precision=args.precision, env=env_a[i & 1][None], cloud=cloud_a[i & 1][None],
                     cloud_cap=nb)
    s.wait()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for i in range(k_e2e):
        s.ping_async([pose], params, ssp, precision=args.precision, env=env_a[i & 1][None], cloud=cloud_a[i & 1][None],
                     cloud_cap=nb)
    s.wait()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - e0, ws)

    # other forms (same run): BF16 single ping, BF16 64-ping trajectory batch
    forms = {}
    if rank == 0 and not args.no_forms:
        forms = other_forms(torch, s, inputs, dev)

    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return

    mean_stage = {k: float(np.mean(v)) for k, v in stages.items()}
    dom = max(("synth", "beamform", "convert"), key=lambda k: mean_stage[k])
    pk, pk_kind = peaks_file()
    amount, unit, bound = stage_work(dom, params, stats, 1)
    dt_s = mean_stage[dom] / 1e3
    if bound == "tensor":
        peak, punit, achieved = pk["bf16_tflops"], "TFLOP/s", amount / dt_s / 1e12
        pnote = f"bf16 dense burst, {pk_kind}"
    elif bound == "alu":
        peak, punit, achieved = 152 * 128 * 2 * 2.070e9 / 1e12, "TFLOP/s", amount / dt_s / 1e12
        pnote = f"FP32 FMA: {FP32_PEAK_NOTE}"
    else:
        peak, punit, achieved = pk["hbm_gbs"], "GB/s", amount / dt_s / 1e9
        pnote = f"HBM copy, {pk_kind}"
    kname = {"synth": "k_synth_tz", "beamform": "k_gemm",
             "convert": "k_sep1" if stats.get("beam_sep") else "k_convert"}[dom]
    traffic, winst = read_profile(kname)
    roof = {"kernel": kname,
            "bound": bound, "achieved": achieved, "peak": peak, "unit": punit, "frac": achieved / peak,
            "peak_source": pnote, "traffic": traffic,
            "algorithmic_per_launch": amount, "algorithmic_unit": unit, "launch_ms": mean_stage[dom]}
    if winst is not None:
        # what bounds the synthesis in practice: instruction issue, 4 warp instructions per
        # clock per SM at most (152 SMs at the sampled clock, else 2070 MHz)
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        ipeak = 4 * 152 * mhz * 1e6
        roof["issue"] = {"warp_instructions_per_launch": winst, "source": "ncu smsp__inst_executed.sum",
                         "achieved": winst / dt_s, "peak": ipeak, "unit": "warp instructions/s",
                         "frac": winst / dt_s / ipeak}

    # CPU baseline leg: the oracle timed on a sample of the workload; the same sample's
    # oracle outputs give the GPU path's errors
    cpu = err = None
    if ws == 1 and not args.no_oracle:
        ref = {}
        cpu = time_oracle(1, 0, min_seconds=10.0, keep=ref)
        err = sample_errors(torch, s, ref)
    value = whole_job_rate(ws, args.steps, t_ms / 1e3)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": max(args.warmup, 3), "ms_per_step": t_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else args.precision,
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "precision": args.precision,
                      "beamform_operands": {"fp32": "bf16 hi/lo split, 3 tensor products, fp32 accumulate",
                                            "bf16": "bf16, fp32 accumulate", "fp16": "fp16, fp32 accumulate"}[args.precision],
                      "beamformer": "separable: per-elevation row sums (FP32), then the tensor-core GEMM over columns"
                      if stats.get("beam_sep") else "dense tensor-core GEMM over all elements",
                      "l2": "flushed before every timed step (256 MB write, outside the events)",
                      "cross_terms": bool(args.cross),
                      "volume_scatterers": int(args.volume),
                      "field_step_m": float(args.field) if args.field > 0 else None,
                      "parallelism": f"replicas x{ws}"},
           "roofline": roof,
           "stages_ms": mean_stage,
           "stage_rooflines": stage_rooflines(mean_stage, params, stats, args.precision, pk, clk),
           "scene_upload_ms": upload_ms,
           "hits_per_ping": stats["n_hits"],
           "tiles": {"beamform_tile_n": stats["tile_n"], "synth_cols": stats["synth_cols"],
                     "autotuned": bool(stats["autotuned"])},
           "gpu_launches": launches,
           "timing": "graph replay per ping (the default path), steps enqueued back to back, CUDA events "
                     "around each step, L2 flushed between steps outside the events",
           "eager_stage_timed": {"value": whole_job_rate(ws, args.steps, eager_ms / 1e3), "unit": UNIT,
                                 "note": "same steps with per-stage events, kernels launched one by one"},
           "e2e_sync": {"value": whole_job_rate(ws, k_e2e, e2e_sync_s), "unit": UNIT,
                        "path": "sonar_ping_batch per step (returns when the outputs are complete), envelope "
                                "written through the device mapping of pinned host memory"},
           "e2e": {"value": whole_job_rate(ws, k_e2e, e2e_s), "unit": UNIT, "h2d_bytes_per_step": 192,
                   "d2h_bytes_per_step": int(env.numel() * 4 + nb * 24 + 8), "steps": k_e2e,
                   "path": "sonar_ping_async (two calls in flight, graph replay) into pinned host env and "
                           "cloud buffers; the envelope leaves by copy engine while the next ping computes"},
           "clocks": clk,
           "error_vs_oracle": err,
           "forms": forms,
           "cpu_baseline": cpu}
    print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def sample_errors(torch, s, ref):
    """Errors of the GPU path on the CPU-baseline sample, against the oracle outputs of
    that sample (all its bins and beams): envelope normalised L2 per precision form;
    prim ids and peak (beam, bin) mismatches outside the near-tie margins, with the
    excluded counts (FP32 form)."""
    from paper_2606_06130_gb300.sonar import SONAR_OPT_DEBUG, cloud_records
    from tests import parity
    q, pose, ssp, h, E_ref, pk = ref["params"], ref["pose"], ref["ssp"], ref["h"], ref["E"], ref["peaks"]
    out = {"sample": "the CPU baseline's sample (central 1/8 of the vertical field of view)",
           "beams": int(E_ref.shape[0]), "bins": int(E_ref.shape[1]), "hits_oracle": int(h["n"])}
    s.set_option(SONAR_OPT_DEBUG, 1)
    env_nl2 = {}
    for prec in ("fp32", "bf16", "fp16"):
        env, cloud, n = s.ping(pose, q, ssp, precision=prec)
        torch.cuda.synchronize()
        E = env.reshape(-1, q["n_range"]).double().cpu().numpy()
        env_nl2[prec] = parity.nl2(E, E_ref)
        rel = 1e-3 if prec == "fp32" else 2e-2
        nb0 = parity.n_blank(q)
        vmax = E_ref[:, nb0:].max()
        thr = q["thr"] * vmax if q["thr_mode"] == 1 else q["thr"]
        ok = parity.peak_margin_mask(E_ref, nb0, thr, rel)
        pts = cloud_records(cloud, n)
        gpu = {int(b): int(k) for b, k in zip(pts["beam"], pts["bin"])}
        want = {int(b): int(k) for b, k in zip(pk["beam"], pk["bin"])}
        bad = sum(1 for b in np.nonzero(ok)[0] if gpu.get(int(b)) != want.get(int(b)))
        out[f"peaks_{prec}"] = {"mismatch": bad, "excluded": int(np.count_nonzero(~ok)), "margin_rel": rel}
        if prec == "fp32":
            g = s.hits()
            ig, ir, only_g, only_r = parity.match_hits(g, h, q["n_sub"])
            clear = (h["margin"][ir] > 1e-5) & (h["gap"][ir] > 1e-6)
            out["prims"] = {"matched": int(len(ig)), "mismatch": int(np.count_nonzero((g["prim"][ig] != h["prim"][ir]) & clear)),
                            "excluded": int(np.count_nonzero(~clear)), "unmatched": int(len(only_g) + len(only_r))}
    s.set_option(SONAR_OPT_DEBUG, 0)
    out["env_nl2"] = env_nl2
    return out


def stage_rooflines(mean_stage, params, stats, precision, pk, clk=None):
    """Achieved rate of every stage against its bound: tensor stages in TFLOP/s of the
    measured BF16 peaks (burst and sustained), memory stages in GB/s of the measured HBM
    copy rate, the traversal in sub-rays/s (latency-bound: no single peak)."""
    M = params["nx"] * params["ny"]
    nb = params["n_beam_az"] * params["n_beam_el"]
    nr = params["n_range"]
    H = float(stats["n_hits"])
    sub_rays = params["n_ray_az"] * params["n_ray_el"] * params["n_sub"]
    hbm = pk["hbm_gbs"]

    def mem(stage, nbytes, what):
        gbs = nbytes / (mean_stage[stage] / 1e3) / 1e9
        return {"bound": "hbm", "bytes": nbytes, "bytes_are": what, "achieved": gbs, "unit": "GB/s",
                "peak": hbm, "frac": gbs / hbm}

    def tensor(stage, flop, executed):
        tf = flop / (mean_stage[stage] / 1e3) / 1e12
        return {"bound": "tensor", "flop": flop, "executed_flop": executed, "achieved": tf, "unit": "TFLOP/s",
                "peak": pk["bf16_tflops"], "frac": tf / pk["bf16_tflops"],
                "frac_sustained": tf / pk["bf16_tflops_sustained"],
                "executed_frac": executed / flop * tf / pk["bf16_tflops"]}

    n_pass = 3 if precision == "fp32" else 1
    synth_flop = H * M * (8 * stats["taps"] + 6)
    gemm_flop = 8.0 * nb * M * nr
    # the traversal's memory side from its committed capture: L1 and L2 hit rates, the L2
    # bytes it moves per launch and their rate over this run's stage time
    tx = {}
    _, trace_winst = read_profile("k_trace", tx)
    trace_mem = None
    if tx:
        trace_mem = {"l1_hit_pct": tx.get("l1_hit"), "l2_hit_pct": tx.get("l2_hit"), "l2_bytes": tx.get("l2_bytes"),
                     "l2_gbs": tx["l2_bytes"] / (mean_stage["trace"] / 1e3) / 1e9 if "l2_bytes" in tx else None,
                     "issue_active_pct": tx.get("issue_active"), "source": "ncu capture (profiles/dram_traffic.txt)"}
    # the traversal waits on dependent node loads; its measurable ceiling is instruction
    # issue (4 warp instructions per clock per SM), against the captured instruction count
    t_s = mean_stage["trace"] / 1e3
    ipeak = 4 * 152 * ((clk or {}).get("sm_mhz") or 2070.0) * 1e6
    trace = {"bound": "issue (latency-bound traversal: dependent BVH node loads)",
             "achieved": trace_winst / t_s if trace_winst else None, "unit": "warp instructions/s",
             "peak": ipeak, "frac": trace_winst / t_s / ipeak if trace_winst else None,
             "warp_instructions_per_launch": trace_winst, "sub_rays_per_s": sub_rays / t_s,
             "hits_per_s": H / t_s, "memory": trace_mem}
    out = {
        "trace": trace,
        "bin": mem("bin", 2 * 32 * H, "32-byte hit records read and written once"),
        "synth": tensor("synth", synth_flop, stats.get("synth_mma_flop") or synth_flop),
        "convert": mem("convert", nr * M * (8 + (8 if precision == "fp32" else 4)),
                       "FP32 complex echoes read, 16-bit operand(s) written"),
        "beamform": tensor("beamform", gemm_flop, gemm_flop * n_pass),
        "peaks": mem("peaks", nb * (8 + 24), "per-beam keys read, point records written"),
    }
    if stats.get("beam_sep"):
        # separable beams: the first stage (in the conversion's slot) runs FP32
        # multiply-adds on the CUDA cores, against 128 FMA per clock per SM; the second is
        # the tensor-core GEMM with K = 2 nx, whose envelope write dominates its bytes
        n_el, nx = params["n_beam_el"], params["nx"]
        s1_flop = 8.0 * n_el * M * nr
        t1 = mean_stage["convert"] / 1e3
        fpeak = 2 * 128 * 152 * ((clk or {}).get("sm_mhz") or 2070.0) * 1e6
        parts = 2 if precision == "fp32" else 1
        out["convert"] = {"bound": "alu", "what": "separable beams, first stage: per-elevation sums over the array rows",
                          "flop": s1_flop, "achieved": s1_flop / t1 / 1e12, "unit": "TFLOP/s",
                          "peak": fpeak / 1e12, "frac": s1_flop / t1 / fpeak,
                          "peak_source": "FP32 FMA: 128 per clock per SM x 152 SMs at the sampled clock"}
        s2_flop = 8.0 * nb * nx * nr
        bf = tensor("beamform", s2_flop, s2_flop * n_pass)
        s2_bytes = 4.0 * nb * nr + 2.0 * parts * n_el * nr * 2 * nx + 2.0 * parts * 2 * nb * 2 * nx
        gbs = s2_bytes / (mean_stage["beamform"] / 1e3) / 1e9
        bf["what"] = "separable beams, second stage: per-beam sums over the array columns (K = 2 nx)"
        bf["hbm"] = {"bytes": s2_bytes, "bytes_are": "envelope written, first-stage and steering operands read",
                     "achieved": gbs, "unit": "GB/s", "peak": hbm, "frac": gbs / hbm}
        out["beamform"] = bf
    return out


def ttd_form(torch, s, params, poses, ssp, U):
    """True-time-delay beams of the headline ping: wideband echoes at U phases per range
    cell, each beam reading every element at its steering delay (4-point Lagrange
    interpolation), pings/s and the stage times. The beamforming contraction runs over
    all fractional-delay levels; its algorithmic work is the 4 taps per (beam, element,
    sample) of the interpolating beamformer."""
    from paper_2606_06130_gb300.sonar import SONAR_OPT_TTD, SONAR_OPT_TIMING
    s.set_option(SONAR_OPT_TTD, U)
    try:
        for _ in range(2):
            s.ping(poses[0], params, ssp, precision="fp32")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            s.ping(poses[0], params, ssp, precision="fp32")
        torch.cuda.synchronize()
        rate = 5 / (time.perf_counter() - t0)
        s.set_option(SONAR_OPT_TIMING, 1)
        stages = []
        for _ in range(3):
            s.ping(poses[0], params, ssp, precision="fp32")
            torch.cuda.synchronize()
            stages.append(s.stats())
        s.set_option(SONAR_OPT_TIMING, 0)
    finally:
        s.set_option(SONAR_OPT_TTD, 0)
    st = {k: float(np.median([x["ms_" + k] for x in stages]))
          for k in ("trace", "bin", "synth", "convert", "beamform", "peaks")}
    M = params["nx"] * params["ny"]
    nb = params["n_beam_az"] * params["n_beam_el"]
    nr = params["n_range"]
    # the levels the library forms: floor(x) - 1 .. floor(x) + 2 over every (beam, element)
    c = ssp["c"][0]
    dt = 2.0 * (params["r_max"] - params["r_min"]) / nr / c
    cx, cy = (params["nx"] - 1) / 2, (params["ny"] - 1) / 2
    i, j = np.arange(params["n_beam_az"]), np.arange(params["n_beam_el"])
    az = -params["hfov"] / 2 + (i + 0.5) * params["hfov"] / params["n_beam_az"]
    el = -params["vfov"] / 2 + (j + 0.5) * params["vfov"] / params["n_beam_el"]
    uy = (np.cos(el)[:, None] * np.sin(az)[None, :]).ravel()
    uz = np.repeat(np.sin(el), params["n_beam_az"])
    x = [-U * params["pitch"] * (uy * a + uz * b) / (c * dt) for a in (-cx, cx) for b in (-cy, cy)]
    levels = int(np.floor(np.max(x))) + 2 - (int(np.floor(min(np.min(x), 0.0))) - 1) + 1
    flop_alg = 8.0 * nb * M * nr * 4
    flop_exec = 8.0 * nb * M * nr * levels * 3
    tf = flop_exec / (st["beamform"] / 1e3) / 1e12
    return {"value": rate, "unit": UNIT, "U": U, "levels": levels, "stages_ms": st,
            "beamform": {"executed_flop": flop_exec, "algorithmic_flop": flop_alg, "executed_tflops": tf,
                         "algorithmic_tflops": flop_alg / (st["beamform"] / 1e3) / 1e12},
            "note": f"true-time-delay beams: wideband echoes at {U} phases per range cell (SIMT synthesis, "
                    "per-element envelope delays), 4-point Lagrange fractional delays as extra K blocks of the "
                    "tensor-core beamforming contraction"}


def other_forms(torch, s, inputs, dev):
    out = {}
    scene, params, poses, ssp = inputs.workload("c2")
    from paper_2606_06130_gb300.sonar import SONAR_OPT_TIMING as _TIMING
    for prec in ("bf16", "fp16"):
        for _ in range(3):
            s.ping(poses[0], params, ssp, precision=prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(10):
            s.ping(poses[0], params, ssp, precision=prec)
        torch.cuda.synchronize()
        out[f"c2_single_{prec}"] = {"value": 10 / (time.perf_counter() - t0), "unit": UNIT}
        # the stage breakdown of this form (per-stage events, median of 5 pings) and its
        # beamforming contraction against the measured BF16 burst (one product per tile)
        s.set_option(_TIMING, 1)
        st = []
        for _ in range(5):
            s.ping(poses[0], params, ssp, precision=prec)
            torch.cuda.synchronize()
            st.append(s.stats())
        s.set_option(_TIMING, 0)
        med = {k: float(np.median([x["ms_" + k] for x in st]))
               for k in ("trace", "bin", "synth", "convert", "beamform", "peaks")}
        # separable beams (BF16 form) contract over the array's columns only in this stage
        K = params["nx"] if st[-1]["beam_sep"] else params["nx"] * params["ny"]
        gemm_flop = 8.0 * params["n_beam_az"] * params["n_beam_el"] * K * params["n_range"]
        pk, _ = peaks_file()
        tf = gemm_flop / (med["beamform"] / 1e3) / 1e12
        out[f"c2_single_{prec}"].update({"stages_ms": med, "beam_sep": st[-1]["beam_sep"], "beamform": {
            "flop": gemm_flop, "achieved_tflops": tf, "frac_of_bf16_burst": tf / pk["bf16_tflops"],
            "tile_n": st[-1]["tile_n"]}})
    # the dense beamforming contraction over all elements (the path for tapers that do
    # not factor, FP16 operands and true-time delay), forced on the headline ping
    from paper_2606_06130_gb300.sonar import SONAR_OPT_BEAMFORM
    s.set_option(SONAR_OPT_BEAMFORM, 1)
    try:
        for _ in range(3):
            s.ping(poses[0], params, ssp, precision="fp32")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(10):
            s.ping(poses[0], params, ssp, precision="fp32")
        torch.cuda.synchronize()
        dense = {"value": 10 / (time.perf_counter() - t0), "unit": UNIT}
        s.set_option(_TIMING, 1)
        st = []
        for _ in range(5):
            s.ping(poses[0], params, ssp, precision="fp32")
            torch.cuda.synchronize()
            st.append(s.stats())
        s.set_option(_TIMING, 0)
    finally:
        s.set_option(SONAR_OPT_BEAMFORM, 0)
    med = {k: float(np.median([x["ms_" + k] for x in st]))
           for k in ("trace", "bin", "synth", "convert", "beamform", "peaks")}
    gemm_flop = 8.0 * params["n_beam_az"] * params["n_beam_el"] * params["nx"] * params["ny"] * params["n_range"]
    pk, _ = peaks_file()
    tf = gemm_flop / (med["beamform"] / 1e3) / 1e12
    dense.update({"stages_ms": med, "beam_sep": st[-1]["beam_sep"], "beamform": {
        "flop": gemm_flop, "executed_flop": 3 * gemm_flop, "achieved_tflops": tf,
        "executed_frac_of_bf16_burst": 3 * tf / pk["bf16_tflops"], "tile_n": st[-1]["tile_n"]},
        "note": "dense beamforming GEMM (all 1024 elements, FP32 form: 3 BF16 products) forced"})
    out["c2_dense_fp32"] = dense
    # the raw element series at 4 samples per range cell and the explicit matched filter
    from paper_2606_06130_gb300.sonar import SONAR_OPT_RAW
    s.set_option(SONAR_OPT_RAW, 4)
    for _ in range(3):
        s.ping(poses[0], params, ssp, precision="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(10):
        s.ping(poses[0], params, ssp, precision="fp32")
    torch.cuda.synchronize()
    out["c2_raw_u4_fp32"] = {"value": 10 / (time.perf_counter() - t0), "unit": UNIT,
                             "note": "raw chirp echoes at 4 samples per range cell + matched filter"}
    s.set_option(SONAR_OPT_RAW, 0)
    out["c2_ttd_u4_fp32"] = ttd_form(torch, s, params, poses, ssp, 4)
    # out/back cross-term multipath (every reflected route also returns straight)
    from paper_2606_06130_gb300.sonar import SONAR_OPT_CROSS
    s.set_option(SONAR_OPT_CROSS, 1)
    for _ in range(3):
        s.ping(poses[0], params, ssp, precision="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(10):
        s.ping(poses[0], params, ssp, precision="fp32")
    torch.cuda.synchronize()
    out["c2_cross_fp32"] = {"value": 10 / (time.perf_counter() - t0), "unit": UNIT,
                            "hits": s.stats()["n_hits"], "note": "out/back cross-term multipath on"}
    s.set_option(SONAR_OPT_CROSS, 0)
    # water-column reverberation: 10^6 scatterers in a box over the wall and the seabed
    s.set_volume(1_000_000, VOLUME_BOX[0], VOLUME_BOX[1], VOLUME_SV)
    for _ in range(3):
        s.ping(poses[0], params, ssp, precision="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(10):
        s.ping(poses[0], params, ssp, precision="fp32")
    torch.cuda.synchronize()
    out["c2_volume1m_fp32"] = {"value": 10 / (time.perf_counter() - t0), "unit": UNIT,
                               "hits": s.stats()["n_hits"],
                               "note": "10^6 water-column scatterers (s_v 1e-4 /m) on top of the mesh"}
    s.set_volume(0)
    # rays through a range-dependent thermocline (RK4 steps of 0.5 m, chords per step)
    s.set_field(dict(THERMOCLINE, h=0.5))
    pf = dict(params, c_ref=1500.0)
    for _ in range(2):
        s.ping(poses[0], pf, ssp, precision="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        s.ping(poses[0], pf, ssp, precision="fp32")
    torch.cuda.synchronize()
    out["c2_field_h0.5_fp32"] = {"value": 5 / (time.perf_counter() - t0), "unit": UNIT,
                                 "note": "range-dependent thermocline, RK4 rays at 0.5 m steps"}
    s.set_field(None)
    # the two straight-ray traversals: per-stage events, ray casting time
    from paper_2606_06130_gb300.sonar import SONAR_OPT_TIMING, SONAR_OPT_TRAVERSAL
    trav = {}
    s.set_option(SONAR_OPT_TIMING, 1)
    for mode, name in ((0, "per_thread"), (1, "warp_cooperative")):
        s.set_option(SONAR_OPT_TRAVERSAL, mode)
        ms = []
        for i in range(13):
            s.ping(poses[0], params, ssp, precision="fp32")
            if i >= 3:
                ms.append(s.stats()["ms_trace"])
        trav[name] = {"ms_trace_median": float(np.median(ms)), "ms_trace_min": float(np.min(ms))}
    s.set_option(SONAR_OPT_TRAVERSAL, 0)
    s.set_option(SONAR_OPT_TIMING, 0)
    out["c2_traversal"] = dict(trav, note="straight-ray casting of the headline ping (524k sub-rays), stage events")
    out.update(surrogate_forms(torch, s, inputs, dev, scene, params, poses, ssp))
    sc4, p4, poses4, ssp4 = inputs.workload("c4")
    s.upload(sc4)
    for prec in ("fp32", "bf16"):
        env = torch.empty((len(poses4), p4["n_beam_el"], p4["n_beam_az"], p4["n_range"]), dtype=torch.float32, device=dev)
        s.ping_batch(poses4, p4, ssp4, precision=prec, env=env)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 3
        for _ in range(reps):
            s.ping_batch(poses4, p4, ssp4, precision=prec, env=env)
        torch.cuda.synchronize()
        st = s.stats()
        out[f"c4_batch64_{prec}"] = {"value": reps * len(poses4) / (time.perf_counter() - t0), "unit": UNIT,
                                     "hits_total": st["n_hits"], "beamform_tile_n": st["tile_n"],
                                     "synth_cols": st["synth_cols"], "autotuned": bool(st["autotuned"])}
        del env
    s.upload(scene)
    return out


def surrogate_forms(torch, s, inputs, dev, scene, params, poses, ssp, warmup=3, reps=10):
    """Throughput of the learned surrogate's training step on the headline ping (1024
    beams: rendering, forward, backward, Adam), of its inference (the rendering plus the
    six-layer network over all 8192 beams x 1024 bins), and of the geometric envelope it
    starts from. The network's weights do not change the work: the seeded initialisation
    is used."""
    out = {}
    nb = params["n_beam_az"] * params["n_beam_el"]
    s.sur_set_weights(inputs.surrogate_init(1), 0.05)
    target, _, _ = s.ping_batch(poses, params, ssp, cloud_cap=0)
    gen = torch.Generator(device=dev)
    gen.manual_seed(3)
    beams = torch.randint(0, nb, (1024,), generator=gen, device=dev, dtype=torch.int32)
    for _ in range(warmup):
        s.sur_train_step(poses, params, ssp, target, beams, lr=1e-4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(2 * reps):
        s.sur_train_step(poses, params, ssp, target, beams, lr=1e-4)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / (2 * reps)
    out["c2_surrogate_train_step"] = {"value": 1.0 / dt, "unit": "steps/s", "beams_per_step": 1024,
                                      "positions_per_s": 1024 * params["n_range"] / dt}
    env = torch.empty((1, params["n_beam_el"], params["n_beam_az"], params["n_range"]), dtype=torch.float32, device=dev)
    for name, call in (("c2_surrogate_bf16", lambda: s.sur_ping(poses, params, ssp, env=env)),
                       ("c2_geometric", lambda: s.sur_geometric(poses, params, ssp, env=env))):
        for _ in range(warmup):
            call()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            call()
        torch.cuda.synchronize()
        out[name] = {"value": reps / (time.perf_counter() - t0), "unit": UNIT}
    out["c2_surrogate_bf16"]["note"] = ("beam-centre rendering + 6-layer conv net (4 hidden layers on tcgen05), "
                                        "8192 beams x 1024 bins, BF16 weights and activations, FP32 accumulation")
    return out


def run_surrogate_forms(args):
    """--surrogate-forms: only the learned surrogate's forms on the headline ping (the
    profiling command of its kernels); --steps sets the timed repetitions."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06130_gb300 import inputs
    from paper_2606_06130_gb300.sonar import Sonar
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    scene, params, poses, ssp = inputs.workload("c2")
    s = Sonar(0)
    s.upload(scene)
    out = surrogate_forms(torch, s, inputs, dev, scene, params, poses, ssp, warmup=args.warmup, reps=args.steps)
    print(json.dumps({"surrogate_forms": out}), flush=True)


def run_ttd_form(args):
    """--ttd U: only the true-time-delay form of the headline ping (the profiling command
    of its kernels)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06130_gb300 import inputs
    from paper_2606_06130_gb300.sonar import Sonar
    torch.cuda.set_device(0)
    scene, params, poses, ssp = inputs.workload("c2")
    s = Sonar(0)
    s.upload(scene)
    out = ttd_form(torch, s, params, poses, ssp, args.ttd)
    print(json.dumps({f"c2_ttd_u{args.ttd}_fp32": out}), flush=True)


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def oracle_timing():
    """The reference arm with --oracle-timing (not part of the default runs): the FP64
    oracle as it stands on this host, whole C1 and C2 pings single-threaded and on all
    cores, and the C4 64-ping trajectory on all cores from 8 pings, extrapolated."""
    import oracle
    from paper_2606_06130_gb300 import inputs
    n_all = oracle.num_threads()
    rows = []
    for threads in (1, n_all):
        oracle.set_threads(threads)
        for name in ("c1", "c2"):
            scene, params, poses, ssp = inputs.workload(name)
            t0 = time.perf_counter()
            h, _, _ = oracle_ping(scene, params, poses[0], ssp)
            dt = time.perf_counter() - t0
            rows.append({"config": name, "threads": threads, "seconds_per_ping": dt, "pings_per_s": 1.0 / dt,
                         "hits": int(h["n"])})
    oracle.set_threads(n_all)
    scene, params, poses, ssp = inputs.workload("c4")
    t0 = time.perf_counter()
    hits = 0
    for k in range(8):
        h, _, _ = oracle_ping(scene, params, poses[k], ssp)
        hits += int(h["n"])
    dt = time.perf_counter() - t0
    rows.append({"config": "c4", "threads": n_all, "pings": 8, "seconds": dt, "pings_per_s": 8 / dt,
                 "hits": hits, "note": f"64 pings extrapolated: {64 * dt / 8:.1f} s"})
    print(json.dumps({"oracle_timing": rows, "cpu": cpu_model(), "nproc": os.cpu_count()}), flush=True)


def run_surrogate_training(args):
    """--surrogate-train N: the learned surrogate trained from its seeded initialisation on
    N pings that the plain method renders over randomised harbour scenes (one training
    step of 1024 beams per ping), then judged on 64 held-out pings (4 unseen scenes x 16
    poses, 8192 beams x 1024 bins each) against the plain method, beside the geometric
    envelope without the network. Prints one JSON line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_06130_gb300 import inputs, surrogate
    from paper_2606_06130_gb300.sonar import Sonar
    torch.cuda.set_device(0)
    s = Sonar(0)
    params, ssp = inputs.sensor_params("c2"), inputs.ssp("c2")
    t0 = time.perf_counter()
    tr = surrogate.train(s, params, ssp, n_pings=args.surrogate_train, seed=1000, batch=8, pings_per_scene=64)
    t_train = time.perf_counter() - t0
    t0 = time.perf_counter()
    ev = surrogate.evaluate(s, params, ssp, scene_seeds=[900001, 900003, 900005, 900007], pings_per_scene=16)
    L = tr["losses"]
    out = {"surrogate_training": {
        "pings": tr["pings"], "steps": tr["steps"], "beams_per_step": tr["beams_per_step"], "e_scale": tr["e_scale"],
        "loss_first_8": float(L[:8].mean()), "loss_last_1000": float(L[-1000:].mean()),
        "loss_curve": [float(L[i:i + max(1, len(L) // 20)].mean()) for i in range(0, len(L), max(1, len(L) // 20))],
        "wall_s": t_train, "plain_render_s": tr["plain_s"], "train_steps_s": tr["train_s"]},
        "held_out": {"pings": 64, "scenes": 4, "metrics_vs_plain": ev, "eval_s": time.perf_counter() - t0,
                     "rel_thr": 0.1}}
    print(json.dumps(out), flush=True)


def run_reference(args, ws, rank):
    if rank != 0:
        return
    if args.oracle_timing:
        oracle_timing()
        return
    r = time_oracle(args.steps, args.warmup, k=sample_divisor(args.steps + args.warmup))
    out = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * r["seconds"] / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "precision": "fp64 oracle"}, "impl": "reference",
           "cpu_baseline": {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                            "sample": r["sample"]},
           "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle error and CPU baseline")
    ap.add_argument("--no-forms", action="store_true", help="skip the BF16/FP16/batch side measurements")
    ap.add_argument("--cross", action="store_true",
                    help="headline workload with out/back cross-term multipath (implies --no-oracle)")
    ap.add_argument("--volume", type=int, default=0,
                    help="headline workload plus this many water-column scatterers (implies --no-oracle)")
    ap.add_argument("--field", type=float, default=0.0,
                    help="headline workload through the range-dependent thermocline, rays integrated at this "
                         "step in m (implies --no-oracle)")
    ap.add_argument("--oracle-timing", action="store_true",
                    help="with --impl reference: time the FP64 oracle in full instead (C1, C2 whole pings at 1 "
                         "and all threads; C4 8 pings)")
    ap.add_argument("--surrogate-train", type=int, default=0,
                    help="train the learned surrogate on this many plain-method pings and evaluate it on 64 "
                         "held-out pings (one JSON line; not part of the default run)")
    ap.add_argument("--surrogate-forms", action="store_true",
                    help="time only the learned surrogate's forms (training step, inference, geometric envelope)")
    ap.add_argument("--synth-cols", type=int, default=0, choices=[0, 32, 64, 96],
                    help="pin the synthesis tile (complex columns) instead of tuning it")
    ap.add_argument("--tile-n", type=int, default=0, choices=[0, 128, 192, 224, 256],
                    help="pin the beamforming N tile instead of tuning it")
    ap.add_argument("--dense", action="store_true",
                    help="form the beams with the dense contraction instead of the separable stages")
    ap.add_argument("--ttd", type=int, default=0,
                    help="time only the true-time-delay form of the headline ping at this many phases per cell")
    args = ap.parse_args()
    if args.ttd > 0:
        run_ttd_form(args)
        return
    if args.surrogate_train > 0:
        run_surrogate_training(args)
        return
    if args.surrogate_forms:
        run_surrogate_forms(args)
        return
    if args.cross or args.volume > 0 or args.field > 0:
        args.no_oracle = True  # the oracle legs sample the default workload
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
