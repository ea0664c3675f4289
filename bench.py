#!/usr/bin/env python
"""Frame-stream benchmark: rigid ZNCC motion correction fused with the segment
summaries, on a synthetic 512x512 uint16 voltage-imaging video of 10,000
frames (the paper-scale workload; content model in paper_2403_16438_gb300.synth).

One step = the whole video through vimg_process (full-window FP32 ZNCC over
+-16 px, 484 patches, resampling, L = 50 summaries), stream state reset between
steps so every step does identical work.  The video (5.2 GB) is resident in HBM
and larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl vimg|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.  Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s (×realtime) and HBM fraction, 1 GB300, ≤0.05 px shift err"
UNIT = "frames/s"
RECORD_FPS = 741.0  # Fig. 1 video: 10,000 frames recorded in 13.5 s
H = W = 512
R = 16
P = 21
L = 50
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": SM_MAX_MHZ_NOMINAL}, "fallback"


def fp32_alu_peak_tflops(sm_max_mhz):
    # 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x max SM clock
    return SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12


def unet_flops_per_patch(layers):
    """Useful FLOPs of one 64x64 patch through the U-Net (3x3 and up-convolutions
    and the output layer; the first layer's 2 input channels, not its padding)."""
    side = {0: 64, 1: 32, 2: 16, 3: 8, 4: 4}
    sides = []
    for l in range(5):
        sides += [side[l]] * 2
    for l in range(3, -1, -1):
        sides += [side[l + 1], side[l], side[l]]
    fl = 0
    for (kind, ci, co), s in zip(layers[:-1], sides):
        fl += 2 * s * s * ci * co * (9 if kind == "conv" else 4)
    return fl + 2 * 64 * 64 * layers[-1][1]


def corr_flops_per_frame():
    ny = nx = (H - 2 * R) // P
    return 2.0 * ny * nx * P * P * (2 * R + 1) ** 2


def temporal_bytes_per_frame():
    # read u16 frame, write f32 corrected frame, write S and T once per L frames
    return H * W * (2 + 4 + 8.0 / L)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                c = [x.strip() for x in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1]))
                    smax.append(float(c[2]))
                    power.append(float(c[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, c[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def kernel_traffic(kernel, source):
    """dram bytes per launch from the committed ncu summary, or None when the
    kernel's source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "kernel_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f).get(kernel)
    if not d:
        return None
    with open(os.path.join(ROOT, "paper_2403_16438_gb300", "csrc", source), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    if d.get("source_sha") != sha:
        return None
    return d


def max_over_ranks(x, ws, device):
    """Max of a host float over all ranks (the job's time is its slowest rank's);
    x itself when there is one rank."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def gpu_local_cpus(index):
    """Host CPUs local to GPU `index` (sysfs local_cpulist of its PCI device), or
    None.  Pinned host buffers first touched from those CPUs live on the GPU's
    NUMA node; from a remote node the host -> device copies run several times
    slower."""
    try:
        bus = subprocess.run(["nvidia-smi", f"--id={index}", "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=20).stdout.strip().lower()
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{int(dom, 16):04x}:{rest}/local_cpulist"
        with open(path) as f:
            return parse_cpulist(f.read()) or None
    except (OSError, ValueError, subprocess.SubprocessError):
        return None


def parse_cpulist(spec):
    """The set of CPUs of a sysfs cpulist such as '0-3,8,10-11'."""
    cpus = set()
    for part in spec.strip().split(","):
        if part:
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
    return cpus


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_fps(frames_cpu, template, budget_s=15.0, max_frames=64):
    """The FP64 oracle, as it stands, on the host cores: a bounded sample of
    the workload's frames through the whole pipeline."""
    import oracle
    import numpy as np
    o = oracle.Oracle(H, W, R=R)
    o.set_template(template.double().numpy())
    t0 = time.perf_counter()
    o.process(frames_cpu[:1].numpy(), want_summary=False)
    t1 = time.perf_counter() - t0
    n = int(max(2, min(max_frames, budget_s / max(t1, 1e-3))))
    n = min(n, frames_cpu.shape[0])
    o2 = oracle.Oracle(H, W, R=R)
    o2.set_template(template.double().numpy())
    t0 = time.perf_counter()
    o2.process(np.ascontiguousarray(frames_cpu[:n].numpy()))
    dt = time.perf_counter() - t0
    return n / dt, n, dt, oracle.num_threads()


def oracle_shift_check(frames, planted, T, gpu_shifts, n_sample=24, R_=R):
    """Shift error of the GPU against the FP64 oracle, and of both against the
    planted drift, on n_sample frames spread evenly over the video (the oracle
    recomputes them one by one)."""
    import numpy as np
    import oracle
    n = frames.shape[0]
    idx = np.unique(np.linspace(0, n - 1, min(n, n_sample)).round().astype(int))
    H_, W_ = frames.shape[1], frames.shape[2]
    o = oracle.Oracle(H_, W_, R=R_)
    o.set_template(T.cpu().double().numpy())
    sample = np.stack([frames[int(i)].cpu().numpy() for i in idx])
    r = o.process(sample, want_corrected=False, want_summary=False)
    g = gpu_shifts[torch.as_tensor(idx, device=gpu_shifts.device)].double().cpu().numpy()
    pl = planted[torch.as_tensor(idx)].double().numpy()

    def stats(e):
        e = np.abs(e).max(axis=1)
        return {"mean": float(e.mean()), "max": float(e.max())}
    off = (r["shifts"] - pl).mean(axis=0)
    return {"frames_sampled": int(len(idx)), "gpu_vs_oracle_px": stats(g - r["shifts"]),
            "oracle_vs_planted_px": stats(r["shifts"] - pl),
            "gpu_vs_planted_px": stats(g - pl),
            "oracle_offset_vs_planted_px": [float(off[0]), float(off[1])],
            "oracle_vs_planted_after_offset_px": stats(r["shifts"] - pl - off),
            "note": "the offset is the noise-induced bias of ZNCC's window-variance "
                    "normalisation on this content (the method, as the oracle computes it)"}


def cpu_oracle_threads(frames_cpu, template, budget_s=6.0):
    """The oracle on 1 host thread and on all host threads (frames/s each), on a
    bounded sample of the workload."""
    import oracle
    all_t = oracle.num_threads()
    out = {}
    for nt in (1, all_t):
        oracle.set_num_threads(nt)
        fps, nf, dt, cores = cpu_oracle_fps(frames_cpu, template, budget_s=budget_s, max_frames=64)
        out[f"{nt}_thread" + ("s" if nt > 1 else "")] = {
            "value": fps, "unit": UNIT, "cores": nt, "frames": nf, "seconds": dt}
    oracle.set_num_threads(all_t)
    return out


def workload_desc(bf16=False, learned=False):
    """The workload string of the JSON line's config (shared by both arms)."""
    return ("paper-scale synthetic video: 512x512 uint16, 10,000 frames per step, "
            + ("full-window BF16 tensor-core ZNCC" if bf16 else
               "learned proposal + +-2 px FP32 ZNCC window, full-window fallback"
               if learned else "full-window FP32 ZNCC")
            + " +-16 px (484 patches x 1089 shifts), bilinear "
            "resampling, L=50 mean and max-median summaries")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import torch
    from paper_2403_16438_gb300 import synth
    cfg = synth.paper_scale_config()
    frames, _, T = synth.make_video(cfg, 128)
    import oracle
    o = oracle.Oracle(H, W, R=R)
    o.set_template(T.double().numpy())
    t0 = time.perf_counter()
    o.process(frames[:1].numpy(), want_summary=False)
    t1 = time.perf_counter() - t0
    # each step: a bounded sample sized so warmup + steps end within ~3 minutes
    per_step = int(max(1, min(64, args.ref_budget / max(1, args.steps + args.warmup) / max(t1, 1e-3))))
    times = []
    for s in range(args.warmup + args.steps):
        o = oracle.Oracle(H, W, R=R)
        o.set_template(T.double().numpy())
        t0 = time.perf_counter()
        o.process(frames[:per_step].numpy())
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = per_step * len(times) / total
    sample = (f"{per_step} frames of the 512x512 paper-scale video per step "
              f"(full pipeline, FP64 direct sums)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(), "frames_per_step": per_step, "H": H, "W": W,
                   "search_radius": R, "segment_len": L, "parallelism": "single",
                   "sample": f"each step runs {per_step} of the workload's 10,000 frames "
                             "(a bounded CPU sample; frames/s is per frame)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_vimg(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2403_16438_gb300 import synth, vimg

    from paper_2403_16438_gb300 import shard
    n = args.frames
    cfg = synth.paper_scale_config()
    if ws > 1:
        # time shards of one (ws x n)-frame video: rank r outputs frames
        # [r n, (r + 1) n) (segment-aligned; the high-pass is off, so no history)
        plan = shard.plan(n * ws, ws, L, 0)
        mine = plan[rank]
        frames, planted, T = synth.make_video_range(cfg, n * ws, mine.hist_start, mine.end,
                                                    device=dev)
        frames = frames[mine.history:]
        planted = planted[mine.history:]
        t_start = mine.start
    else:
        plan = None
        frames, planted, T = synth.make_video(cfg, n, device=dev)
        t_start = 0
    stream = torch.cuda.current_stream(dev)
    bf16 = args.corr == "bf16"
    learned = args.corr == "proposal"
    flags = vimg.CORR_BF16 if bf16 else (vimg.PROPOSAL_CNN if learned else 0)
    h = vimg.Handle(H, W, stream=stream, max_chunk=args.bf16_chunk if bf16 else args.chunk,
                    flags=flags)
    h.set_template(T)
    if learned:
        from paper_2403_16438_gb300 import proposal
        params, _ = proposal.train(total_frames=args.train_frames)
        h.load_proposal(params)
    shifts = torch.empty((n, 2), device=dev)
    corrected = torch.empty((n, H, W), device=dev)
    k_max = n // L
    summary = torch.empty((max(1, k_max), 2, H, W), device=dev)

    def step():
        h.seek(t_start)
        k = h.process(frames, shifts=shifts, corrected=corrected, summary=summary)
        assert k == k_max

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # shift error against the planted drift (content model; parity is in the tests)
    err_planted = (shifts.double().cpu() - planted).abs()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    h.profile(True)
    h.profile_read(reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    prof = h.profile_read(reset=True)
    h.profile(False)
    ms = max_over_ranks(e0.elapsed_time(e1), ws, dev)
    total_frames = n * args.steps * ws
    value = total_frames / (ms / 1000.0)

    pk, pk_kind = peaks()
    smax = pk.get("sm_max_mhz", SM_MAX_MHZ_NOMINAL)
    corr_ms, corr_launches = prof["corr"]
    corr_flops = corr_flops_per_frame() * n * args.steps
    achieved = corr_flops / (corr_ms / 1000.0) / 1e12 if corr_ms > 0 else None
    alu_derived = fp32_alu_peak_tflops(smax)
    alu_peak = vimg.fma_rate(stream) / 1e12  # measured on this GPU, like the HBM and BF16 peaks
    if bf16:
        tpk = pk["bf16_tflops_sustained"]
        roofline = {
            "kernel": "k_corr_bf16 (+ k_fc pre-pass and k_zncc_reduce)", "bound": "tensor",
            "achieved": achieved, "peak": tpk, "unit": "TFLOP/s",
            "frac": achieved / tpk if achieved else None, "traffic": None,
            "per_launch_frames": round(n * args.steps / max(1, corr_launches), 3),
            "avg_launch_ms": corr_ms / max(1, corr_launches),
            "peak_kind": pk_kind + " (sustained cuBLAS bf16)",
            "note": "achieved counts the useful 2 x 484 x 441 x 1089 FLOP per frame",
        }
    elif learned:
        t_ms, t_launches = prof["temporal"]
        gbs = temporal_bytes_per_frame() * n * args.steps / (t_ms / 1000.0) / 1e9 if t_ms > 0 else None
        roofline = {
            "kernel": "k_temporal (the largest stage of this path)", "bound": "hbm",
            "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / pk["hbm_gbs"] if gbs else None, "traffic": None,
            "per_launch_frames": round(n * args.steps / max(1, t_launches), 3),
            "avg_launch_ms": t_ms / max(1, t_launches), "peak_kind": pk_kind,
        }
    else:
        tr = kernel_traffic("k_corr_f32", "motion.cu")
        plf = n * args.steps / max(1, corr_launches)
        # DRAM bytes grow with the frames of a launch (each frame and its isf map
        # read once): the captured launch's bytes scaled to this launch's frames
        traffic = (tr["dram_bytes_per_launch"] * plf / tr["frames_per_launch"]) if tr else None
        roofline = {
            "kernel": "k_corr_f32", "bound": "alu", "achieved": achieved,
            "peak": alu_peak, "unit": "TFLOP/s",
            "frac": achieved / alu_peak if achieved else None,
            "traffic": traffic,
            "traffic_captured_frames_per_launch": tr["frames_per_launch"] if tr else None,
            "per_launch_frames": round(plf, 3),
            "avg_launch_ms": corr_ms / max(1, corr_launches),
            "peak_kind": "measured (vimg_fma_rate: independent FFMA chains on every SM)",
            "peak_derived": alu_derived,
            "peak_derived_kind": f"{SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                 f"{smax:.0f} MHz",
        }
    temp_ms, temp_launches = prof["temporal"]
    temp_gbs = temporal_bytes_per_frame() * n * args.steps / (temp_ms / 1000.0) / 1e9 \
        if temp_ms > 0 else None
    kernel_launches = sum(prof[s][1] for s in ("stats", "corr", "peak", "temporal", "proposal"))

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if bf16 else "f32",
        "data": "synthetic",
        "config": {
            "workload": workload_desc(bf16, learned),
            "frames_per_step": n, "frames_per_launch": args.bf16_chunk if bf16 else args.chunk,
            "H": H, "W": W, "search_radius": R, "segment_len": L,
            "l2": "no flush: each step reads 5.2 GB of frames, larger than L2",
            "parallelism": f"time shards of one video over {ws} GPUs" if ws > 1 else "single",
            "x_realtime_741fps": value / RECORD_FPS / ws,
        },
        "x_realtime": value / RECORD_FPS / ws,
        "x_realtime_1000fps": value / 1000.0 / ws,
        "hbm_fraction": {"kernel": "k_temporal (fused resample+summaries)",
                         "achieved_gbs": temp_gbs, "peak_gbs": pk["hbm_gbs"],
                         "frac": temp_gbs / pk["hbm_gbs"] if temp_gbs else None,
                         "peak_kind": pk_kind},
        "roofline": roofline,
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "stage_launches_per_step": {k: v[1] / args.steps for k, v in prof.items()},
        "gpu_launches": kernel_launches,
        "clocks": clk,
        "shift_err_vs_planted_px": {"mean": float(err_planted.mean()),
                                    "p99": float(err_planted.flatten().quantile(0.99)),
                                    "max": float(err_planted.max())},
        "paper_context": {"mc_stage_fps_2080ti_450x138": 10000 / 5.5,
                          "source": "Fig. 1: MC 5.5 s for 10,000 frames on 1 RTX 2080 Ti"},
    }
    if plan is not None:
        line["config"]["shards"] = [{"rank": r, "first_frame": x.start, "frames": x.frames}
                                    for r, x in enumerate(plan)]
    if rank == 0:
        line["shift_check"] = oracle_shift_check(frames, planted, T, shifts)

    # end to end through the public API with host buffers
    if not args.no_e2e:
        ke = max(1, min(args.steps, args.e2e_steps))
        # host work of this leg on the GPU's own NUMA node (pinned buffers included)
        prev_aff = os.sched_getaffinity(0)
        local_cpus = gpu_local_cpus(local)
        if local_cpus:
            try:
                os.sched_setaffinity(0, local_cpus & set(range(os.cpu_count() or 1)) or prev_aff)
            except OSError:
                local_cpus = None
        fh = torch.empty((n, H, W), dtype=torch.uint16, pin_memory=True)
        fh.copy_(frames.cpu())
        sh_h = torch.empty((n, 2), pin_memory=True)
        sm_h = torch.empty((max(1, k_max), 2, H, W), pin_memory=True)
        h.reset()
        h.process_host(fh, shifts_host=sh_h, summary_host=sm_h, corrected=corrected)
        # the box's pinned host -> device bandwidth, which bounds the copies e2e overlaps
        torch.cuda.synchronize()
        tc0 = time.perf_counter()
        frames.copy_(fh, non_blocking=True)
        torch.cuda.synchronize()
        h2d_gbs = fh.numel() * 2 / (time.perf_counter() - tc0) / 1e9
        barrier()
        eclk = Clocks(local)
        eclk.start()
        step_ms = []
        t0 = time.perf_counter()
        for _ in range(ke):
            ts = time.perf_counter()
            h.reset()
            h.process_host(fh, shifts_host=sh_h, summary_host=sm_h, corrected=corrected)
            step_ms.append((time.perf_counter() - ts) * 1000.0)  # the call synchronises
        torch.cuda.synchronize()
        barrier()
        te = max_over_ranks(time.perf_counter() - t0, ws, dev)
        e2e_clocks = eclk.stop()
        line["e2e"] = {"value": n * ke * ws / te, "unit": UNIT,
                       "h2d_bytes_per_step": n * H * W * 2,
                       "d2h_bytes_per_step": n * 2 * 4 + k_max * 2 * H * W * 4,
                       "steps": ke, "step_ms": step_ms,
                       "step_ms_median": sorted(step_ms)[len(step_ms) // 2],
                       "clocks": e2e_clocks,
                       "h2d_GBs_measured": h2d_gbs,
                       "host_cpus": (f"{min(local_cpus)}-{max(local_cpus)} ({len(local_cpus)} "
                                     "CPUs local to the GPU)") if local_cpus else "not pinned",
                       "note": "vimg_process_host: pinned host frames in, shifts and summaries "
                               "out; corrected frames stay in device memory"}
        del fh, sh_h, sm_h
        os.sched_setaffinity(0, prev_aff)
    if not args.no_variants:
        line["variants"] = run_variants(args, frames, planted, T, shifts, corrected, summary, stream,
                                        dev, k_max, ws)
    if not args.no_batched:
        line.setdefault("variants", {})["batched_6_videos"] = run_batched(args, stream, dev, ws)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        fps, nf, dt, cores = cpu_oracle_fps(frames[:512].cpu(), T.cpu(), budget_s=args.cpu_budget,
                                            max_frames=512)
        line["cpu_baseline"] = {"value": fps, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{nf} frames of the same video, full pipeline, "
                                          f"{dt:.1f} s wall"}
        line["cpu_baseline"]["threads"] = cpu_oracle_threads(frames[:64].cpu(), T.cpu(),
                                                             budget_s=args.cpu_budget / 2)
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def time_variant(h, frames, outs, steps, warmup, stream, traces=None):
    shifts, corrected, summary = outs

    def step():
        h.reset()
        h.process(frames, shifts=shifts, corrected=corrected, summary=summary, traces=traces)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    h.profile(True)
    h.profile_read(reset=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    prof = h.profile_read(reset=True)
    h.profile(False)
    return e0.elapsed_time(e1), prof


def run_config_variant(cfg, args, stream, dev, ws, chunk=200, check=True):
    """The full-window FP32 path on another synthetic video: frames/s, realtime
    multiples, the temporal pass's HBM fraction, and the shift error against
    the oracle and the planted drift on sampled frames."""
    from paper_2403_16438_gb300 import synth, vimg
    n_ = cfg.n_frames
    frames, planted, Tv = synth.make_video(cfg, n_, device=dev)
    h = vimg.Handle(cfg.H, cfg.W, stream=stream, max_chunk=chunk)
    h.set_template(Tv)
    sh = torch.empty((n_, 2), device=dev)
    co = torch.empty((n_, cfg.H, cfg.W), device=dev)
    sm = torch.empty((max(1, n_ // L), 2, cfg.H, cfg.W), device=dev)
    ms, prof = time_variant(h, frames, (sh, co, sm), args.steps, args.warmup, stream)
    h.close()
    value = n_ * args.steps * ws / (ms / 1000.0)
    t_ms = prof["temporal"][0]
    pk, pk_kind = peaks()
    gbs = cfg.H * cfg.W * (2 + 4 + 8.0 / L) * n_ * args.steps / (t_ms / 1000.0) / 1e9
    out = {
        "value": value, "unit": UNIT, "ms_per_step": ms / args.steps,
        "x_realtime_741fps": value / RECORD_FPS / ws, "x_realtime_1000fps": value / 1000.0 / ws,
        "hbm_fraction": {"kernel": "temporal pass", "achieved_gbs": gbs, "peak_gbs": pk["hbm_gbs"],
                         "frac": gbs / pk["hbm_gbs"], "peak_kind": pk_kind},
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": sum(prof[s_][1] for s_ in ("stats", "corr", "peak", "temporal")) / args.steps,
        "config": {"H": cfg.H, "W": cfg.W, "frames_per_step": n_, "search_radius": R,
                   "segment_len": L, "neurons": cfg.n_neurons, "read_sigma": cfg.read_sigma,
                   "walk_sigma_px": cfg.walk_sigma, "clamp_px": cfg.clamp,
                   "jump_frac": cfg.jump_frac},
    }
    if check:
        out["shift_check"] = oracle_shift_check(frames, planted, Tv, sh)
    del frames, co
    return out


def run_variants(args, frames, planted, T, ref_shifts, corrected, summary, stream, dev, k_max, ws):
    """Other configurations on the same video: voltage traces of the neuron
    ROIs, the spiking-pixel U-Net on the summary pairs, the BF16 tensor-core
    correlation and the learned shift proposal (CNN + +-2 px window +
    full-window fallback), the last two compared with the full-window shifts."""
    from paper_2403_16438_gb300 import proposal, synth, vimg
    n = frames.shape[0]
    out = {}
    ref = ref_shifts.clone()
    checks = dist_env()[1] == 0  # the oracle's sampled checks run on rank 0 only
    # the tiny configuration (128x128, 1,000 frames) and the paper's own frame
    # shape (138 x 450, the Fig. 1 video) with paper-scale content
    out["config1_tiny_128x128"] = run_config_variant(synth.tiny_config(), args, stream, dev, ws,
                                                     check=checks)
    v2p = run_config_variant(synth.scaled_config(138, 450, 10000, seed=1012), args, stream, dev, ws,
                             check=checks)
    v2p["paper_context"] = {
        "mc_stage_seconds_2080ti": 5.5, "mc_stage_fps_2080ti": 10000 / 5.5,
        "video": "HPC2 mouse hippocampus, 450 x 138 px, 10,000 frames at 741 fps",
        "hardware": "1 of 2 NVIDIA RTX 2080 Ti, CUDA 12.0; AMD Threadripper 3960X",
        "source": "Fig. 1 and Table I of the paper (another GPU, another video: context only)"}
    out["config2p_paper_shape_138x450"] = v2p
    # voltage traces of the scene's neuron ROIs, fused into the temporal pass
    masks = synth.roi_masks(synth.paper_scale_config(seed=1002 + dist_env()[1])).to(dev)
    h = vimg.Handle(H, W, stream=stream, max_chunk=args.chunk, flags=vimg.VIDEO_SUMMARY)
    h.set_template(T)
    h.set_rois(masks)
    tr = torch.empty((n, masks.shape[0]), device=dev)
    sh = torch.empty_like(ref)
    ms, prof = time_variant(h, frames, (sh, corrected, summary), args.steps, args.warmup, stream,
                            traces=tr)
    avg_img = torch.empty((H, W), device=dev)
    corr_img = torch.empty((H, W), device=dev)
    h.video_summary(avg_img, corr_img)
    torch.cuda.synchronize()
    h.close()
    roi_any = masks.any(dim=0)
    out["voltage_traces"] = {
        "value": n * args.steps * ws / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms / args.steps,
        "n_rois": int(masks.shape[0]), "roi_pixels": int(masks.sum().item()),
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "correlation_image_mean_in_rois": float(corr_img[roi_any].mean()),
        "correlation_image_mean_outside": float(corr_img[~roi_any].mean()),
        "config": "full-window FP32 path, corrected frames and summaries as the main line, plus "
                  "the mean corrected intensity of every neuron footprint of the scene per frame "
                  "(traces) and the whole-video average and local correlation images "
                  "(stage 'downstream' holds both)",
    }
    # spiking-pixel U-Net on every segment's summary pair (Sec. III-C), random
    # weights of the architecture: alone on the 200 summary pairs, and attached
    # to the pipeline (corrected frames, summaries and probability maps)
    layers = vimg.unet_layers()
    up = synth.unet_params(layers, seed=7).to(dev)
    un = vimg.Unet(H, W, max_segments=8, stream=stream)
    un.load(up)
    prob = torch.empty((k_max, H, W), device=dev)
    for _ in range(args.warmup):
        un.run(summary, prob)
    un.synchronize()
    un.profile(True)
    un.profile_read(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        un.run(summary, prob)
    e1.record(stream)
    torch.cuda.synchronize()
    conv_ms, run_ms, conv_launches = un.profile_read(reset=True)
    un.profile(False)
    ms_alone = e0.elapsed_time(e1)
    n_patch = k_max * ((H - 64 + 31) // 32 + 1) * ((W - 64 + 31) // 32 + 1)
    fl = unet_flops_per_patch(layers) * n_patch * args.steps
    pk, _ = peaks()
    tflops = fl / (conv_ms / 1e3) / 1e12 if conv_ms > 0 else None
    h = vimg.Handle(H, W, stream=stream, max_chunk=args.chunk)
    h.set_template(T)
    h.attach_unet(un)

    def pipe_step():
        h.reset()
        h.process(frames, shifts=torch.empty_like(ref), corrected=corrected, summary=summary,
                  prob=prob)
    for _ in range(args.warmup):
        pipe_step()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        pipe_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_pipe = e0.elapsed_time(e1)
    h.close()
    un.close()
    out["unet_segmentation"] = {
        "value": n * args.steps * ws / (ms_pipe / 1000.0), "unit": UNIT,
        "x_realtime": n * args.steps / (ms_pipe / 1000.0) / RECORD_FPS,
        "ms_per_step": ms_pipe / args.steps,
        "unet_alone_ms_per_step": ms_alone / args.steps,
        "unet_segments_per_s": k_max * args.steps / (ms_alone / 1000.0),
        "unet_patches_per_step": n_patch,
        "conv_roofline": {"kernel": "k_conv_tc (22 tensor-core layers)", "bound": "tensor",
                          "achieved": tflops, "peak": pk["bf16_tflops_sustained"],
                          "unit": "TFLOP/s",
                          "frac": tflops / pk["bf16_tflops_sustained"] if tflops else None,
                          "useful_gflop_per_patch": unet_flops_per_patch(layers) / 1e9,
                          "conv_ms_per_step": conv_ms / args.steps,
                          "conv_launches_per_step": conv_launches / args.steps},
        "config": "summary pairs of the same 10,000-frame video (200 segments), 64x64 patches "
                  "every 32 px (225 per segment), 8 segments per internal pass; random weights "
                  "of the U-Net reading (16..256 channels, 4 pooling steps)",
    }
    # footprint reconstruction (Sec. III-D) on planted probability maps of the
    # scene (the random-weight U-Net's maps carry no neurons): 200 segments
    pm = synth.planted_prob_maps(synth.paper_scale_config(seed=1002 + dist_env()[1]), k_max,
                                 seed=3).to(dev)
    sg = vimg.Segmenter(H, W, k_max, stream=stream)
    for _ in range(args.warmup):
        sg.run(pm, max_neurons=512)
    t0 = time.time()
    reps = max(1, args.steps)
    for _ in range(reps):
        foot, actv, _, nreg = sg.run(pm, max_neurons=512)
    t_seg = (time.time() - t0) / reps
    sg.close()
    out["footprints"] = {
        "seconds_per_video": t_seg, "segments": k_max, "regions": nreg,
        "neurons": int(foot.shape[0]), "scene_neurons": int(masks.shape[0]),
        "config": "planted probability maps (scene footprints at 0.6-0.95 when a neuron spikes "
                  "in the segment, p = 0.4; vessels and specks to be removed; background "
                  "< 0.35); host-timed, synchronous call",
    }
    # BF16 tensor-core correlation (tcgen05), FP32 accumulation
    h = vimg.Handle(H, W, stream=stream, max_chunk=args.bf16_chunk, flags=vimg.CORR_BF16)
    h.set_template(T)
    sh = torch.empty_like(ref)
    ms, prof = time_variant(h, frames, (sh, corrected, summary), args.steps, args.warmup, stream)
    h.synchronize()
    h.close()
    d = (sh - ref).abs().max(dim=1).values.double().cpu()
    bf16_check = oracle_shift_check(frames, planted, T, sh) if checks else None
    value = n * args.steps * ws / (ms / 1000.0)
    corr_ms = prof["corr"][0]
    pk, _ = peaks()
    tflops = corr_flops_per_frame() * n * args.steps / (corr_ms / 1000.0) / 1e12
    out["bf16_tensor_core"] = {
        "value": value, "unit": UNIT, "x_realtime": value / RECORD_FPS / ws,
        "ms_per_step": ms / args.steps,
        "shift_err_vs_fp32_full_window_px": {"max": float(d.max()), "p99": float(d.quantile(0.99)),
                                             "frac_le_0.05": float((d <= 0.05).double().mean())},
        "corr_roofline": {"kernel": "k_corr_bf16 (+ frame offset pre-pass)", "bound": "tensor",
                          "achieved_useful_tflops": tflops,
                          "peak_tflops": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                          "frac_useful": tflops / pk["bf16_tflops_sustained"],
                          "note": "useful = 2 x 484 x 441 x 1089 FLOP per frame; the implicit GEMM "
                                  "executes 4x that (padding of dy, dx and the x-Toeplitz)"},
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": sum(prof[s][1] for s in ("stats", "corr", "peak", "temporal", "proposal")),
        "shift_check": bf16_check,
    }
    # learned proposal: trained here, on the GPU, by the library's own kernels
    t0 = time.time()
    params, hist = proposal.train(log_every=500)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    h = vimg.Handle(H, W, stream=stream, max_chunk=args.chunk, flags=vimg.PROPOSAL_CNN)
    h.set_template(T)
    h.load_proposal(params)
    sh = torch.empty_like(ref)
    ms, prof = time_variant(h, frames, (sh, corrected, summary), args.steps, args.warmup, stream)
    fr, fb = h.proposal_stats()
    h.close()
    d = (sh - ref).abs().max(dim=1).values.double().cpu()
    learned_check = oracle_shift_check(frames, planted, T, sh) if checks else None
    value = n * args.steps * ws / (ms / 1000.0)
    out["learned_proposal"] = {
        "value": value, "unit": UNIT, "x_realtime": value / RECORD_FPS / ws,
        "ms_per_step": ms / args.steps,
        "fallback_rate": fb / max(1, fr),
        "shift_err_vs_full_window_px": {"max": float(d.max()), "p99": float(d.quantile(0.99)),
                                        "frac_le_0.05": float((d <= 0.05).double().mean())},
        "train_s": t_train, "train_frames": 200000, "final_train_loss": hist[-1][1],
        "stages_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "gpu_launches": sum(prof[s][1] for s in ("stats", "corr", "peak", "temporal", "proposal")),
        "config": "same video; 6-layer CNN on 128x128 centre crops, correlation on +-2 px "
                  "(+1 ring) around the proposal, full +-16 px search when C(d*) < 0.5 or the "
                  "peak is on the window border",
        "shift_check": learned_check,
    }
    return out



# Six concurrent videos of uneven size (H, W, frames): 44.6 GB of uint16 frames.
SERVE_CHUNK = 64  # frames per video per step in the serving-granularity comparison
BATCH_VIDEOS = [(256, 256, 20000), (384, 512, 15000), (512, 512, 12000), (512, 1024, 10000),
                (768, 768, 7500), (1024, 1024, 5000)]


def run_batched(args, stream, dev, ws):
    """Serving-shaped load: the six videos processed together by
    vimg_process_batch (one launch per kernel for all videos of a step, CUDA
    graph replay, step shape picked by the autotuner on a 500-frame probe),
    against the plain per-video path on the same videos."""
    from paper_2403_16438_gb300 import autotune, synth, vimg
    t0 = time.time()
    vids = []
    for i, (H_, W_, n_) in enumerate(BATCH_VIDEOS):
        n_ = max(L, int(n_ * args.batch_scale))
        cfg = synth.scaled_config(H_, W_, n_, seed=5000 + i)
        f, _, T = synth.make_video(cfg, n_, device=dev)
        vids.append((f, T))
    torch.cuda.synchronize()
    t_gen = time.time() - t0
    frames = [f for f, _ in vids]
    total = sum(f.shape[0] for f in frames)
    px = sum(f.numel() for f in frames)
    maxc = 512
    # tile shape: the correlation's patch group per video, timed on a probe
    groups, group_table = autotune.tune_groups(frames, [T for _, T in vids], probe_frames=200,
                                               stream=stream)
    hs = [vimg.Handle(f.shape[1], f.shape[2], stream=stream, max_chunk=maxc, corr_group=g)
          for f, g in zip(frames, groups)]
    for h, (_, T) in zip(hs, vids):
        h.set_template(T)
    shifts = [torch.empty((f.shape[0], 2), device=dev) for f in frames]
    rings = [torch.empty((2 * maxc, f.shape[1], f.shape[2]), device=dev) for f in frames]
    summ = [torch.empty((max(1, f.shape[0] // L), 2, f.shape[1], f.shape[2]), device=dev)
            for f in frames]
    probe = 500
    choice, table = autotune.tune_batch(
        hs, frames, probe_frames=probe,
        outputs=dict(shifts=[x[:probe] for x in shifts], corrected=rings,
                     summary=[m[:probe // L] for m in summ]))
    chunk, graph = choice

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def batched():
        for h in hs:
            h.reset()
        vimg.process_batch(hs, frames, shifts=shifts, corrected=rings, summary=summ, chunk=chunk,
                           ring_chunks=2, use_graph=graph)

    steps = max(1, args.batch_steps)
    ms_b = timed(batched, steps, 1)
    ref_shifts = [x.clone() for x in shifts]
    for h in hs:
        h.close()
    # the plain per-video path: each video on its own, 500-frame calls, same rings;
    # with the default patch group (the path as a user runs it) and with the
    # batched form's groups (the same arithmetic: shifts identical)
    def sequential_run(group_of):
        plain = [vimg.Handle(f.shape[1], f.shape[2], stream=stream, max_chunk=args.chunk,
                             corr_group=group_of(i)) for i, f in enumerate(frames)]
        for h, (_, T) in zip(plain, vids):
            h.set_template(T)

        def sequential():
            for h, f, sh, r, m in zip(plain, frames, shifts, rings, summ):
                h.reset()
                k = 0
                for i, t in enumerate(range(0, f.shape[0], 500)):
                    c = f[t:t + 500]
                    k += h.process(c, shifts=sh[t:t + 500], corrected=r[(i % 2) * 500:],
                                   summary=m[k:])

        ms = timed(sequential, steps, 1)
        for h in plain:
            h.close()
        return ms

    ms_pt = sequential_run(lambda i: groups[i])
    same = all(torch.equal(a, b) for a, b in zip(ref_shifts, shifts))
    ms_p = sequential_run(lambda i: 0)

    # serving granularity: every video advances by SERVE_CHUNK frames per step
    # (the smallest streaming chunk of the load); batched = one call per step
    # for all videos, plain = one call per video per step, round robin
    serve = SERVE_CHUNK
    hs = [vimg.Handle(f.shape[1], f.shape[2], stream=stream, max_chunk=maxc, corr_group=g)
          for f, g in zip(frames, groups)]
    for h, (_, T) in zip(hs, vids):
        h.set_template(T)
    n_min = min(f.shape[0] for f in frames)
    n_serve = (n_min // serve) * serve  # frames per video in the serving comparison
    s_rings = [torch.empty((2 * serve, f.shape[1], f.shape[2]), device=dev) for f in frames]

    def serving_batched():
        for h in hs:
            h.reset()
        ks = [0] * len(hs)
        for t in range(0, n_serve, serve):
            segs = vimg.process_batch(hs, [f[t:t + serve] for f in frames],
                                      shifts=[sh[t:t + serve] for sh in shifts],
                                      corrected=s_rings,
                                      summary=[m[k:] for m, k in zip(summ, ks)], chunk=serve)
            ks = [k + g for k, g in zip(ks, segs)]

    def serving_plain():
        for h in hs:
            h.reset()
        ks = [0] * len(hs)
        for t in range(0, n_serve, serve):
            for v, (h, f) in enumerate(zip(hs, frames)):
                ks[v] += h.process(f[t:t + serve], shifts=shifts[v][t:t + serve],
                                   corrected=s_rings[v], summary=summ[v][ks[v]:])

    ms_sb = timed(serving_batched, 1, 1)
    sb_shifts = [sh[:n_serve].clone() for sh in shifts]
    ms_sp = timed(serving_plain, 1, 1)
    s_same = all(torch.equal(a, b[:n_serve]) for a, b in zip(sb_shifts, shifts))
    for h in hs:
        h.close()
    serving = {"frames_per_video_per_step": serve, "frames": n_serve * len(frames),
               "batched_value": n_serve * len(frames) / (ms_sb / 1000.0),
               "plain_per_video_value": n_serve * len(frames) / (ms_sp / 1000.0),
               "speedup_vs_plain": ms_sp / ms_sb, "shifts_identical": s_same,
               "note": "the first n frames of every video (n = the shortest video's length, "
                       "whole chunks), same handles and groups, direct launches for both (each "
                       "step's call differs, so there is no graph to replay)"}
    value = total / (ms_b / 1000.0)
    del vids, frames, rings, summ
    torch.cuda.empty_cache()
    return {
        "value": value, "unit": UNIT, "ms_per_step": ms_b,
        "x_realtime": value / RECORD_FPS,
        "x_realtime_note": "video-seconds processed per second: sum of frames / 741 fps / time",
        "megapixels_per_s": px / (ms_b / 1000.0) / 1e6,
        "plain_per_video_value": total / (ms_p / 1000.0),
        "plain_per_video_ms_per_step": ms_p,
        "speedup_vs_plain": ms_p / ms_b,
        "plain_same_groups_value": total / (ms_pt / 1000.0),
        "speedup_vs_plain_same_groups": ms_pt / ms_b,
        "shifts_identical_to_plain_same_groups": same,
        "serving": serving,
        "autotune": {"choice": {"chunk": chunk, "use_graph": graph, "corr_group": groups},
                     "corr_group_seconds_on_200_frames": {
                         f"{BATCH_VIDEOS[i][0]}x{BATCH_VIDEOS[i][1]}": {str(g): t for g, t in tg.items()}
                         for i, tg in group_table.items()},
                     "probe_frames_per_video": probe,
                     "seconds": {f"{c}/{'graph' if g else 'direct'}": t
                                 for (c, g), t in table.items()}},
        "config": {"videos": [{"H": H_, "W": W_, "frames": int(f_)}
                              for (H_, W_, _), f_ in zip(BATCH_VIDEOS,
                                                         [max(L, int(n * args.batch_scale))
                                                          for _, _, n in BATCH_VIDEOS])],
                   "frames_per_step": total, "gb_uint16": round(px * 2 / 1e9, 2),
                   "outputs": "shifts, summaries, corrected frames into 2-slot rings",
                   "generate_s": t_gen},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["vimg", "reference"], default="vimg")
    ap.add_argument("--frames", type=int, default=10000)
    ap.add_argument("--chunk", type=int, default=1000,
                    help="frames per internal batch (one launch per stage)")
    ap.add_argument("--e2e-steps", type=int, default=10,
                    help="timed end-to-end steps (at most --steps); ~0.13 s each at the default size")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="seconds of host work for the reference arm's warm-up and timed steps")
    ap.add_argument("--bf16-chunk", type=int, default=1000,
                    help="frames per internal batch of the tensor-core path (eight 128-frame groups, so the (group, patch) work units leave a small last wave)")
    ap.add_argument("--corr", choices=["f32", "bf16", "proposal"], default="f32",
                    help="correlation path of the main line (f32 = the full-window FP32 method)")
    ap.add_argument("--train-frames", type=int, default=200000,
                    help="training pool of the learned proposal (--corr proposal)")
    ap.add_argument("--batch-scale", type=float, default=1.0)
    ap.add_argument("--batch-steps", type=int, default=2)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_vimg(args)


if __name__ == "__main__":
    main()
