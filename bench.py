#!/usr/bin/env python
"""Power-Doppler frames/s of the localized EVD clutter filter on B300.

Workload: 256 x 128 px, Nt = 100 complex64 packets, 8 x 8 Gaussian windows
(64 subsets, 3-sigma supports), adaptive curvature threshold (method 1),
alpha by Eq. 13.  One step = one packet -> one PD image.  Inputs are a ring of
8 distinct seeded synthetic packets (210 MB, larger than the 126 MB L2),
resident in HBM before the timed region.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (the reference arm of this build).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NZ, NX, NT, WZ, WX = 256, 128, 100, 8, 8
RING = 8
METRIC = "power-Doppler frames/s (256x128 px, Nt=100, 8x8 subsets) vs plain FP32 path"
WORKLOAD = "256x128 px x Nt=100 complex64 packets, 8x8 Gaussian windows (3-sigma support), adaptive curvature threshold"
SUM_P = 778752          # pixels summed over the 64 window supports
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of
# the stage's kernels on this workload, valid only while their sources hash as they did then
CAPTURED_TRAFFIC = {
    # the one-sided EVD stage: evd_prep_kernel 10.42 MB + evd_os_kernel 3.96 MB
    ("evd", "os"): {"bytes": 14.38e6, "profile": "profiles/evd_os_kernel_256x128x100_8x8.md",
                    "sources": {"paper_2405_11105_b300/csrc/k_evd_os.cu":
                                "8d62c741b5101e16eb4d05782250bfe92fdd39a8416b05f0a10e69fda5e06f33",
                                "paper_2405_11105_b300/csrc/k_evd_dist.cu":
                                "8c289eda9c7e7231dae1028e56bbd723621b784f046164a1530f2268e80bf034",
                                "paper_2405_11105_b300/csrc/evd_common.cuh":
                                "0f0ae737dea39388208244c9264a3fb8da86ac8d54d0816e2b38660ff92a5563",
                                "paper_2405_11105_b300/csrc/lcf_internal.cuh":
                                "1e0aa59856ef34cb4cfdb48503a50b03a87dd782a8fce27ded9e732ed9cdd007"}},
    ("evd", "pair"): {"bytes": 10.55e6, "profile": "profiles/evd_pair_kernel_256x128x100_8x8.md",
                      "sources": {"paper_2405_11105_b300/csrc/k_evd_pair.cu":
                                  "1009f85991485b46621e713d25b5986447e5b8d30cb1cd7cbbef818ea32fe087",
                                  "paper_2405_11105_b300/csrc/evd_common.cuh":
                                  "5f49c4e22ff1c65643b5fa3ad4b49488b54f5289a099077851b31487f275d22d"}},
}


def captured_traffic(stage, evd="os"):
    """Bytes per launch from the capture, or None once a source of the stage's kernels has changed."""
    import hashlib
    rec = CAPTURED_TRAFFIC.get((stage, evd))
    if not rec:
        return None
    for rel, digest in rec["sources"].items():
        try:
            with open(os.path.join(ROOT, rel), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None
        except OSError:
            return None
    return rec["bytes"]


def max_over_ranks(x, dist=None, device="cpu"):
    """The slowest rank's time, on every rank (replicas: the job takes as long as its slowest GPU).
    `dist` is torch.distributed once a process group is up, else None (one rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput: every rank processed units_per_rank units in (at most) `seconds`."""
    return world * units_per_rank / seconds


def ring_seed(rank):
    """Seed of a rank's packet ring: each replica filters its own packets."""
    return 1000 * rank


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def algorithmic_work(nt=NT, nd=WZ * WX, sum_p=SUM_P):
    """Per-launch algorithmic FLOPs of each stage (8 real flops per complex MAC)."""
    return {
        "gram": 0.5 * 8.0 * sum_p * nt * nt,          # Hermitian upper triangle of each R_k
        "project": 8.0 * sum_p * nt * nt,             # C_w V for every window (one GEMM)
        "evd": nd * 240.0 * nt ** 3,                  # cyclic Jacobi with vectors, ~240 Nt^3 real flops per window
        "prep": None, "assemble": None,
    }


def stage_bytes(nt=NT, npix=NZ * NX, nd=WZ * WX):
    return {"prep": npix * nt * 8 * 2 + npix * (nt + 1) * 8, "assemble": None}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = max(mx, float(f[2]))
                except ValueError:
                    continue
                names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        except Exception:
            pass
        finally:
            try:
                os.remove(self.path)
            except Exception:
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_ring(seed0=0):
    import numpy as np
    from synth import REALTIME_256x128x100, generate_packet
    return np.stack([generate_packet(REALTIME_256x128x100, seed=seed0 + i) for i in range(RING)])


def cpu_oracle_rate(ring, n_packets, nthreads, thresh="curvature"):
    """Oracle packets/s on the host (FP64, OpenMP over windows)."""
    import oracle as O
    rule = {"curvature": dict(thresh_mode=O.T_CURVATURE, beta=1.0), "ncc": dict(thresh_mode=O.T_NCC),
            "median": dict(thresh_mode=O.T_MEDIAN, beta=1.43), "fixed": dict(thresh_mode=O.T_FIXED, k_fixed=8)}[thresh]
    cfg = O.OracleConfig(NZ, NX, NT, WZ, WX, **rule)
    t0 = time.perf_counter()
    for i in range(n_packets):
        O.filter(ring[i % len(ring)], cfg, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return n_packets / dt, dt


def reference_arm(args):
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    nthreads = os.cpu_count() or 1
    ring = make_ring(0)
    cpu_oracle_rate(ring, max(0, args.warmup and 1), nthreads)   # page in, one warm-up packet
    rate, dt = cpu_oracle_rate(ring, args.steps, nthreads)
    line = {"metric": METRIC, "value": rate, "unit": "frames/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "nz": NZ, "nx": NX, "nt": NT, "windows": [WZ, WX]},
            "cpu_baseline": {"value": rate, "unit": "frames/s", "cores": nthreads, "kind": "oracle",
                             "sample": f"{args.steps} full packets of the workload"},
            "e2e": {"value": rate, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


LEARNED_WEIGHTS = os.path.join(ROOT, "paper_2405_11105_b300", "weights", "learned_384x256x128_16x16.npy")


def learned_workload(args):
    """384x256 px, Nt=128, 16x16 windows: the learned cutoff on a 2-sweep EVD against method 1 on
    the converged EVD (its fallback and its reference), same kernels otherwise."""
    import numpy as np
    import torch
    import paper_2405_11105_b300 as L
    from synth import LEARNED_384x256x128, generate_packet
    nz, nx, nt, wz, wx = 384, 256, 128, 16, 16
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    ring = np.stack([generate_packet(LEARNED_384x256x128, seed=50000 + i) for i in range(4)])   # 403 MB > L2
    d_ring = torch.from_numpy(ring).to(f"cuda:{local}")
    out = torch.empty((nz, nx), dtype=torch.float32, device=f"cuda:{local}")
    common = dict(device=local, gram_path=L.LCF_PATH_TC, project_path=L.LCF_PATH_TC, evd_path=L.LCF_EVD_PAIR)
    conv = L.Plan.make(nz, nx, nt, wz, wx, thresh_mode=L.LCF_T_CURVATURE, beta=1.0, **common)
    meta = json.load(open(os.path.splitext(LEARNED_WEIGHTS)[0] + ".json"))
    fast = L.Plan.make(nz, nx, nt, wz, wx, thresh_mode=L.LCF_T_LEARNED, k_src=L.LCF_T_CURVATURE, beta_src=1.0,
                       max_sweeps=meta["fast_sweeps"], **common)
    net = L.Mlp(nt, hidden=meta["hidden"], max_batch=1, device=local)
    net.set_params(np.load(LEARNED_WEIGHTS))
    fast.set_mlp(net, p_min=0.5)
    st = torch.cuda.current_stream()

    def timed(plan):
        for i in range(args.warmup):
            plan.filter(d_ring[i % 4], out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for i in range(args.steps):
            plan.filter(d_ring[i % 4], out)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    # the same capped plan with the network switched off: every window takes method 1 on the
    # capped spectrum (p_min above 1)
    off = L.Plan.make(nz, nx, nt, wz, wx, thresh_mode=L.LCF_T_LEARNED, k_src=L.LCF_T_CURVATURE, beta_src=1.0,
                      max_sweeps=meta["fast_sweeps"], **common)
    off.set_mlp(net, p_min=1.01)
    with ClockSampler(local) as clk:
        ms_fast = timed(fast)
    ms_conv = timed(conv)
    ms_off = timed(off)

    def judge(plan):
        db, agree, fb = [], [], 0
        for i in range(4):
            a = conv.filter(d_ring[i]).cpu().numpy().astype(np.float64)
            b = plan.filter(d_ring[i]).cpu().numpy().astype(np.float64)
            m = a >= a.max() * 1e-3
            db.append(float(np.mean(np.abs(10 * np.log10(b[m] / a[m])))))
            agree.append(float(np.mean(conv.debug()["k"] == plan.debug()["k"])))
            fb += int(np.sum(np.asarray(plan.status()[1]) & L.LCF_WFLAG_FALLBACK != 0))
        return db, agree, fb
    db, agree, fb = judge(fast)
    db_off, agree_off, _ = judge(off)
    fast.profile(True)
    timed(fast)
    stages, n = fast.profile_read()
    fast.profile(False)
    line = {"metric": "power-Doppler frames/s (384x256 px, Nt=128, 16x16 subsets), learned cutoff vs method 1",
            "value": args.steps / (ms_fast / 1e3), "unit": "frames/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_fast / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (MLP: bf16 weights, f32 accumulate)",
            "data": "synthetic", "impl": "ours",
            "config": {"workload": "384x256 px x Nt=128, 16x16 windows, learned cutoff on a "
                                   f"{meta['fast_sweeps']}-sweep EVD", "l2": "ring of 4 packets (403 MB) > L2"},
            "method1_converged": {"value": args.steps / (ms_conv / 1e3), "unit": "frames/s",
                                  "ms_per_step": ms_conv / args.steps},
            "speedup_vs_method1": ms_conv / ms_fast,
            "pd_db_error": {"mean_abs_db": float(np.mean(db)), "max_packet_mean_abs_db": float(np.max(db)),
                            "pixels": "PD >= 1e-3 x max of the method-1 image"},
            "cutoff_agreement": float(np.mean(agree)), "fallback_windows": fb, "windows": 4 * wz * wx,
            "network_off": {"value": args.steps / (ms_off / 1e3), "unit": "frames/s",
                            "mean_abs_db": float(np.mean(db_off)), "max_packet_mean_abs_db": float(np.max(db_off)),
                            "cutoff_agreement": float(np.mean(agree_off)),
                            "note": "same capped plan, every window method 1 on the capped spectrum"},
            "stage_ms_per_launch": {k: v / max(n, 1) for k, v in stages.items()},
            "training": meta, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def stream_workload(args):
    """512x256 px, Nt=200, 16x16 windows, method 6 (soft weights), packets every 50 frames of one frame
    ring: the whole stream is one CUDA graph launch; per-packet latency from packets launched alone."""
    import numpy as np
    import torch
    import paper_2405_11105_b300 as L
    from synth import STREAM_512x256x200, generate_frames
    nz, nx, nt, wz, wx, stride, npk = 512, 256, 200, 16, 16, 50, args.stream_packets
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    n_frames = (npk - 1) * stride + nt
    t0 = time.perf_counter()
    frames = generate_frames(STREAM_512x256x200, n_frames, seed=7)
    gen_s = time.perf_counter() - t0
    d = torch.from_numpy(frames).to(f"cuda:{local}")
    del frames
    out = torch.empty((npk, nz, nx), dtype=torch.float32, device=f"cuda:{local}")
    plan = L.Plan.make(nz, nx, nt, wz, wx, device=local, thresh_mode=L.LCF_T_ADAPTIVE_SOFT, beta=1.0,
                       gram_path=L.LCF_PATH_TC, project_path=L.LCF_PATH_TC,
                       evd_path=L.LCF_EVD_OS if args.evd == "os" else L.LCF_EVD_PAIR)
    st = torch.cuda.current_stream()
    plan.filter_stream(d, stride, out)          # captures the stream graph
    torch.cuda.synchronize()
    n0 = plan.launch_count()
    reps = max(1, args.steps // npk)
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            plan.filter_stream(d, stride, out)
        e1.record(st)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = plan.launch_count() - n0
    lat = []
    one = torch.empty((nz, nx), dtype=torch.float32, device=f"cuda:{local}")
    for i in range(npk):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        plan.filter(d[i * stride:i * stride + nt], one)
        b.record(st)
        b.synchronize()
        lat.append(a.elapsed_time(b))
    plan.profile(True)   # four packets of the stream, launched one by one
    plan.filter_stream(d[:nt + 3 * stride], stride)
    stages, n = plan.profile_read()
    plan.profile(False)
    stc, flags = plan.status()
    line = {"metric": "power-Doppler frames/s (512x256 px, Nt=200, 16x16 subsets, sliding packets)",
            "value": reps * npk / (ms / 1e3), "unit": "frames/s", "n_gpus": 1, "steps": reps * npk, "warmup": npk,
            "ms_per_step": ms / (reps * npk), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "impl": "ours",
            "config": {"workload": f"{npk} packets of 512x256 px x Nt=200 sliding by {stride} frames over one "
                                   f"frame ring ({n_frames} frames, {d.numel() * 8 / 1e9:.2f} GB), 16x16 windows, "
                                   "method 6 soft weights; each stream one CUDA graph launch",
                       "l2": "frame ring >> L2", "evd": args.evd},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "note": "one packet launched alone, CUDA events"},
            "stage_ms_per_launch": {k: v / max(n, 1) for k, v in stages.items()},
            "gpu_launches": launches, "status": L.lcf_status_string(stc),
            "frame_generation_s": round(gen_s, 1), "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def studies_workload(args):
    """The paper's image-quality studies re-run on a synthetic sequence whose vessel masks are
    known (180x180 px, packets of 50 frames every 5, tissue motion that grows across the field
    of view): maximum achievable CR / CNR per rule and subset grid over each rule's factor
    sweep, against packet length, and the GPU time per packet; not a throughput benchmark."""
    import torch
    import paper_2405_11105_b300 as L
    from paper_2405_11105_b300 import studies as S
    from synth import Recipe, generate_frames
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)

    def recipe(nt):
        return Recipe(180, 180, nt, n_vessels=6, width_px=(3.0, 8.0), phi_rad=(0.1, 0.8), tbr_db=45.0,
                      noise_db=-60.0, motion_amp_px=1.0, motion_period=40.0, motion_lateral_gain=(0.1, 2.0))

    def make(nt):
        f, t = generate_frames(recipe(nt), nt + 5 * 9, seed=21, return_truth=True)
        return f, t["blood_mask"]
    frames, mask = make(50)
    base = S.score_sequence(frames, mask, 50, 5, (1, 1), L.LCF_T_NONE, 1.0, device=local)
    rules = (L.LCF_T_CURVATURE, L.LCF_T_MEDIAN, L.LCF_T_NCC, L.LCF_T_SIGMOID, L.LCF_T_ADAPTIVE_SOFT)
    subsets = S.subset_study(frames, mask, 50, 5, grids=((1, 1), (2, 2), (3, 3), (8, 8)), rules=rules, device=local)
    sizes = S.packet_size_study(make, nts=(50, 70, 90), grids=((1, 1), (3, 3)), device=local)
    best = subsets[(S.RULE_NAMES[L.LCF_T_CURVATURE], "3x3")]
    line = {"metric": "maximum achievable CNR (dB), method 1, 3x3 subsets (synthetic 180x180 px, Nt=50, stride 5)",
            "value": best["cnr"], "unit": "dB", "higher_is_better": True, "n_gpus": 1, "impl": "ours",
            "data": "synthetic", "config": {"workload": "paper's quality studies on a synthetic sequence "
                                                       "(6 vessels, 45 dB, 1 px motion growing 0.1-2x across x)"},
            "unfiltered": base,
            "subsets": [{"rule": k[0], "grid": k[1], **v} for k, v in subsets.items()],
            "packet_sizes": [{"nt": k[0], "grid": k[1], **v} for k, v in sizes.items()]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="tc", choices=["simt", "tc"])
    ap.add_argument("--cpu-packets", type=int, default=10)
    ap.add_argument("--workload", default="realtime", choices=["realtime", "learned", "stream", "studies"],
                    help="realtime: 256x128x100 8x8 (the headline); learned: 384x256x128 16x16 with the learned "
                         "cutoff; stream: 512x256x200 16x16, sliding packets (stride 50) as one CUDA graph; "
                         "studies: the paper's CR/CNR studies on a synthetic sequence")
    ap.add_argument("--stream-packets", type=int, default=64)
    # options of the headline workload's optimized plan (defaults: the library's)
    ap.add_argument("--thresh", default="curvature", choices=["curvature", "ncc", "median", "fixed"],
                    help="thresholding rule: method 1 (default), method 4, method 3 (beta 1.43), fixed k = 8")
    ap.add_argument("--gram-precision", default="f16x3", choices=["f16x3", "bf16x3", "f16", "bf16", "e4m3"])
    ap.add_argument("--evd-precision", default="fp32", choices=["fp32", "polish"])
    ap.add_argument("--project-form", default="identity", choices=["identity", "subtract"])
    ap.add_argument("--deflate", type=int, default=0)
    ap.add_argument("--evd", default="os", choices=["pair", "os"],
                    help="EVD kernel of the optimized path: two-sided CTA pair or one-sided on the Cholesky factor")
    ap.add_argument("--tune-cache", default=None,
                    help="autotuner cache file (a profiler run can reuse the tuning of a plain run)")
    ap.add_argument("--inflight", type=int, default=4,
                    help="packets the optimized plan keeps in progress at once (lcf_filter_many)")
    ap.add_argument("--no-variants", action="store_true", help="skip the variant arms (untuned, graph, one-pass fp16)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "learned":
        return learned_workload(args)
    if args.workload == "stream":
        return stream_workload(args)
    if args.workload == "studies":
        return studies_workload(args)

    import numpy as np
    import torch
    import paper_2405_11105_b300 as L

    rank, world, local = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    ring = make_ring(seed0=ring_seed(rank))
    d_ring = torch.from_numpy(ring).to(f"cuda:{local}")
    out = torch.empty((NZ, NX), dtype=torch.float32, device=f"cuda:{local}")
    st = torch.cuda.current_stream()

    rule = {"curvature": dict(thresh_mode=L.LCF_T_CURVATURE, beta=1.0), "ncc": dict(thresh_mode=L.LCF_T_NCC),
            "median": dict(thresh_mode=L.LCF_T_MEDIAN, beta=1.43),
            "fixed": dict(thresh_mode=L.LCF_T_FIXED, k_fixed=8)}[args.thresh]
    options = dict(gram_precision=getattr(L, "LCF_GP_" + args.gram_precision.upper()),
                   evd_precision=L.LCF_EP_FP64_POLISH if args.evd_precision == "polish" else L.LCF_EP_FP32,
                   project_form=L.LCF_PF_SUBTRACT if args.project_form == "subtract" else L.LCF_PF_IDENTITY,
                   deflate=args.deflate)

    def plan_for(path, **extra):
        # optimized path: tensor-core Gram and projection, CTA-pair EVD; plain path: CUDA cores only
        evd = (L.LCF_EVD_OS if args.evd == "os" else L.LCF_EVD_PAIR) if path == L.LCF_PATH_TC else L.LCF_EVD_CTA
        # the ring is resident before the timed loop: the optimized plan may start each packet's
        # basis prep while the previous packet's kernels run (inputs_ready)
        kw = dict(device=local, gram_path=path, project_path=path, evd_path=evd,
                  inputs_ready=1 if path == L.LCF_PATH_TC else 0, **rule)
        if path == L.LCF_PATH_TC:
            kw.update(options)
            kw["inflight"] = args.inflight
        kw.update(extra)
        return L.Plan.make(NZ, NX, NT, WZ, WX, **kw)

    def barrier():
        if dist is not None:
            dist.barrier()

    out_many = torch.empty((RING, NZ, NX), dtype=torch.float32, device=f"cuda:{local}")

    def run_packets(plan, n, single=False):
        # n packets of the ring; a plan with packets in flight takes them RING at a time through
        # lcf_filter_many, the others (and single=True: stage profiling) one lcf_filter each
        if plan.cfg.inflight > 1 and not single:
            done = 0
            while done < n:
                b = min(RING, n - done)
                plan.filter_many(d_ring[:b], out_many[:b])
                done += b
        else:
            for i in range(n):
                plan.filter(d_ring[i % RING], out)

    def timed(plan, steps, warmup, single=False):
        run_packets(plan, warmup, single)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        run_packets(plan, steps, single)
        e1.record(st)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), dist, f"cuda:{local}")

    path = L.LCF_PATH_TC if args.path == "tc" else L.LCF_PATH_SIMT
    plan = plan_for(path)
    variants = {}
    if path == L.LCF_PATH_TC and not args.no_variants:
        # the launch shapes as plan_create chose them, then autotuned on the first packet
        ms_untuned = timed(plan, args.steps, args.warmup)
        variants["untuned"] = {"value": job_rate(world, args.steps, ms_untuned / 1e3), "tuning": plan.tuning().as_dict()}
    if path == L.LCF_PATH_TC:
        plan.autotune(d_ring[0], cache_path=args.tune_cache)
    run_packets(plan, args.warmup)
    n_launch0 = plan.launch_count()
    with ClockSampler(local) as clk:
        ms = timed(plan, args.steps, args.warmup)
    # kernels of this library launched per timed step (the warm-up inside timed() is excluded)
    launches_per_step = (plan.launch_count() - n_launch0) // (args.steps + args.warmup)
    clocks = clk.summary()
    value = job_rate(world, args.steps, ms / 1e3)

    # plain FP32 path (the metric's denominator) on the same ring
    plain = plan if path == L.LCF_PATH_SIMT else plan_for(L.LCF_PATH_SIMT)
    ms_plain = ms if plain is plan else timed(plain, args.steps, args.warmup)
    plain_value = job_rate(world, args.steps, ms_plain / 1e3)

    if path == L.LCF_PATH_TC and not args.no_variants:
        # the same workload as one CUDA graph launch per packet (stream order, no early basis
        # prep), and with the one-pass fp16 Gram (TF32's significand), each tuned like the headline plan
        for name, kw in (("graph", {"graph": 1, "inputs_ready": 0}), ("gram_f16", {"gram_precision": L.LCF_GP_F16})):
            vp = plan_for(path, **kw)
            vp.autotune(d_ring[0], cache_path=args.tune_cache)
            ms_v = timed(vp, args.steps, args.warmup)
            variants[name] = {"value": job_rate(world, args.steps, ms_v / 1e3), "tuning": vp.tuning().as_dict()}
            vp.close()

    # per-stage device times (CUDA events between the stages on the launch stream)
    plan.profile(True)   # one packet at a time on the plan's own workspace: stage times without overlap
    ms_prof = timed(plan, args.steps, 0, single=True)
    stages, ncalls = plan.profile_read()
    plan.profile(False)
    per_launch = {k: v / max(ncalls, 1) for k, v in stages.items()}
    work = algorithmic_work()
    dom = max(per_launch, key=per_launch.get)
    if dom in ("gram", "project") and path == L.LCF_PATH_TC:
        bound, peak, peak_src = "tensor", None, "measured bf16 (dense fp16 rate is equal)"
    else:
        bound, peak, peak_src = "alu", FP32_PEAK_TFLOPS, "FP32 SIMT: 148 SMs x 128 lanes x 2 x 2.032 GHz"
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        peaks = {}
    if bound == "tensor":
        peak = peaks.get("bf16_tflops", 1800.0)
    achieved = (work.get(dom) or 0.0) / (per_launch[dom] * 1e-3) / 1e12 if work.get(dom) else None
    roofline = {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved and peak else None,
                "traffic": captured_traffic(dom, args.evd) if path == L.LCF_PATH_TC else None,
                # SMs the dominant stage holds per packet: the one-sided EVD one per window, the CTA
                # pair two; the packets in flight share the rest of the 148
                "sms_held": (WZ * WX * (1 if args.evd == "os" else 2)) if dom == "evd" and path == L.LCF_PATH_TC else None,
                "traffic_unit": "bytes per launch (ncu capture)",
                "peak_source": peak_src,
                "stage_ms_per_launch": per_launch}
    if roofline["sms_held"] and roofline["frac"]:   # the same rate against the peak of the SMs it holds
        roofline["frac_of_held_sms"] = roofline["frac"] * 148 / roofline["sms_held"]

    # end to end through the public API with host buffers (pinned)
    # (pipelined host calls: each packet's input copy overlaps the previous packet's kernels;
    # every step still copies its packet in and its image out)
    host_ring = torch.from_numpy(ring).pin_memory()
    host_out = [torch.empty((NZ, NX), dtype=torch.float32).pin_memory() for _ in range(RING)]
    for i in range(args.warmup):
        plan.filter_host_async(host_ring[i % RING], host_out[i % RING])
    plan.sync()
    barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        plan.filter_host_async(host_ring[i % RING], host_out[i % RING])
    plan.sync()
    t1 = time.perf_counter()
    e2e_s = max_over_ranks(t1 - t0, dist, f"cuda:{local}")
    e2e = {"value": job_rate(world, args.steps, e2e_s), "unit": "frames/s",
           "h2d_bytes_per_step": int(NT * NZ * NX * 8), "d2h_bytes_per_step": int(NZ * NX * 4)}

    st_code, flags = plan.status()
    line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if path == L.LCF_PATH_SIMT else "f32 (Gram: split-f16 tensor core, f32 accumulate)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if args.thresh == "curvature" else WORKLOAD.replace(
                "adaptive curvature threshold", f"rule {args.thresh}"), "nz": NZ, "nx": NX, "nt": NT, "windows": [WZ, WX],
                       "options": {"gram_precision": args.gram_precision, "evd_precision": args.evd_precision,
                                   "project_form": args.project_form, "deflate": args.deflate or "default",
                                   "evd": args.evd},
                       "path": args.path, "l2": f"ring of {RING} packets ({RING * NT * NZ * NX * 8 / 1e6:.0f} MB) > L2",
                       "parallelism": f"replicas x{world} (independent packets), "
                                      f"{args.inflight if path == L.LCF_PATH_TC else 1} packets in flight per GPU",
                       "tuning": plan.tuning().as_dict() if path == L.LCF_PATH_TC else None},
            "variants": variants,
            "plain_fp32": {"value": plain_value, "unit": "frames/s", "ms_per_step": ms_plain / args.steps},
            "vs_plain": value / plain_value,
            "clocks": clocks, "roofline": roofline, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "status": L.lcf_status_string(st_code)}
    if rank == 0:
        nthreads = os.cpu_count() or 1
        rate, dt = cpu_oracle_rate(ring, args.cpu_packets, nthreads, args.thresh)
        line["cpu_baseline"] = {"value": rate, "unit": "frames/s", "cores": nthreads, "kind": "oracle",
                                "sample": f"{args.cpu_packets} full packets of the workload ({dt:.1f} s)"}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
