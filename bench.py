"""Benchmark of the Sub-R-HOSVD hot path (Alg. 1) on GB300.

Workload: one step = one full decomposition (fiber sample, sketch, QR, W-step,
core multi-TTM) of the order-4 128x128x128x128 float32 Tucker tensor (graded
32^4 core, Haar factors, 1e-6 noise), ranks 32, oversampling 10, s_k = 1280,
input resident in HBM.  The tensor (1.07 GB) exceeds the 129 MB L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: each rank decomposes its own copy (independent
problems, no data-path collective: weak scaling).  ``--impl reference`` times
the float64 oracle on the host cores instead (a bounded sample of the same
workload; rank 0 only).  Prints one JSON line.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "input GB/s & decomps/s at fixed rel-err, BF16/batched vs FP32 plain, % roofline"
WORKLOAD = ("Sub-R-HOSVD, order-4 128x128x128x128 float32 Tucker tensor (graded 32^4 core "
            "10^(-(i1+..+i4)/16) xi, Haar factors, N(0,1e-6^2) noise), r=32, p=10, s_k=1280, seed 1")
DOMINANT = "k_core2_tc (tcgen05 pass over X: last two core contractions, 3xBF16)"


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_traffic():
    """dram bytes per launch of the dominant kernel from the committed ncu
    summary, or None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "core2_tc_128x4.json")
    src = os.path.join(ROOT, "paper_2603_21379_gb300", "csrc", "core_tc.cu")
    try:
        with open(path) as f:
            rec = json.load(f)
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if rec.get("source_sha256") != sha:
            return None
        return rec.get("traffic_bytes_per_launch")
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons, loaded = [], 0.0, set(), []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                clk, cmax, util = float(f[1]), float(f[2]), float(f[9])
            except ValueError:
                continue
            mx = max(mx, cmax)
            sm.append(clk)
            if util > 0:
                loaded.append(clk)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        use = loaded or sm
        if not use:
            return None
        return {"sm_mhz": statistics.median(use), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(use)}


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- oracle arm
def oracle_sample(X, cfg):
    """Bounded sample of the workload on the float64 oracle: the whole factor
    stage (all 4 modes) plus the core projection of 16 of the 128 mode-1
    slices; the full-decomposition time is the factor time plus 8x the slice
    time (the core is linear in the slices)."""
    import numpy as np
    from oracle import tucker
    t0 = time.perf_counter()
    out = tucker.sub_r_hosvd(X, list(cfg["ranks"]), cfg["p"], seed=cfg["seed"], with_core=False)
    t1 = time.perf_counter()
    part = np.asarray(X[:16], dtype=np.float64)
    tucker.multi_ttm_t(part, [out["U"][0][:16]] + out["U"][1:])
    t2 = time.perf_counter()
    return (t1 - t0) + (t2 - t1) * (X.shape[0] / 16.0)


def run_reference(args):
    import numpy as np
    import synth
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    cfg = synth.ORDER4_128
    X = synth.named(cfg)
    nbytes = X.nbytes
    for _ in range(args.warmup):
        oracle_sample(X, cfg)
    times = [oracle_sample(X, cfg) for _ in range(args.steps)]
    t = sum(times)
    value = nbytes * args.steps / t / 1e9
    cores = os.cpu_count()
    sample = ("float64 oracle: factor stage of all 4 modes + core projection of 16/128 mode-1 slices "
              "per step, full-step time extrapolated linearly in the slices")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "decomps_per_s": args.steps / t,
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    import paper_2603_21379_gb300 as rt
    import synth
    from paper_2603_21379_gb300 import build

    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    build.build()
    rt.load_library()

    cfg = synth.ORDER4_128
    Xh = synth.named(cfg)
    X = torch.from_numpy(Xh).cuda()
    r, p, seed = list(cfg["ranks"]), cfg["p"], cfg["seed"]
    n = list(Xh.shape)
    nbytes = Xh.nbytes
    U = torch.empty(sum(nk * rk for nk, rk in zip(n, r)), dtype=torch.float32, device="cuda")
    G = torch.empty(r, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        rt.rtucker_decompose(X, r, p, seed=seed, out=(U, G))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches_per_step = rt.last_launch_count()
    sampler = ClockSampler(dev) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    rt.set_timing(True)
    rt.get_timing(reset=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    stages = rt.get_timing(reset=True)
    rt.set_timing(False)
    clocks = sampler.stop() if sampler else None
    if ws > 1:
        tt = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms = float(tt.item())

    # fixed-error report (untimed): relative reconstruction error of this result
    Us = [u for u in torch.split(U, [nk * rk for nk, rk in zip(n, r)])]
    Us = [u.view(nk, rk) for u, nk, rk in zip(Us, n, r)]
    relerr = rt.rtucker_relerr(X, G, Us)

    # end to end through the public API with host buffers (pinned)
    Xpin = torch.from_numpy(Xh).pin_memory()
    Uh = torch.empty(U.numel(), dtype=torch.float32).pin_memory()
    Gh = torch.empty(r, dtype=torch.float32).pin_memory()
    rt.rtucker_decompose_host(Xpin, r, p, seed=seed, out=(Uh, Gh))
    e2e_steps = max(3, min(args.steps, 10))
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rt.rtucker_decompose_host(Xpin, r, p, seed=seed, out=(Uh, Gh))
    t_e2e = time.perf_counter() - t0
    if ws > 1:
        tt = torch.tensor([t_e2e], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_e2e = float(tt.item())

    if rank == 0:
        peak, peak_src = measured_peaks()
        x_ms, x_cnt = stages["core_x_pass"]
        avg_x = x_ms / max(1, x_cnt)
        achieved = nbytes / (avg_x * 1e-3) / 1e9
        value = ws * nbytes * args.steps / (ms * 1e-3) / 1e9
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            t_cpu = oracle_sample(Xh, cfg)
            cpu = {"value": nbytes / t_cpu / 1e9, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "float64 oracle: factor stage of all 4 modes + core projection of 16/128 "
                             "mode-1 slices, full-step time extrapolated linearly in the slices"}
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "input 1.07 GB > 129 MB L2 (no flush)",
                       "parallelism": "independent problem per GPU" if ws > 1 else "single GPU"},
            "decomps_per_s": ws * args.steps / (ms * 1e-3),
            "relerr": relerr,
            "stage_ms_per_step": {k: v[0] / max(1, args.steps) for k, v in stages.items() if v[1]},
            "roofline": {"bound": "hbm", "kernel": DOMINANT, "achieved": achieved, "peak": peak,
                         "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": profile_traffic(),
                         "step_frac": (nbytes / (ms / args.steps * 1e-3) / 1e9) / peak},
            "cpu_baseline": cpu,
            "e2e": {"value": ws * nbytes * e2e_steps / t_e2e / 1e9, "unit": "GB/s",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": (U.numel() + G.numel()) * 4},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
