"""Benchmark of the Sub-R-HOSVD hot path (Alg. 1) on GB300.

Workload: one step = one full decomposition (fiber sample, sketch, QR, W-step,
core multi-TTM) of the order-4 128x128x128x128 float32 Tucker tensor (graded
32^4 core, Haar factors, 1e-6 noise), ranks 32, oversampling 10, s_k = 1280,
input resident in HBM.  The tensor (1.07 GB) exceeds the 129 MB L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

After the timed region, rank 0 also measures (CUDA events; extra keys of the
same JSON line, skipped with --no-extras): the BF16 compute form and bfloat16-
stored X of the same workload ("forms"), 256 order-3 tensors in one batched call
against a loop of plain calls ("batched"), and the H-Tucker decomposition of
the 17.2 GB 16^8 tensor with its root-pass roofline ("ht").

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


def max_over_ranks(value, device=None):
    """The largest ``value`` over all ranks of the default process group (the
    identity without one).  Timing lines report the slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def whole_job_rate(bytes_per_rank, steps, world, ms):
    """Whole-job input rate (GB/s): every rank decomposes its own tensor each step
    (independent problems, weak scaling), timed by the slowest rank."""
    return world * bytes_per_rank * steps / (ms * 1e-3) / 1e9


# ---------------------------------------------------------------- oracle arm
def oracle_sample(X, cfg):
    """One whole decomposition of the workload on the float64 oracle, timed on the
    host cores: the factor stage of all 4 modes (fiber sample, sketch, QR, W-step)
    and the full core projection G = X x_1 U_1^T ... x_4 U_4^T.  Returns seconds."""
    from oracle import tucker
    t0 = time.perf_counter()
    tucker.sub_r_hosvd(X, list(cfg["ranks"]), cfg["p"], seed=cfg["seed"], with_core=True)
    return time.perf_counter() - t0


ORACLE_SAMPLE = ("float64 NumPy oracle, one whole decomposition per step (factor stage of all 4 modes + "
                 "the full core projection), measured on the host cores (OpenBLAS threads: all)")


def bench_config(ws):
    """The workload's config object, shared by both arms."""
    return {"workload": WORKLOAD, "l2": "input 1.07 GB > 129 MB L2 (no flush)",
            "parallelism": "independent problem per GPU" if ws > 1 else "single GPU",
            "api": "rtucker_decompose, use_graph=1 (kernel sequence replayed as a CUDA graph; "
                   "tables uploaded per call)"}


def run_reference(args):
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
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(ws),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": ORACLE_SAMPLE},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "decomps_per_s": args.steps / t,
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- other forms and workloads
def _event_time(fn, steps, warmup):
    """ms per call of ``fn`` on the current stream, CUDA events, after warm-up."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _inflight_time(streams, fns, steps, warmup):
    """ms per step with len(fns) steps in flight: step i calls fns[i % P] on
    streams[i % P] (each slot with its own library handle, inputs and outputs)."""
    import torch
    P = len(fns)
    for i in range(warmup * P):
        with torch.cuda.stream(streams[i % P]):
            fns[i % P]()
    torch.cuda.synchronize()
    main = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for sk in streams:
        sk.wait_event(e0)
    for i in range(steps):
        with torch.cuda.stream(streams[i % P]):
            fns[i % P]()
    for sk in streams:
        main.wait_stream(sk)
    e1.record(main)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def measure_forms(rt, X, r, p, seed, relerr_fp32, steps):
    """BF16 compute form, bfloat16-stored X, the BF16 sketch and float8-stored X on the
    128^4 workload, against the float32 plain form: time per decomposition and the error of the
    result measured against the float32 X (the fixed-error bar is
    |delta relerr| <= 1e-5)."""
    import torch
    nbytes32 = X.numel() * 4
    out = {}
    ms = _event_time(lambda: rt.rtucker_decompose(X, r, p, seed=seed, prec="bf16"), steps, 3)
    G, U = rt.rtucker_decompose(X, r, p, seed=seed, prec="bf16")
    e = rt.rtucker_relerr(X, G, U)
    out["bf16_compute"] = {"ms_per_decomp": ms, "input_gbs": nbytes32 / (ms * 1e-3) / 1e9, "relerr": e,
                           "delta_relerr": e - relerr_fp32, "meets_fixed_relerr": abs(e - relerr_fp32) <= 1e-5}
    Xb = X.to(torch.bfloat16)
    ms = _event_time(lambda: rt.rtucker_decompose(Xb, r, p, seed=seed), steps, 3)
    G, U = rt.rtucker_decompose(Xb, r, p, seed=seed)
    e = rt.rtucker_relerr(X, G, U)
    out["bf16_stored"] = {"ms_per_decomp": ms, "input_gbs": Xb.numel() * 2 / (ms * 1e-3) / 1e9,
                          "relerr": e, "delta_relerr": e - relerr_fp32,
                          "meets_fixed_relerr": abs(e - relerr_fp32) <= 1e-5}
    del Xb
    ms = _event_time(lambda: rt.rtucker_decompose(X, r, p, seed=seed, sketch="bf16"), steps, 3)
    G, U = rt.rtucker_decompose(X, r, p, seed=seed, sketch="bf16")
    e = rt.rtucker_relerr(X, G, U)
    out["bf16_sketch"] = {"ms_per_decomp": ms, "input_gbs": nbytes32 / (ms * 1e-3) / 1e9, "relerr": e,
                          "delta_relerr": e - relerr_fp32, "meets_fixed_relerr": abs(e - relerr_fp32) <= 1e-5,
                          "form": "Z = Y Omega from bfloat16-rounded fibers and Omega, CholeskyQR2 of Z"}
    # float8 storage: E4M3 codes with one power-of-two scale per 128 x 128 slab, packed
    # once (timed apart); the decomposition reads the packed buffer
    pack_ms = _event_time(lambda: rt.quantize_fp8(X), 3, 1)
    Xq = rt.quantize_fp8(X)
    ms = _event_time(lambda: rt.rtucker_decompose(Xq, r, p, seed=seed), steps, 3)
    G, U = rt.rtucker_decompose(Xq, r, p, seed=seed)
    e = rt.rtucker_relerr(X, G, U)
    e_stored = rt.rtucker_relerr(Xq, G, U)
    rt.set_timing(True)
    rt.get_timing(reset=True)
    for _ in range(steps):
        rt.rtucker_decompose(Xq, r, p, seed=seed)
    stg = rt.get_timing(reset=True)
    rt.set_timing(False)
    out["fp8_stored"] = {"ms_per_decomp": ms, "input_gbs": Xq.data.numel() / (ms * 1e-3) / 1e9,
                         "relerr": e, "relerr_vs_stored_values": e_stored, "delta_relerr": e - relerr_fp32,
                         "meets_fixed_relerr": abs(e - relerr_fp32) <= 1e-5, "pack_ms": pack_ms,
                         "stage_ms_per_decomp": {k: v[0] / steps for k, v in stg.items() if v[1]},
                         "form": "X as E4M3 codes + per-slab power-of-two scales (1 byte/element); "
                                 "core pass kind::f8f6f4 with U_2 in four E4M3 terms"}
    del Xq
    return out


def measure_rhkron(rt, X, r, seed, relerr_plain, steps, peak):
    """Randomized HOSVD with Kronecker-structured test matrices (rHKron, the
    comparison method of Sec. 3.3) on the 128^4 workload, l = 4 per mode (64
    sketch columns): the one-pass sketch of all four modes against the HBM
    roofline, the whole method, and its error beside the subsampled form's."""
    ell = [4] * X.dim()
    nbytes = X.numel() * X.element_size()
    sk_ms = _event_time(lambda: rt.rtucker_kron_sketch(X, ell, seed=seed), steps, 3)
    ms = _event_time(lambda: rt.rtucker_rhkron(X, r, ell, seed=seed), steps, 3)
    G, U = rt.rtucker_rhkron(X, r, ell, seed=seed)
    e = rt.rtucker_relerr(X, G, U)
    ach = nbytes / (sk_ms * 1e-3) / 1e9
    return {"workload": "rHKron on the 128^4 float32 tensor, r = 32, l = 4 per mode (Z_k: 128 x 64)",
            "sketch_ms": sk_ms, "sketch_input_gbs": ach,
            "sketch_roofline": {"bound": "hbm", "kernel": "k_kron_sketch (all four sketches, one read of X)",
                                "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak},
            "ms_per_decomp": ms, "input_gbs": nbytes / (ms * 1e-3) / 1e9, "relerr": e,
            "relerr_subsampled_form": relerr_plain}


def measure_batched(rt, steps):
    """256 order-3 float32 tensors (n_k ~ U{32..160}): one batched call against a
    loop of plain calls; tensors/s, input GB/s and the largest relerr difference."""
    import torch
    import synth
    cfg = synth.BATCHED_256
    Xh, shapes, ranks = synth.batched_tensors(cfg["T"], cfg["nmin"], cfg["nmax"], cfg["rmin"], cfg["rmax"],
                                              cfg["noise"], cfg["data_seed"])
    Xs = [torch.from_numpy(x).cuda() for x in Xh]
    nbytes = sum(x.nbytes for x in Xh)
    seeds = [cfg["seed"] + t for t in range(cfg["T"])]
    p = cfg["p"]
    plan = rt.BatchedDecomposition(Xs, ranks, p, seeds, graph=True, core="tune")
    plan.run()                     # the first call times each level's schedules once
    ms_b = _event_time(plan.run, steps, 2)
    sched = plan.schedule()
    dflt = rt.BatchedDecomposition(Xs, ranks, p, seeds, graph=True)
    ms_d = _event_time(dflt.run, steps, 2)
    del dflt
    # two batches in flight (two streams, each with its own plan, handle and copy of the
    # 256 tensors): one batch's range finder runs beside the other's contractions
    streams = [torch.cuda.Stream() for _ in range(2)]
    plans = []
    for k in range(2):
        with torch.cuda.stream(streams[k]):
            Xk = Xs if k == 0 else [x.clone() for x in Xs]
            pk = rt.BatchedDecomposition(Xk, ranks, p, seeds, graph=True, core="tune")
            pk.run()
            plans.append((pk, Xk))
    torch.cuda.synchronize()
    ms_b2 = _inflight_time(streams, [pl.run for pl, _ in plans], 2 * steps, 1)
    del plans

    def plain():
        for X, rk, sd in zip(Xs, ranks, seeds):
            rt.rtucker_decompose(X, list(rk), p, seed=sd)
    ms_p = _event_time(plain, max(1, steps // 2), 1)
    res = plan.run().results()
    dmax = 0.0
    for t in range(0, cfg["T"], 16):
        Gb, Ub = res[t]
        Gp, Up = rt.rtucker_decompose(Xs[t], list(ranks[t]), p, seed=seeds[t])
        dmax = max(dmax, abs(rt.rtucker_relerr(Xs[t], Gb, Ub) - rt.rtucker_relerr(Xs[t], Gp, Up)))
    return {"workload": "256 order-3 float32 Tucker tensors, n_k ~ U{32..160}, r_k ~ U{4..min(24, n_k/4)}, "
                        "p=5, Gaussian cores, Haar factors, 1e-6 noise, %.3f GB" % (nbytes / 1e9),
            "api": "rtucker_decompose_batched, use_graph=1, core=3 (schedules tuned on the first call)",
            "schedule": sched, "ms_per_batch_default_schedule": ms_d,
            "ms_per_batch": ms_b, "tensors_per_s": cfg["T"] / (ms_b * 1e-3),
            "inflight2": {"ms_per_batch": ms_b2, "tensors_per_s": cfg["T"] / (ms_b2 * 1e-3),
                          "input_gbs": nbytes / (ms_b2 * 1e-3) / 1e9,
                          "how": "two batches in flight on two streams, one plan and copy of the tensors each"},
            "input_gbs": nbytes / (ms_b * 1e-3) / 1e9,
            "plain_loop_ms": ms_p, "plain_loop_tensors_per_s": cfg["T"] / (ms_p * 1e-3),
            "max_delta_relerr_vs_plain": dmax}


def measure_ht(rt, steps, peak, n=None, d=None):
    """Sub-R-RtL-HT of f = 1/||x|| on the 16^8 grid (17.2 GB float32), rank 10,
    p = 5, w = 320: time per decomposition, input GB/s, the root pass (one read of
    X) against the HBM roofline, and the relative error of the format.  ``n`` and
    ``d`` replace the grid size and order (profiling runs use a smaller tensor)."""
    import torch
    import synth
    cfg = dict(synth.INVNORM_16_8)
    if n is not None:
        cfg["n"] = n
    if d is not None:
        cfg["d"] = d
    X = synth.inv_norm_tensor_torch(cfg["n"], cfg["d"], cfg["lo"], cfg["hi"], device="cuda")
    nbytes = X.numel() * 4

    def step():
        return rt.rhtucker_decompose(X, cfg["rank"], cfg["p"], w=cfg["w"], seed=cfg["seed"])
    step()
    rt.set_timing(True)
    rt.get_timing(reset=True)
    ms = _event_time(step, steps, 1)
    stg = rt.get_timing(reset=True)
    rt.set_timing(False)
    root_ms = stg["ht_root_pass"][0] / max(1, stg["ht_root_pass"][1])
    U_leaf, B = step()
    e = rt.rhtucker_relerr(X, U_leaf, B, cfg["rank"])
    del U_leaf, B
    # two decompositions in flight (two streams, each with its own handle and copy of X):
    # one's range finder runs beside the other's root pass
    streams = [torch.cuda.Stream() for _ in range(2)]
    Xs = [X, X.clone()]
    fns = [lambda k=k: rt.rhtucker_decompose(Xs[k], cfg["rank"], cfg["p"], w=cfg["w"], seed=cfg["seed"])
           for k in range(2)]
    ms2 = _inflight_time(streams, fns, 2 * max(1, steps // 2), 1)
    del Xs, fns, X
    torch.cuda.empty_cache()
    return {"workload": "Sub-R-RtL-HT, f=1/||x|| on a %d^%d grid over [1,2]^%d (%.2f GB float32), balanced "
                        "tree, rank 10, p=5, w=320 columns per node, seed 3"
                        % (cfg["n"], cfg["d"], cfg["d"], nbytes / 1e9),
            "ms_per_decomp": ms, "input_gbs": nbytes / (ms * 1e-3) / 1e9, "relerr": e,
            "inflight2": {"ms_per_decomp": ms2, "input_gbs": nbytes / (ms2 * 1e-3) / 1e9,
                          "how": "two decompositions in flight on two streams, one handle and copy of X each"},
            "stage_ms": {k: v[0] / max(1, v[1]) for k, v in stg.items() if v[1]},
            "root_roofline": {"bound": "hbm", "kernel": "k_root (B_R = U_l^T X U_r, one read of X)",
                              "achieved": nbytes / (root_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                              "frac": nbytes / (root_ms * 1e-3) / 1e9 / peak}}


def measure_scaling(rt, steps, ns=None):
    """The paper's scaling workloads on one GPU (its parallel experiments):
    Sub-R-HOSVD of order-8 low-rank tensors (rank 5, n = 16, 18, 20: 17 to 102 GB
    float32, s = 10^4 fibers per mode) and Sub-R-RtL-HT of f = 1/||x|| on n^8 grids
    (rank 6, 20 n fibers per node).  Each: graph replay, CUDA events, stage times,
    input GB/s and the relative error of the result."""
    import torch
    import synth
    out = {"tucker": [], "ht": []}
    ct = synth.SCALING_TUCKER
    for n in (ns or ct["ns"]):
        shape, r = (n,) * ct["d"], [ct["rank"]] * ct["d"]
        X = synth.tucker_tensor_torch(shape, tuple(r), noise=ct["noise"], data_seed=n, device="cuda")
        nbytes = X.numel() * 4
        U = torch.empty(sum(n * k for k in r), dtype=torch.float32, device="cuda")
        G = torch.empty(r, dtype=torch.float32, device="cuda")
        s = [ct["s"]] * ct["d"]

        def step():
            rt.rtucker_decompose(X, r, ct["p"], s=s, seed=ct["seed"], out=(U, G), graph=True)
        rt.set_timing(True)
        ms = _event_time(step, steps, 2)
        stg = rt.get_timing(reset=True)
        rt.set_timing(False)
        Us = [u.view(n, k) for u, k in zip(torch.split(U, [n * k for k in r]), r)]
        e = rt.rtucker_relerr(X, G, Us)
        calls = steps + 2
        out["tucker"].append({"n": n, "gb": nbytes / 1e9, "ms_per_decomp": ms,
                              "input_gbs": nbytes / (ms * 1e-3) / 1e9, "relerr": e,
                              "stage_ms_per_decomp": {k: v[0] / calls for k, v in stg.items() if v[1]}})
        del X, U, G, Us
        torch.cuda.empty_cache()
    ch = synth.SCALING_HT
    for n in (ns or ch["ns"]):
        X = synth.inv_norm_tensor_torch(n, ch["d"], ch["lo"], ch["hi"], device="cuda")
        nbytes = X.numel() * 4
        w = ch["w_per_n"] * n

        def step():
            return rt.rhtucker_decompose(X, ch["rank"], ch["p"], w=w, seed=ch["seed"])
        step()
        rt.set_timing(True)
        rt.get_timing(reset=True)
        ms = _event_time(step, steps, 1)
        stg = rt.get_timing(reset=True)
        rt.set_timing(False)
        U_leaf, B = step()
        e = rt.rhtucker_relerr(X, U_leaf, B, ch["rank"])
        calls = steps + 1
        out["ht"].append({"n": n, "gb": nbytes / 1e9, "ms_per_decomp": ms,
                          "input_gbs": nbytes / (ms * 1e-3) / 1e9, "relerr": e,
                          "stage_ms_per_decomp": {k: v[0] / calls for k, v in stg.items() if v[1]}})
        del X, U_leaf, B
        torch.cuda.empty_cache()
    out["workload"] = ("Sub-R-HOSVD: order-8 float32 tensors n^8, n = %s (Gaussian 5^8 core, Q-of-Gaussian "
                       "factors, 1e-6 noise, built on the device), r = 5, p = 5, s = 10^4 per mode; "
                       "Sub-R-RtL-HT: f = 1/||x|| on n^8 grids over [1,2]^8, rank 6, p = 5, w = 20 n"
                       % (list(ns or ct["ns"]),))
    return out


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

    # (1) one decomposition at a time, its kernel sequence replayed as a CUDA graph, with
    # the library's stage timing on: the latency of a decomposition, its stages and the
    # dominant kernel's duration
    def step():
        rt.rtucker_decompose(X, r, p, seed=seed, out=(U, G), graph=True)

    rt.set_timing(True)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    rt.get_timing(reset=True)
    launches_per_step = rt.last_launch_count()
    rank_barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    rank_barrier()
    ms_serial = max_over_ranks(e0.elapsed_time(e1), device="cuda")
    stages = rt.get_timing(reset=True)
    rt.set_timing(False)

    # (2) the timed run: P decompositions in flight, step i on CUDA stream i % P, each
    # stream with its own library handle, its own copy of X and its own outputs, so that
    # the latency-bound range finder of one decomposition runs beside the HBM-bound
    # pass over X of another.  Every step is a whole decomposition of a 1.07 GB input.
    P = max(1, args.inflight)
    streams = [stream] + [torch.cuda.Stream() for _ in range(P - 1)]
    Xs = [X] + [X.clone() for _ in range(P - 1)]
    outs = [(U, G)] + [(torch.empty_like(U), torch.empty_like(G)) for _ in range(P - 1)]

    def pstep(i):
        k = i % P
        with torch.cuda.stream(streams[k]):
            rt.rtucker_decompose(Xs[k], r, p, seed=seed, out=outs[k], graph=True)

    for i in range(max(args.warmup, 1) * P):
        pstep(i)
    torch.cuda.synchronize()
    sampler = ClockSampler(dev) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    rank_barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for sk in streams[1:]:
        sk.wait_event(e0)
    for i in range(args.steps):
        pstep(i)
    for sk in streams[1:]:
        stream.wait_stream(sk)
    e1.record(stream)
    torch.cuda.synchronize()
    rank_barrier()
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(ms, device="cuda")
    del Xs, outs

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
    rank_barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        rt.rtucker_decompose_host(Xpin, r, p, seed=seed, out=(Uh, Gh))
    t_sync = max_over_ranks(time.perf_counter() - t0, device="cuda")
    # pipelined host call: each step's copy of X overlaps the previous step's
    # decomposition; every step's copies in and out are inside the timed region
    for _ in range(2):   # both input slots, their graphs captured
        rt.rtucker_decompose_host_async(Xpin, r, p, seed=seed, out=(Uh, Gh), graph=True)
    rt.sync()
    e2e_pipe = max(3, min(args.steps, 20))
    rank_barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_pipe):
        rt.rtucker_decompose_host_async(Xpin, r, p, seed=seed, out=(Uh, Gh), graph=True)
    rt.sync()
    t_e2e = max_over_ranks(time.perf_counter() - t0, device="cuda")

    extra = {}
    if rank == 0 and not args.no_extras:
        peak0, _ = measured_peaks()
        xs = min(args.steps, 20)
        extra["forms"] = measure_forms(rt, X, r, p, seed, relerr, xs)
        extra["rhkron"] = measure_rhkron(rt, X, r, seed, relerr, xs, peak0)
        extra["batched"] = measure_batched(rt, max(2, min(args.steps, 5)))
        del Xpin, Uh, Gh
        extra["ht"] = measure_ht(rt, max(2, min(args.steps, 5)), peak0)
        extra["grad"] = measure_grad(rt, max(3, min(args.steps, 10)), peak0)
        # the paper's order-8 scaling workloads at n = 16 (17.2 GB each); 18 and 20 with
        # --only scaling
        extra["scaling_n16"] = measure_scaling(rt, max(2, min(args.steps, 3)), ns=(16,))

    if rank == 0:
        peak, peak_src = measured_peaks()
        x_ms, x_cnt = stages["core_x_pass"]
        avg_x = x_ms / max(1, x_cnt)
        achieved = nbytes / (avg_x * 1e-3) / 1e9
        value = whole_job_rate(nbytes, args.steps, ws, ms)
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            # bounded: whole oracle decompositions until about 10 s of host time
            ts = []
            while not ts or (sum(ts) < 10.0 and len(ts) < 8):
                ts.append(oracle_sample(Xh, cfg))
            cpu = {"value": nbytes * len(ts) / sum(ts) / 1e9, "unit": "GB/s", "cores": os.cpu_count(),
                   "kind": "oracle", "sample": ORACLE_SAMPLE + ", %d decompositions" % len(ts)}
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 storage, 3xbf16-split compute, f32 accumulate", "data": "synthetic",
            "config": bench_config(ws),
            "decomps_per_s": ws * args.steps / (ms * 1e-3),
            "execution": {"inflight": P, "how": "step i on CUDA stream i %% %d, one library handle, input copy "
                          "and output per stream" % P,
                          "one_at_a_time": {"ms_per_decomp": ms_serial / args.steps,
                                            "value": whole_job_rate(nbytes, args.steps, ws, ms_serial),
                                            "unit": "GB/s"}},
            "relerr": relerr,
            "stage_ms_per_step": {k: v[0] / max(1, args.steps) for k, v in stages.items() if v[1]},
            "stage_note": "stages and the roofline kernel timed in the one-at-a-time run",
            "roofline": {"bound": "hbm", "kernel": DOMINANT, "achieved": achieved, "peak": peak,
                         "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": profile_traffic(),
                         "step_frac": (nbytes / (ms / args.steps * 1e-3) / 1e9) / peak},
            "cpu_baseline": cpu,
            "e2e": {"value": ws * nbytes * e2e_pipe / t_e2e / 1e9, "unit": "GB/s",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": (U.numel() + G.numel()) * 4,
                    "api": "rtucker_decompose_host_async x%d + sync (pinned host X, graph replay)" % e2e_pipe,
                    "synchronous_value": ws * nbytes * e2e_steps / t_sync / 1e9},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
        }
        line.update(extra)
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def measure_grad(rt, steps, peak):
    """Differentiable Tucker on the order-4 96 workload (96^4 float32, Gaussian 16^4
    core, Haar factors, 1e-4 noise): the misfit 1/2 ||X - G x_k U_k||^2 and all its
    gradients (dX, dG, dU) at the Sub-R-HOSVD result (r = 16, p = 8), one
    rtucker_loss_grad call per step.  Rate against the minimal traffic of the
    step (X read twice, the residual dX written once: 3 x 0.34 GB)."""
    import torch
    import synth
    cfg = synth.ORDER4_96
    X = torch.from_numpy(synth.named(cfg)).cuda()
    r, p = list(cfg["ranks"]), cfg["p"]
    G, U = rt.rtucker_decompose(X, r, p, seed=cfg["seed"])
    Uf = torch.cat([u.reshape(-1) for u in U])
    Ul = list(torch.split(Uf, [u.numel() for u in U]))
    Ul = [u.view(t.shape) for u, t in zip(Ul, U)]
    nbytes = X.numel() * 4

    def step():
        return rt.rtucker_loss_grad(X, G, Ul)
    ms = _event_time(step, steps, 3)
    loss = step()[0].item()
    launches = rt.last_launch_count()
    floor_bytes = 3 * nbytes
    del X
    torch.cuda.empty_cache()
    return {"workload": "misfit and gradients (dX, dG, dU) of a Tucker model of a 96^4 float32 tensor "
                        "(Gaussian 16^4 core, Haar factors, 1e-4 noise) at its Sub-R-HOSVD result, r=16, p=8",
            "ms_per_step": ms, "input_gbs": nbytes / (ms * 1e-3) / 1e9, "loss": loss, "launches": launches,
            "floor": {"bytes": floor_bytes, "ms_at_peak": floor_bytes / (peak * 1e9) * 1e3,
                      "frac": (floor_bytes / (ms * 1e-3) / 1e9) / peak, "peak_gbs": peak}}


def run_only(args):
    """One workload alone (for profiling): prints its JSON object."""
    import torch
    import paper_2603_21379_gb300 as rt
    from paper_2603_21379_gb300 import build
    torch.cuda.set_device(0)
    build.build()
    rt.load_library()
    peak, _ = measured_peaks()
    if args.only == "ht":
        out = measure_ht(rt, args.steps, peak, n=args.ht_n, d=args.ht_d)
    elif args.only == "grad":
        out = measure_grad(rt, args.steps, peak)
    elif args.only == "scaling":
        out = measure_scaling(rt, args.steps)
    elif args.only == "rhkron":
        import synth
        cfg = synth.ORDER4_128
        X = torch.from_numpy(synth.named(cfg)).cuda()
        G, U = rt.rtucker_decompose(X, list(cfg["ranks"]), cfg["p"], seed=cfg["seed"])
        out = measure_rhkron(rt, X, list(cfg["ranks"]), cfg["seed"], rt.rtucker_relerr(X, G, U), args.steps, peak)
    else:
        out = measure_batched(rt, args.steps)
    print(json.dumps({"only": args.only, **out}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--inflight", type=int, default=8,
                    help="decompositions in flight in the timed run (one CUDA stream each)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", choices=["ht", "batched", "grad", "scaling", "rhkron"], default=None,
                    help="run one extra workload alone (profiling), not the benchmark line")
    ap.add_argument("--ht-n", type=int, default=None, help="grid size of the H-Tucker workload with --only ht")
    ap.add_argument("--ht-d", type=int, default=None, help="order of the H-Tucker workload with --only ht")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the BF16 forms, the batched, H-Tucker and gradient workloads (untimed extras)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
