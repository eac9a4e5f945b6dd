"""Benchmark of the GB300 jump-SDE proton dose engine.

One step = one pass of the whole transport path over one batch: zero the tally, prepare
the spots (device-resident), and transport every history of the workload (persistent
kernel: source sampling, Euler-Maruyama steps, jumps, voxel lookup, fixed-point tally).
The default workload is the longitudinally heterogeneous slab phantom: 150 MeV beam,
lateral sigma 3 mm, 10^6 protons, 60 x 60 x 200 mm at 0.5 mm voxels (water / bone-like /
lung-like / water).  Its inputs (29 MB phantom + 46 MB tally) fit in L2, so L2 is flushed
(256 MB write) before every timed step, outside the timed events.

Prints one JSON line (rank 0).  Under torchrun (N > 1) the ranks split one plan of N x 10^6
histories by global history id (each rank its own 10^6, weak scaling, no collective in
the timed steps) and the step time is the maximum over ranks; after timing, one exact
integer all-reduce of the tallies gives the combined dose, and its time is reported.

``--impl reference`` times the FP64 CPU oracle instead (on the host cores, rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic lane operations per Euler-Maruyama step of the transport kernel (one
# Philox4x32-10 block, two Box-Muller transforms, table interpolation of five fields,
# kinematic factors, Lynch-Dahl width, spherical Brownian rotation, exponential jump
# clock, two voxel lookups, fixed-point conversion and one 64-bit atomic).  The
# breakdown is listed with the roofline in the design notes.
ALGO_OPS_PER_STEP = 200
SMS = 152
LANE_OPS_PER_CLK_PER_SM = 128  # 4 schedulers x 32 lanes, one instruction per clock each
# DRAM traffic (read + write bytes) per transport launch from the ncu capture of the
# same launch configuration; None until captured for the current kernel.
TRANSPORT_DRAM_BYTES = 70_678_528  # 60.26 MB read + 10.42 MB written, ncu 1-pass capture of the bench launch (profiles/k_transport_slab150.md)

CT_DESC = ("ct_sobp: thorax-like synthetic CT 120x120x240 mm at 1 mm (air, lung, adipose, soft tissue, "
           "cortical bone from HU), 16-layer spread-out Bragg peak 90-140 mm, 256 spots, 1e6 protons per GPU")
WORKLOAD_DESC = ("slab150: 150 MeV pencil beam (sigma_xy 3 mm), 1e6 protons per GPU, "
                 "60x60x200 mm at 0.5 mm (120x120x400 voxels), water/bone-like/lung-like/water slabs")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        top = max(sm)
        loaded = [s for s in sm if s >= 0.5 * top] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power), "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(target_s: float = 25.0):
    """The oracle as it stands on the host cores, on a bounded sample of the workload."""
    import oracle
    from sde_workloads import slab150

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    cal = 20_000
    t0 = time.perf_counter()
    oracle.run_workload(slab150(cal), seed=12345)
    dt = time.perf_counter() - t0
    n = int(min(5_000_000, max(cal, cal * target_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    _, _, bal = oracle.run_workload(slab150(n), seed=777)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "histories/s", "cores": cores, "kind": "oracle",
            "sample": f"slab150 workload, {n} histories (seed 777), FP64 oracle, {cores} threads, "
                      f"{dt:.1f} s", "steps_per_s": bal["steps"] / dt}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from sde_workloads import slab150

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    n = args.ref_histories
    for w in range(args.warmup):
        oracle.run_workload(slab150(n), seed=10_000 + w)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        oracle.run_workload(slab150(n), seed=20_000 + k)
        times.append(time.perf_counter() - t0)
    T = sum(times) / len(times)
    v = n / T
    line = {
        "impl": "reference", "metric": "proton histories/s on 1 GB300; time-to-dose at \u226595% gamma 2%/0.5mm, learned vs plain", "value": v,
        "unit": "histories/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": T * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC.replace("1e6 protons per GPU", f"{n} protons per step (bounded sample)"),
                   "histories_per_step": n, "parallelism": f"{cores} host threads"},
        "cpu_baseline": {"value": v, "unit": "histories/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n} histories of the slab150 workload per step"},
        "e2e": {"value": v, "unit": "histories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def plan_benchmark(torch, S, dev, total=100_000_000, per_spot_sample=200):
    """The 2000-spot plan phantom (200x200x300 mm, 30 spheres) with 1e8 protons:
    default launch shape, autotuned shape, graph launch, and one launch per spot
    (timed on the first ``per_spot_sample`` spots and scaled to all 2000)."""
    from sde_workloads import plan2000
    wl = plan2000(total)
    st = torch.cuda.Stream(device=dev)
    d = S.SdeDose(wl, stream=st)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sp = torch.from_numpy(wl.spots.view(np.uint8).copy()).to(dev)

    def timed(fn, reps=3):
        ts = []
        for r in range(reps + 1):
            with torch.cuda.stream(st):
                flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            d.reset()
            a.record(st)
            fn(r)
            b.record(st)
            st.synchronize()
            if r:
                ts.append(a.elapsed_time(b))
        return min(ts)

    out = {"workload": "plan2000: 2000 spots, E U(70,200) MeV, lognormal weights, 1e8 protons, "
                       "200x200x300 mm at 1 mm, water + 30 spheres"}
    out["one_launch_default_ms"] = timed(lambda r: d.run_device(sp.data_ptr(), len(wl.spots), seed=r))
    out["autotuned"] = d.autotune(wl.spots, seed=5, max_histories=2_000_000)
    out["one_launch_autotuned_ms"] = timed(lambda r: d.run_device(sp.data_ptr(), len(wl.spots), seed=r))
    d.set_tuning(graph=2)
    out["one_launch_graph_ms"] = timed(lambda r: d.run_device(sp.data_ptr(), len(wl.spots), seed=r))
    d.set_tuning(graph=1)
    n = per_spot_sample
    rec = int(wl.spots.dtype.itemsize)

    def per_spot(r):
        for i in range(n):
            d.run_device(sp.data_ptr() + i * rec, 1, seed=r * 10_000 + i)

    t_sample = timed(per_spot, reps=1)
    hist_sample = int(wl.spots["n_hist"][:n].sum())
    out["per_spot_sample"] = {"spots": n, "histories": hist_sample, "ms": t_sample}
    out["per_spot_all_2000_ms_estimated"] = t_sample * len(wl.spots) / n
    out["histories_per_s_one_launch"] = wl.n_histories / (min(out["one_launch_default_ms"],
                                                             out["one_launch_autotuned_ms"]) * 1e-3)
    out["histories_per_s_per_spot"] = hist_sample / (t_sample * 1e-3)
    d.close()
    return out


# Executed multiply-adds of one denoiser inference on 128 x 128 x 192 (16-channel padded
# input and output layers): (voxels, Cin, Cout) per convolution, 27 taps each.
DENOISER_LAYERS = [(3_145_728, 16, 32), (3_145_728, 32, 32), (393_216, 32, 64), (393_216, 64, 64),
                   (49_152, 64, 128), (49_152, 128, 128), (393_216, 192, 64), (393_216, 64, 64),
                   (3_145_728, 96, 32), (3_145_728, 32, 32), (3_145_728, 32, 16)]
DENOISER_WEIGHTS = os.path.join(ROOT, "paper_2511_03115_gb300", "weights", "denoiser_128x128x192.npy")


def time_to_dose(torch, S, seeds=(100_000, 100_001, 100_002, 100_003), ladder=(300_000, 1_000_000, 3_000_000)):
    """Learned vs plain time to a dose that passes gamma 2 %/0.5 mm (1 % threshold) against
    the 10^7-history dose of the same plan: device time of the 10^5-history run plus
    inference with the trained weights, and of plain runs at the ladder's history counts."""
    from paper_2511_03115_gb300 import denoise as DN
    if not os.path.exists(DENOISER_WEIGHTS):
        return {"unavailable": "no trained weights at paper_2511_03115_gb300/weights/"}
    net = S.Denoiser(DN.SHAPE[2], DN.SHAPE[1], DN.SHAPE[0], batch_max=1, seed=1)
    net.set_params(np.load(DENOISER_WEIGHTS).astype(np.float32))
    st = torch.cuda.current_stream()
    rows = []
    for seed in seeds:
        r = DN.transport_doses(seed)
        ref = S.scale_(r["high"], DN.N_LOW / DN.N_HIGH)
        net.infer(r["low"], r["density"])  # warm
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        den = net.infer(r["low"], r["density"])
        b.record(st)
        st.synchronize()
        S.denoise_status()
        t_inf = a.elapsed_time(b)
        rmax = float(ref.max())
        row = {"seed": seed, "t_low_ms": r["low_ms"], "t_infer_ms": t_inf, "t_high_ms": r["high_ms"],
               "gamma_low": S.gamma3d(ref, r["low"], (1.0, 1.0, 1.0)),
               "gamma_learned": S.gamma3d(ref, den, (1.0, 1.0, 1.0)),
               "max_err_low": float((r["low"] - ref).abs().max()) / rmax,
               "max_err_learned": float((den - ref).abs().max()) / rmax,
               "plain": DN.plain_ladder(seed, ref, DN.N_LOW, ladder=ladder)}
        rows.append(row)
    net.close()
    mean = lambda k: float(np.mean([r[k] for r in rows]))
    learned_ms = mean("t_low_ms") + mean("t_infer_ms")
    plain = [{"histories": n, "ms": float(np.mean([r["plain"][j]["ms"] for r in rows])),
              "gamma": float(np.mean([r["plain"][j]["gamma"] for r in rows])),
              "all_ge_95": all(r["plain"][j]["gamma"] >= 0.95 for r in rows)} for j, n in enumerate(ladder)]
    first_pass = next((p for p in plain if p["all_ge_95"]), None)
    return {"cases": len(rows), "learned_ms": learned_ms, "gamma_learned": mean("gamma_learned"),
            "learned_all_ge_95": all(r["gamma_learned"] >= 0.95 for r in rows),
            "max_err_learned": mean("max_err_learned"), "gamma_low": mean("gamma_low"),
            "max_err_low": mean("max_err_low"), "plain_1e7_ms": mean("t_high_ms"), "plain_ladder": plain,
            "plain_ms_at_95": first_pass["ms"] if first_pass else None,
            "plain_histories_at_95": first_pass["histories"] if first_pass else None,
            "note": "device time (CUDA events) of transport + dose conversion (+ inference); gamma 2%/0.5mm, "
                    "1% threshold, local, vs the 1e7-history plain dose; held-out seeds of the denoiser workload"}


def denoiser_roofline(torch, S, peaks):
    """Inference time of the denoiser on 128 x 128 x 192 and its tensor throughput."""
    net = S.Denoiser(192, 128, 128, batch_max=1, seed=1)
    low = torch.rand(192, 128, 128, device="cuda")
    rho = torch.ones_like(low)
    st = torch.cuda.current_stream()
    for _ in range(3):
        net.infer(low, rho)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(5):
        net.infer(low, rho)
    b.record(st)
    st.synchronize()
    S.denoise_status()
    net.close()
    ms = a.elapsed_time(b) / 5
    flop = sum(2.0 * v * 27 * ci * co for v, ci, co in DENOISER_LAYERS)
    peak = peaks.get("bf16_tflops")
    tf = flop / (ms * 1e-3) / 1e12
    return {"infer_ms": ms, "flop_per_inference": flop, "achieved_tflops": tf, "bound": "tensor",
            "peak_tflops": peak, "frac": tf / peak if peak else None,
            "peak_note": "measured bf16 burst peak (MEASURED_PEAKS.json)" if peak else "no measured peak"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--histories", type=int, default=1_000_000)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-histories", type=int, default=20_000)
    ap.add_argument("--workload", default="slab150", choices=["slab150", "ct_sobp"],
                    help="slab150 (default) or ct_sobp: thorax-like synthetic CT with a 16-layer spread-out Bragg peak")
    ap.add_argument("--theta-cut-sigmas", type=float, default=0.0,
                    help="energy-dependent elastic cut-off theta_c = k sigma(E) (0: the paper's fixed 0.02 rad)")
    ap.add_argument("--physics-mask", type=int, default=15,
                    help="ablation: SDE_PHYS_* bits of the transport (15 = all terms; 11 = no large-angle "
                         "elastic events, 3 = no jumps); a run with terms switched off is not the benchmark")
    ap.add_argument("--no-denoiser", action="store_true",
                    help="skip the learned-vs-plain time-to-dose and the denoiser throughput")
    ap.add_argument("--plan", action="store_true",
                    help="also time the 2000-spot plan (1e8 protons): one persistent launch, "
                         "autotuned, graph-launched, and one launch per spot")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2511_03115_gb300 as S
    from sde_workloads import ct_sobp, slab150

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # one plan; this rank runs its shard of the history ids
    wl = (ct_sobp if args.workload == "ct_sobp" else slab150)(args.histories * ws)
    first, count = S.history_shard(wl.n_histories, rank, ws)
    stream = torch.cuda.Stream(device=dev)
    d = S.SdeDose(wl, stream=stream, theta_cut_sigmas=args.theta_cut_sigmas, physics_mask=args.physics_mask)
    spots_dev = torch.from_numpy(wl.spots.view(np.uint8).copy()).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    seed_base = 1_000_003

    def step(k):
        d.reset()
        d.run_device(spots_dev.data_ptr(), len(wl.spots), seed=seed_base + k, first=first, count=count)

    for w in range(args.warmup):
        step(10_000 + w)
    d.sync()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    evs = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        s = torch.cuda.Event(enable_timing=True)
        m = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        d.reset()
        m.record(stream)
        d.run_device(spots_dev.data_ptr(), len(wl.spots), seed=seed_base + k, first=first, count=count)
        e.record(stream)
        evs.append((s, m, e))
    stream.synchronize()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [s.elapsed_time(e) for s, _, e in evs]
    kern_ms = [m.elapsed_time(e) for _, m, e in evs]
    T = sum(step_ms) / len(step_ms)
    Tk = sum(kern_ms) / len(kern_ms)
    _, _, bal = d.fetch(dose=False, edep=False)
    if ws > 1:
        t = torch.tensor([T, Tk], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        T, Tk = float(t[0]), float(t[1])
    hist_per_step = wl.n_histories  # all ranks' shards
    value = hist_per_step / (T * 1e-3)
    steps_per_launch = bal["steps"]

    # end to end through the public API with host buffers: spots H2D, dose D2H (pinned)
    host_dose = torch.empty(wl.n_voxels, dtype=torch.float64).pin_memory()
    e2e_times = []
    for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d.reset()
        d.run(wl.spots, seed=seed_base + 50_000 + k, first=first, count=count)
        d.fetch_into(dose_ptr=host_dose.data_ptr())
        t1 = time.perf_counter()
        if k > 0:
            e2e_times.append(t1 - t0)
    e2e_T = sum(e2e_times) / len(e2e_times) if e2e_times else float("nan")
    if ws > 1:
        t = torch.tensor([e2e_T], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_T = float(t[0])

    combine = None
    if ws > 1:  # the one exchange step of the split: an exact integer sum of the tallies
        d.reset()
        d.run_device(spots_dev.data_ptr(), len(wl.spots), seed=seed_base + 90_000, first=first, count=count)
        tally = torch.empty(wl.n_voxels, dtype=torch.int64, device=dev)
        rb = d.fetch_device(edep_ptr=tally.data_ptr(), balance=True)
        bt = torch.tensor([rb[k] for k in ("incident", "deposited", "escaped", "removed", "histories")],
                          dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        dist.barrier()
        c0 = time.perf_counter()
        dist.all_reduce(tally, op=dist.ReduceOp.SUM)
        torch.cuda.synchronize()
        c1 = time.perf_counter()
        dist.all_reduce(bt, op=dist.ReduceOp.SUM)
        inc, dep, esc, rem, nh = [int(v) for v in bt.tolist()]
        combine = {"allreduce_ms": (c1 - c0) * 1e3, "bytes": wl.n_voxels * 8, "histories": nh,
                   "balance_exact": inc == dep + esc + rem and nh == wl.n_histories,
                   "tally_sum_equals_deposited": int(tally.sum()) == dep}

    peaks = _peaks()
    clk_mhz = peaks.get("sm_max_mhz", 2070.0)
    peak_ops = SMS * LANE_OPS_PER_CLK_PER_SM * clk_mhz * 1e6
    achieved = steps_per_launch * ALGO_OPS_PER_STEP / (Tk * 1e-3)
    line = {
        "metric": "proton histories/s on 1 GB300; time-to-dose at \u226595% gamma 2%/0.5mm, learned vs plain",
        "value": value,
        "unit": "histories/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": T,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC if args.workload == "slab150" else CT_DESC,
                   "histories_per_step": hist_per_step,
                   "split": f"history ids {first}..{first + count - 1} of {wl.n_histories} on rank {rank}",
                   "euler_steps_per_launch": steps_per_launch, "parallelism": f"replicas x{ws}",
                   "l2": "flushed (256 MB write) before every timed step", "tally": "int64 fixed point 2^-24 MeV",
                   "elastic_cut_off": (f"theta_c = {args.theta_cut_sigmas} sigma(E)" if args.theta_cut_sigmas > 0
                                       else "fixed 0.02 rad"),
                   "physics_mask": args.physics_mask,
                   "tuning": d.get_tuning()},
        "e2e": {"value": hist_per_step / e2e_T, "unit": "histories/s",
                "h2d_bytes_per_step": int(wl.spots.nbytes),
                "d2h_bytes_per_step": int(wl.n_voxels * 8 + 64)},
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_ops / 1e9,
                     "unit": "Gop/s", "frac": achieved / peak_ops, "traffic": TRANSPORT_DRAM_BYTES,
                     "kernel": "k_transport (+ single-block spot prep)", "kernel_ms": Tk,
                     "ops_per_step": ALGO_OPS_PER_STEP,
                     "peak_note": f"{SMS} SMs x {LANE_OPS_PER_CLK_PER_SM} lane-ops/clk x {clk_mhz:.0f} MHz (max SM clock)"},
        "clocks": clocks,
        "balance_exact": bal["incident"] == bal["deposited"] + bal["escaped"] + bal["removed"],
        "combine": combine,
    }
    if args.plan:
        line["batched_plan"] = plan_benchmark(torch, S, dev)
    if rank == 0 and ws == 1 and not args.no_denoiser:
        line["time_to_dose"] = time_to_dose(torch, S)
        line["denoiser"] = denoiser_roofline(torch, S, peaks)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    d.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
