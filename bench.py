"""Benchmark of the GB300 jump-SDE proton dose engine.

One step = one pass of the whole transport path over one batch: zero the tally, prepare
the spots (device-resident), and transport every history of the workload in one
persistent launch (source sampling, Euler-Maruyama steps, jumps, voxel lookup,
fixed-point tally).  The default workload is the batched treatment plan: 2000 spots on a
5 mm lateral grid, energies uniform in 70-200 MeV, lognormal(0, 0.7) weights, 10^8
protons in total (histories per spot proportional to weight), 200 x 200 x 300 mm at
1 mm, water with 30 random spherical inserts.  The launch shape is picked by the
library's autotuner before the warm-up steps.  Its inputs (48 MB phantom + 96 MB tally)
exceed L2, and L2 is also flushed (256 MB write) before every timed step, outside the
timed events.

Secondary keys of the same line: the plan run as one launch per spot (all 2000 spots),
the slab phantom (150 MeV, 10^6 protons, 0.5 mm voxels), the learned-vs-plain time to
dose and the denoiser's tensor throughput.

Prints one JSON line (rank 0).  Under torchrun (N > 1) the ranks split one plan of N x
10^8 histories by global history id (each rank its own 10^8, weak scaling, no collective
in the timed steps) and the step time is the maximum over ranks; after timing, one exact
integer all-reduce of the tallies gives the combined dose, and its time is reported.

``--impl reference`` times the FP64 CPU oracle instead (on the host cores, rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "proton histories/s on 1 GB300; time-to-dose at \u226595% gamma 2%/0.5mm, learned vs plain"

# Algorithmic lane operations per Euler-Maruyama step of the transport kernel (one
# Philox4x32-10 block, two Box-Muller transforms, table interpolation of five fields,
# kinematic factors, Lynch-Dahl width, spherical Brownian rotation, exponential jump
# clock, two voxel lookups, fixed-point conversion and one 64-bit atomic).  The
# breakdown is listed with the roofline in the design notes.
ALGO_OPS_PER_STEP = 200
LANE_OPS_PER_CLK_PER_SM = 128  # 4 schedulers x 32 lanes, one instruction per clock each

# DRAM traffic (read + write bytes) of one transport launch, from a one-pass ncu capture of
# the benchmark's own launch, valid only for the transport source it was taken on (the
# hash of the kernel's source files); otherwise the line reports null.
TRANSPORT_SOURCES = ("sde_transport.cu", "sde_internal.cuh", "sde_transport.h")
TRANSPORT_DRAM = {  # workload -> {"src": sha256 prefix, "bytes": per launch, "note": ...}
    "plan2000": {"src": "2c263b682767634b", "bytes": 1_496_984_320 + 1_409_387_520, "histories": 100_000_000,
                 "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the first timed launch of "
                         "`bench.py --steps 2 --warmup 1 --no-denoiser --no-cpu-baseline --no-secondary` "
                         "(1 pass; profiles/k_transport_plan2000.md)"},
}

# L2 reduction (tally `red.add.u64`) rate of the transport kernel, from ncu on the plan's first
# 2e6 histories; reported only while the transport sources match the hash it was taken on.
TRANSPORT_ATOMICS = {
    "plan2000": {"src": "2c263b682767634b", "l2_red_pct_of_peak": 14.78, "busiest_l2_slice_pct": 16.77,
                 "red_sectors": 433_046_965, "euler_steps": 525_487_490,
                 "note": "ncu lts__t_sectors_srcunit_tex_op_red (.sum, .avg/.max pct_of_peak_sustained_elapsed) of "
                         "k_transport in `bench.py --histories 2000000 --no-autotune --steps 1 --warmup 1 "
                         "--e2e-steps 0 --no-denoiser --no-cpu-baseline --no-secondary` "
                         "(profiles/k_transport_plan2000.md)"},
}

# Instruction issue of the transport kernel (ncu --set full on the plan's first 2e6 histories,
# same command as the L2 reduction figures); reported only while the sources match its hash.
TRANSPORT_ISSUE = {
    "plan2000": {"src": "2c263b682767634b", "issue_active_pct": 79.81, "lanes_per_warp_instruction": 24.86,
                 "warp_instructions": 7_517_505_206, "euler_steps": 525_487_490,
                 "pipe_pct": {"alu": 47.96, "fma": 41.16, "fp64": 25.43, "xu_cycles": 40.29, "lsu": 5.87},
                 "eligible_warps_per_issue": 3.15,
                 "note": "ncu smsp__issue_active (of active cycles), smsp__thread_inst_executed_per_inst_executed, "
                         "smsp__inst_executed.sum, sm__pipe_*_cycles_active, smsp__average_warps_issue_stalled_"
                         "not_selected_per_issue_active of k_transport in `bench.py --histories 2000000 --no-autotune "
                         "--steps 1 --warmup 1 --e2e-steps 0 --no-denoiser --no-cpu-baseline --no-secondary` "
                         "(profiles/k_transport_plan2000.md)"},
}

WORKLOADS = {
    "plan2000": ("plan2000: 2000 spots on a 5 mm grid, E U(70,200) MeV, lognormal(0,0.7) weights, "
                 "1e8 protons per GPU, 200x200x300 mm at 1 mm, water + 30 random spheres (tissue/bone, "
                 "0.2-1.9 g/cm3); one persistent autotuned launch", 100_000_000),
    "slab150": ("slab150: 150 MeV pencil beam (sigma_xy 3 mm), 1e6 protons per GPU, "
                "60x60x200 mm at 0.5 mm (120x120x400 voxels), water/bone-like/lung-like/water slabs", 1_000_000),
    "insert150": ("insert150: 150 MeV beam (sigma_xy 3 mm), 1e7 protons per GPU, 80x80x200 mm at 1 mm, water with "
                  "a bone-like half-space insert (x > 0, z 30-80 mm) whose edge lies on the beam axis", 10_000_000),
    "ct_sobp": ("ct_sobp: thorax-like synthetic CT 120x120x240 mm at 1 mm (air, lung, adipose, soft tissue, "
                "cortical bone from HU), 16-layer spread-out Bragg peak 90-140 mm, 256 spots, 1e6 protons per GPU",
                1_000_000),
}


def _make_workload(name, total):
    from sde_workloads import ct_sobp, insert150, plan2000, slab150
    return {"plan2000": plan2000, "slab150": slab150, "insert150": insert150, "ct_sobp": ct_sobp}[name](total)


def transport_source_hash():
    h = hashlib.sha256()
    for f in TRANSPORT_SOURCES:
        with open(os.path.join(ROOT, "paper_2511_03115_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


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


def _oracle_rate(wl, n, seed, handle=None):
    """Histories/s of the oracle on ``wl`` rescaled to ``n`` histories (same phantom and
    spots, each spot's count in proportion); returns (rate, seconds, balance)."""
    import oracle
    sample = wl.with_histories(n)
    own = handle is None
    d = oracle.OracleDose(sample) if own else handle
    try:
        d.reset()
        t0 = time.perf_counter()
        d.run(spots=sample.spots, seed=seed)
        dt = time.perf_counter() - t0
        bal = _oracle_balance(d)
    finally:
        if own:
            d.close()
    return n / dt, dt, bal


def _oracle_balance(d):
    import ctypes as C
    import oracle
    b = oracle.Balance()
    oracle._check(oracle.lib().oracle_fetch(d.h, None, None, C.byref(b)))
    return b.as_dict()


def cpu_baseline(workload: str, target_s: float = 20.0):
    """The oracle as it stands on the host cores, on a bounded sample of the workload: the
    same phantom and spot list with the history count scaled down (each spot keeps its share)."""
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    wl = _make_workload(workload, WORKLOADS[workload][1])
    d = oracle.OracleDose(wl)
    try:
        # calibrate on a sample long enough that the per-run setup (per-thread tallies of the
        # whole grid, their sum) does not dominate, then size the timed sample to target_s
        cal = 200_000
        rate, dt, _ = _oracle_rate(wl, cal, 12345, d)
        n = int(min(10_000_000, max(cal, rate * target_s)))
        rate, dt, bal = _oracle_rate(wl, n, 777, d)
    finally:
        d.close()
    return {"value": rate, "unit": "histories/s", "cores": cores, "kind": "oracle",
            "sample": f"{workload} phantom and spots, histories scaled to {n} (seed 777), FP64 oracle, "
                      f"{cores} threads, {dt:.1f} s", "steps_per_s": bal["steps"] / dt}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, on the same workload, each step a
    bounded sample of it (same phantom and spots, histories scaled down)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    desc, full = WORKLOADS[args.workload]
    wl = _make_workload(args.workload, full)
    n = args.ref_histories
    d = oracle.OracleDose(wl)
    try:
        for w in range(args.warmup):
            _oracle_rate(wl, n, 10_000 + w, d)
        times = [_oracle_rate(wl, n, 20_000 + k, d)[1] for k in range(args.steps)]
    finally:
        d.close()
    T = sum(times) / len(times)
    v = n / T
    line = {
        "impl": "reference", "metric": METRIC, "value": v,
        "unit": "histories/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": T * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "histories_per_step": n,
                   "sample": f"{n} histories per step: the workload's phantom and spots, each spot's "
                             f"history count scaled down in proportion", "parallelism": f"{cores} host threads"},
        "cpu_baseline": {"value": v, "unit": "histories/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n} histories of the {args.workload} workload per step"},
        "e2e": {"value": v, "unit": "histories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def time_steps(torch, d, spots_dev, n_spots, steps, warmup, stream, flush, first=None, count=None,
               seed_base=1_000_003, barrier=None):
    """W untimed steps, then K timed steps on the handle's stream (CUDA events), L2 flushed
    before each timed step outside the events.  Returns (step ms, transport ms) lists: a
    step is reset + spot prep + transport; the second time excludes the reset."""
    def step(k):
        d.reset()
        d.run_device(spots_dev.data_ptr(), n_spots, seed=seed_base + k, first=first, count=count)

    for w in range(warmup):
        step(10_000 + w)
    d.sync()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    evs = []
    for k in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        s = torch.cuda.Event(enable_timing=True)
        m = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        d.reset()
        m.record(stream)
        d.run_device(spots_dev.data_ptr(), n_spots, seed=seed_base + k, first=first, count=count)
        e.record(stream)
        evs.append((s, m, e))
    stream.synchronize()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    return [s.elapsed_time(e) for s, _, e in evs], [m.elapsed_time(e) for _, m, e in evs]


def alu_roofline(steps_per_launch, kernel_ms, sms, clk_mhz):
    peak = sms * LANE_OPS_PER_CLK_PER_SM * clk_mhz * 1e6
    achieved = steps_per_launch * ALGO_OPS_PER_STEP / (kernel_ms * 1e-3)
    return achieved, peak


def per_spot_benchmark(torch, S, wl, d, spots_dev, stream, flush):
    """The plan as one launch per spot (all spots, one after another on the handle's stream),
    against the one persistent launch: device time of the whole sequence."""
    rec = int(wl.spots.dtype.itemsize)
    n = len(wl.spots)

    def seq(seed):
        for i in range(n):
            d.run_device(spots_dev.data_ptr() + i * rec, 1, seed=seed * 10_000 + i)

    ts = []
    for r in range(2):
        with torch.cuda.stream(stream):
            flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        d.reset()
        a.record(stream)
        seq(r)
        b.record(stream)
        stream.synchronize()
        ts.append(a.elapsed_time(b))
    d.sync()
    ms = min(ts[1:] or ts)
    return {"spots": n, "launches": 2 * n, "ms": ms, "histories_per_s": wl.n_histories / (ms * 1e-3),
            "note": "every spot of the plan as its own prep + transport launch (no extrapolation)"}


def slab_secondary(torch, S, dev, stream, flush, sms, clk_mhz, steps=10, warmup=3):
    """The slab phantom (150 MeV, 10^6 protons, 0.5 mm voxels) as a secondary line."""
    wl = _make_workload("slab150", WORKLOADS["slab150"][1])
    sp = torch.from_numpy(wl.spots.view(np.uint8).copy()).to(dev)
    with S.SdeDose(wl, stream=stream) as d:
        step_ms, kern_ms = time_steps(torch, d, sp, len(wl.spots), steps, warmup, stream, flush)
        _, _, bal = d.fetch(dose=False, edep=False)
    T, Tk = float(np.mean(step_ms)), float(np.mean(kern_ms))
    ach, peak = alu_roofline(bal["steps"], Tk, sms, clk_mhz)
    return {"workload": WORKLOADS["slab150"][0], "value": wl.n_histories / (T * 1e-3), "unit": "histories/s",
            "ms_per_step": T, "kernel_ms": Tk, "euler_steps_per_launch": bal["steps"],
            "alu_frac": ach / peak, "balance_exact": bal["incident"] == bal["deposited"] + bal["escaped"] + bal["removed"]}


# Executed multiply-adds of one denoiser inference on 128 x 128 x 192 (16-channel padded
# input and output layers): (voxels, Cin, Cout) per convolution, 27 taps each.
# (voxels, live input channels, live output channels) per convolution of one inference: the
# input layer reads 2 live channels (dose, density) of its 16, the output layer writes 1 of its
# 16; the kernels compute the padded channels too (DENOISER_LAYERS_PADDED).
DENOISER_LAYERS = [(3_145_728, 2, 32), (3_145_728, 32, 32), (393_216, 32, 64), (393_216, 64, 64),
                   (49_152, 64, 128), (49_152, 128, 128), (393_216, 192, 64), (393_216, 64, 64),
                   (3_145_728, 96, 32), (3_145_728, 32, 32), (3_145_728, 32, 1)]
DENOISER_LAYERS_PADDED = [(v, 16 if i == 0 else ci, 16 if i == len(DENOISER_LAYERS) - 1 else co)
                          for i, (v, ci, co) in enumerate(DENOISER_LAYERS)]
DENOISER_WEIGHTS = os.path.join(ROOT, "paper_2511_03115_gb300", "weights", "denoiser_128x128x192.npy")
# FP64-oracle doses of held-out denoiser plans, written by tests/golden/make_denoise_reference.py
# (which calls only the oracle): the benchmark reads them as stored reference values.
DENOISER_REFERENCE = os.path.join(ROOT, "tests", "golden", "denoise_reference_{}.npz")


def _oracle_reference(torch, seed, n_low):
    """The stored oracle dose of held-out plan ``seed`` in the units of an n_low-history GPU
    dose (device FP32 [nz, ny, nx]), or None."""
    path = DENOISER_REFERENCE.format(seed)
    if not os.path.exists(path):
        return None, 0
    z = np.load(path)
    ref = z["dose_rel"].astype(np.float32) * np.float32(float(z["dmax_per_history"]) * n_low)
    return torch.from_numpy(ref).cuda(), int(z["histories"])


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
        r = DN.transport_doses(seed, timing=True)
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
        oref, n_or = _oracle_reference(torch, seed, DN.N_LOW)
        if oref is not None:  # against the FP64 oracle's dose of the same plan
            omax = float(oref.max())
            row["vs_fp64_oracle"] = {
                "oracle_histories": n_or,
                **{f"gamma_{k}": S.gamma3d(oref, v, (1.0, 1.0, 1.0)) for k, v in
                   (("low", r["low"]), ("learned", den), ("high", ref))},
                **{f"max_err_{k}": float((v - oref).abs().max()) / omax for k, v in
                   (("low", r["low"]), ("learned", den), ("high", ref))}}
        rows.append(row)
    net.close()
    mean = lambda k: float(np.mean([r[k] for r in rows]))
    learned_ms = mean("t_low_ms") + mean("t_infer_ms")
    plain = [{"histories": n, "ms": float(np.mean([r["plain"][j]["ms"] for r in rows])),
              "gamma": float(np.mean([r["plain"][j]["gamma"] for r in rows])),
              "all_ge_95": all(r["plain"][j]["gamma"] >= 0.95 for r in rows)} for j, n in enumerate(ladder)]
    first_pass = next((p for p in plain if p["all_ge_95"]), None)
    vs_oracle = [dict(seed=r["seed"], **r["vs_fp64_oracle"]) for r in rows if "vs_fp64_oracle" in r]
    return {"cases": len(rows), "learned_ms": learned_ms, "gamma_learned": mean("gamma_learned"),
            "vs_fp64_oracle": vs_oracle or None,
            "learned_all_ge_95": all(r["gamma_learned"] >= 0.95 for r in rows),
            "max_err_learned": mean("max_err_learned"), "gamma_low": mean("gamma_low"),
            "max_err_low": mean("max_err_low"), "plain_1e7_ms": mean("t_high_ms"), "plain_ladder": plain,
            "plain_ms_at_95": first_pass["ms"] if first_pass else None,
            "plain_histories_at_95": first_pass["histories"] if first_pass else None,
            "note": "device time (CUDA events) of transport + dose conversion (+ inference) on a warm handle "
                    "(one untimed run of the same size first, both arms); gamma 2%/0.5mm, 1% threshold, local, "
                    "vs the 1e7-history plain dose; held-out seeds of the denoiser workload"}


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
    flop_padded = sum(2.0 * v * 27 * ci * co for v, ci, co in DENOISER_LAYERS_PADDED)
    peak = peaks.get("bf16_tflops")
    tf = flop / (ms * 1e-3) / 1e12
    return {"infer_ms": ms, "flop_per_inference": flop, "flop_per_inference_padded": flop_padded,
            "flop_note": "live channels (2 in, 1 out at the ends); padded counts 16 and 16",
            "achieved_tflops": tf, "bound": "tensor",
            "peak_tflops": peak, "frac": tf / peak if peak else None,
            "peak_note": "measured bf16 burst peak (MEASURED_PEAKS.json)" if peak else "no measured peak"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="plan2000", choices=sorted(WORKLOADS),
                    help="plan2000 (default): the batched 2000-spot plan with 1e8 protons; slab150; insert150; ct_sobp")
    ap.add_argument("--histories", type=int, default=0, help="protons per GPU (0: the workload's own count)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-histories", type=int, default=100_000,
                    help="histories per step of the reference arm (a bounded sample of the workload)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch shape")
    ap.add_argument("--theta-cut-sigmas", type=float, default=0.0,
                    help="energy-dependent elastic cut-off theta_c = k sigma(E) (0: the paper's fixed 0.02 rad)")
    ap.add_argument("--secondary-fraction", type=float, default=0.0,
                    help="branching model: each non-elastic event of a primary also emits a secondary "
                         "proton with this fraction of the energy deficit (0: the paper's model)")
    ap.add_argument("--physics-mask", type=int, default=15,
                    help="ablation: SDE_PHYS_* bits of the transport (15 = all terms; 11 = no large-angle "
                         "elastic events, 3 = no jumps); a run with terms switched off is not the benchmark")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the per-spot launches of the plan and the slab-phantom line")
    ap.add_argument("--no-denoiser", action="store_true",
                    help="skip the learned-vs-plain time-to-dose and the denoiser throughput")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2511_03115_gb300 as S

    ws, rank, local = _dist()
    barrier = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        barrier = dist.barrier
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    desc, per_gpu = WORKLOADS[args.workload]
    per_gpu = args.histories or per_gpu
    # one plan; this rank runs its shard of the history ids
    wl = _make_workload(args.workload, per_gpu * ws)
    first, count = S.history_shard(wl.n_histories, rank, ws)
    stream = torch.cuda.Stream(device=dev)
    d = S.SdeDose(wl, stream=stream, theta_cut_sigmas=args.theta_cut_sigmas, physics_mask=args.physics_mask,
                  secondary_fraction=args.secondary_fraction)
    spots_dev = torch.from_numpy(wl.spots.view(np.uint8).copy()).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    tuned = None
    if not args.no_autotune:
        # launch shape picked on a 2e6-history subsample of this rank's plan (outside timing)
        tuned = d.autotune(wl.spots, seed=5, max_histories=2_000_000)

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    step_ms, kern_ms = time_steps(torch, d, spots_dev, len(wl.spots), args.steps, args.warmup, stream, flush,
                                  first=first, count=count, barrier=barrier)
    clocks = sampler.stop()
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
        d.run(wl.spots, seed=1_000_003 + 50_000 + k, first=first, count=count)
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
        d.run_device(spots_dev.data_ptr(), len(wl.spots), seed=1_000_003 + 90_000, first=first, count=count)
        tally = torch.empty(wl.n_voxels, dtype=torch.int64, device=dev)
        rb = d.fetch_device(edep_ptr=tally.data_ptr(), balance=True)
        torch.cuda.synchronize()
        dist.barrier()
        c0 = time.perf_counter()
        tot = S.combine_shards(tally, rb)
        torch.cuda.synchronize()
        c1 = time.perf_counter()
        inc, dep, esc, rem, nh = (tot[k] for k in ("incident", "deposited", "escaped", "removed", "histories"))
        combine = {"allreduce_ms": (c1 - c0) * 1e3, "bytes": wl.n_voxels * 8, "histories": nh,
                   "balance_exact": inc == dep + esc + rem and nh == wl.n_histories,
                   "tally_sum_equals_deposited": int(tally.sum()) == dep}

    peaks = _peaks()
    clk_mhz = peaks.get("sm_max_mhz", 2070.0)
    achieved, peak_ops = alu_roofline(steps_per_launch, Tk, sms, clk_mhz)
    src = transport_source_hash()
    traffic_rec = TRANSPORT_DRAM.get(args.workload)
    traffic = traffic_rec["bytes"] if traffic_rec and traffic_rec["src"] == src and count == traffic_rec.get(
        "histories", count) else None
    atom_rec = TRANSPORT_ATOMICS.get(args.workload)
    atomics = ({"bound": "l2_red", "pct_of_peak": atom_rec["l2_red_pct_of_peak"],
                "busiest_slice_pct_of_peak": atom_rec["busiest_l2_slice_pct"],
                "red_sectors_per_euler_step": atom_rec["red_sectors"] / atom_rec["euler_steps"],
                "note": atom_rec["note"], "transport_src": src}
               if atom_rec and atom_rec["src"] == src else None)
    iss_rec = TRANSPORT_ISSUE.get(args.workload)
    issue = ({"issue_active_pct": iss_rec["issue_active_pct"],
              "lanes_per_warp_instruction": iss_rec["lanes_per_warp_instruction"],
              "lane_instructions_per_euler_step":
                  iss_rec["warp_instructions"] * iss_rec["lanes_per_warp_instruction"] / iss_rec["euler_steps"],
              "pipe_pct": iss_rec["pipe_pct"], "eligible_warps_per_issue": iss_rec["eligible_warps_per_issue"],
              "note": iss_rec["note"], "transport_src": src}
             if iss_rec and iss_rec["src"] == src else None)
    line = {
        "metric": METRIC,
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
        "config": {"workload": desc, "histories_per_step": hist_per_step,
                   "split": f"history ids {first}..{first + count - 1} of {wl.n_histories} on rank {rank}",
                   "euler_steps_per_launch": steps_per_launch, "parallelism": f"replicas x{ws}",
                   "l2": "inputs (phantom + tally) and a 256 MB flush write before every timed step",
                   "tally": "int64 fixed point 2^-24 MeV",
                   "elastic_cut_off": (f"theta_c = {args.theta_cut_sigmas} sigma(E)" if args.theta_cut_sigmas > 0
                                       else "fixed 0.02 rad"),
                   "physics_mask": args.physics_mask,
                   "secondaries": (f"branching model, kappa {args.secondary_fraction} (one queued generation)"
                                   if args.secondary_fraction > 0 else "none (the paper's single-proton model)"),
                   "autotuned": tuned is not None, "tuning": d.get_tuning()},
        "e2e": {"value": hist_per_step / e2e_T, "unit": "histories/s",
                "h2d_bytes_per_step": int(wl.spots.nbytes),
                "d2h_bytes_per_step": int(wl.n_voxels * 8 + 64)},
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_ops / 1e9,
                     "unit": "Gop/s", "frac": achieved / peak_ops, "traffic": traffic,
                     "traffic_note": (traffic_rec or {}).get("note") if traffic is not None else
                     "null: no ncu capture of this transport source (hash %s) for this workload" % src,
                     "kernel": "k_transport (+ single-block spot prep)", "kernel_ms": Tk,
                     "ops_per_step": ALGO_OPS_PER_STEP, "euler_steps_per_s": steps_per_launch / (Tk * 1e-3),
                     "transport_src": src,
                     "peak_note": f"{sms} SMs (device attribute) x {LANE_OPS_PER_CLK_PER_SM} lane-ops/clk x "
                                  f"{clk_mhz:.0f} MHz (measured max SM clock)"},
        "tally_atomics": atomics,
        "transport_issue": issue,
        "clocks": clocks,
        "balance_exact": bal["incident"] == bal["deposited"] + bal["escaped"] + bal["removed"],
        "combine": combine,
    }
    if rank == 0 and ws == 1 and not args.no_secondary:
        if args.workload == "plan2000":
            line["per_spot_launches"] = per_spot_benchmark(torch, S, wl, d, spots_dev, stream, flush)
            line["per_spot_launches"]["one_launch_ms"] = T
        if args.workload != "slab150":
            line["slab150"] = slab_secondary(torch, S, dev, stream, flush, sms, clk_mhz)
    d.close()
    del flush
    if rank == 0 and ws == 1 and not args.no_denoiser:
        line["time_to_dose"] = time_to_dose(torch, S)
        line["denoiser"] = denoiser_roofline(torch, S, peaks)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
