"""Training data, training loop and evaluation of the learned dose denoiser.

Pairs are generated by the SDE transport itself: for a seeded random phantom and
spot plan (``sde_workloads.denoise_case``), a 1e5-history dose is the input and the
1e7-history dose of the same plan is the target (scaled by 1e5/1e7 so both are
doses of the same fluence).  Every numerical step runs in the library's kernels
(transport, denoiser forward/backward/Adam, gamma); this module only sequences
the calls and owns the tensors (PyTorch device memory).

Run ``python -m paper_2511_03115_gb300.denoise --help`` for the full experiment.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

import paper_2511_03115_gb300 as S
from sde_workloads import denoise_case

N_LOW = 100_000
N_HIGH = 10_000_000
SHAPE = (128, 128, 192)  # nx, ny, nz (1 mm voxels)


def _torch():
    import torch
    return torch


def transport_doses(seed, n_low=N_LOW, n_high=N_HIGH, stream=None, want_high=True, timing=False):
    """Low- and high-history doses (device FP32, [nz, ny, nx]) and the density of one case.
    With ``timing`` also the device time of each transport run (run + dose conversion), after
    one untimed run of the same size on the handle (a warm handle, as in repeated use)."""
    torch = _torch()
    wl = denoise_case(seed, n_low, shape=SHAPE)
    nx, ny, nz = wl.shape
    st = stream or torch.cuda.current_stream()
    out = {}
    with S.SdeDose(wl, stream=st) as d:
        for name, n, rs in (("low", n_low, 2 * seed + 1), ("high", n_high, 2 * seed + 2)):
            if name == "high" and not want_high:
                continue
            spots = wl.with_histories(n).spots
            dose = torch.empty(nz, ny, nx, dtype=torch.float32, device="cuda")
            if timing:  # the handle's launch graph for this shape is built outside the timed run
                d.reset()
                d.run(spots, seed=rs + 1_000_003)
                d.dose_into(dose)
                st.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            d.reset()
            a.record(st)
            d.run(spots, seed=rs)
            d.dose_into(dose)
            b.record(st)
            st.synchronize()
            out[name] = dose
            out[name + "_ms"] = a.elapsed_time(b)
    out["density"] = torch.from_numpy(np.ascontiguousarray(wl.density)).cuda()
    return out


def generate(seeds, n_low=None, n_high=None):
    n_low = n_low or N_LOW
    n_high = n_high or N_HIGH
    pairs = []
    for s in seeds:
        r = transport_doses(s, n_low, n_high)
        pairs.append((r["low"], r["density"], r["high"]))
    return pairs


def train(net, pairs, epochs=2, lr=1e-4, lr_end=1e-6, warmup=50, seed=0, log_every=0, scale=None):
    """Adam with linear warm-up and a cosine learning-rate decay; one pair per step."""
    scale = scale or N_LOW / N_HIGH
    order_rng = np.random.default_rng(seed)
    steps = epochs * len(pairs)
    losses = []
    k = 0
    for ep in range(epochs):
        for i in order_rng.permutation(len(pairs)):
            lr_k = lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * k / max(steps - 1, 1)))
            lr_k *= min(1.0, (k + 1) / warmup)
            low, rho, high = pairs[i]
            want = log_every and (k % log_every == 0 or k == steps - 1)
            loss = net.train_step(low, rho, high, lr=lr_k, want_loss=bool(want), target_scale=scale)
            if want:
                losses.append((k, loss))
            k += 1
    return losses


LADDER = (10_000, 30_000, 100_000, 300_000, 1_000_000)


def plain_ladder(seed, ref, shape_scale, ladder=LADDER, dd=0.02, dta_mm=0.5, threshold=0.01):
    """Gamma pass rate and device time of the plain method at each history count of the
    ladder (doses scaled to the fluence of ``ref``), each timed after one untimed run of
    the same size on the handle."""
    torch = _torch()
    out = []
    wl = denoise_case(seed, N_LOW, shape=SHAPE)
    nx, ny, nz = wl.shape
    st = torch.cuda.current_stream()
    with S.SdeDose(wl, stream=st) as d:
        for j, n in enumerate(ladder):
            dose = torch.empty(nz, ny, nx, dtype=torch.float32, device="cuda")
            d.reset()  # untimed run of the same size first: a warm handle, as for the learned path
            d.run(wl.with_histories(n).spots, seed=8_000_000 + 10 * seed + j)
            d.dose_into(dose)
            st.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            d.reset()
            a.record(st)
            d.run(wl.with_histories(n).spots, seed=7_000_000 + 10 * seed + j)
            d.dose_into(dose)
            b.record(st)
            st.synchronize()
            S.scale_(dose, shape_scale / n)
            out.append({"histories": n, "ms": a.elapsed_time(b),
                        "gamma": S.gamma3d(ref, dose, (1.0, 1.0, 1.0), dd, dta_mm, threshold)})
    return out


def evaluate(net, seeds, dd=0.02, dta_mm=0.5, threshold=0.01, ladder=True, n_low=None, n_high=None):
    """Gamma pass rate and maximum dose error of the low-history dose and of the denoised
    dose against the high-history dose, the time to each dose, and (ladder) the gamma
    and time of the plain method over a range of history counts."""
    torch = _torch()
    rows = []
    n_low = n_low or N_LOW
    n_high = n_high or N_HIGH
    scale = n_low / n_high
    st = torch.cuda.current_stream()
    for s in seeds:
        r = transport_doses(s, n_low, n_high, timing=True)
        ref = S.scale_(r["high"], scale)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        den = net.infer(r["low"], r["density"])
        b.record(st)
        st.synchronize()
        S.denoise_status()
        infer_ms = a.elapsed_time(b)
        rmax = float(ref.max())
        rows.append({
            "seed": int(s),
            "gamma_low": S.gamma3d(ref, r["low"], (1.0, 1.0, 1.0), dd, dta_mm, threshold),
            "gamma_denoised": S.gamma3d(ref, den, (1.0, 1.0, 1.0), dd, dta_mm, threshold),
            "max_err_low": float((r["low"] - ref).abs().max()) / rmax,
            "max_err_denoised": float((den - ref).abs().max()) / rmax,
            "t_low_ms": r["low_ms"], "t_high_ms": r["high_ms"], "t_infer_ms": infer_ms,
        })
        if ladder:
            rows[-1]["plain"] = plain_ladder(s, ref, n_low, dd=dd, dta_mm=dta_mm, threshold=threshold)
    agg = {k: float(np.mean([row[k] for row in rows])) for k in rows[0] if k not in ("seed", "plain")}
    if ladder:
        agg["plain_ladder"] = [{"histories": n,
                                "gamma_mean": float(np.mean([row["plain"][j]["gamma"] for row in rows])),
                                "frac_gamma_ge_95": float(np.mean([row["plain"][j]["gamma"] >= 0.95 for row in rows])),
                                "ms_mean": float(np.mean([row["plain"][j]["ms"] for row in rows]))}
                               for j, n in enumerate(LADDER)]
    agg["time_to_dose_learned_ms"] = agg["t_low_ms"] + agg["t_infer_ms"]
    agg["time_to_dose_plain_ms"] = agg["t_high_ms"]
    agg["speedup"] = agg["time_to_dose_plain_ms"] / agg["time_to_dose_learned_ms"]
    agg["frac_denoised_gamma_ge_95"] = float(np.mean([row["gamma_denoised"] >= 0.95 for row in rows]))
    agg["frac_low_gamma_ge_95"] = float(np.mean([row["gamma_low"] >= 0.95 for row in rows]))
    return agg, rows


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--train", type=int, default=64, help="training pairs (seeds first-seed .. first-seed+n-1)")
    ap.add_argument("--first-seed", type=int, default=0, help="seed of the first training pair (below 100000)")
    ap.add_argument("--epochs", type=int, default=2)
    ap.add_argument("--eval", type=int, default=8, help="held-out pairs (seeds 100000..)")
    ap.add_argument("--lr", type=float, default=1e-4)
    ap.add_argument("--out", default=None, help="write the report as JSON here")
    ap.add_argument("--n-low", type=int, default=N_LOW, help="histories of the input dose")
    ap.add_argument("--n-high", type=int, default=N_HIGH, help="histories of the target dose")
    ap.add_argument("--save", default=None, help="write the trained FP32 parameters here (.npy)")
    ap.add_argument("--load", default=None, help="start from these parameters (.npy) instead of training from scratch")
    args = ap.parse_args()
    torch = _torch()
    torch.cuda.init()
    t0 = time.time()
    if args.first_seed + args.train > 100_000:
        raise SystemExit("training seeds must stay below the held-out seeds (100000 on)")
    pairs = generate(range(args.first_seed, args.first_seed + args.train), args.n_low, args.n_high)
    t_gen = time.time() - t0
    net = S.Denoiser(SHAPE[2], SHAPE[1], SHAPE[0], batch_max=1, seed=1)
    if args.load:
        net.set_params(np.load(args.load).astype(np.float32))
    t0 = time.time()
    losses = train(net, pairs, epochs=args.epochs, lr=args.lr, log_every=max(1, args.train // 4),
                   scale=args.n_low / args.n_high)
    torch.cuda.synchronize()
    S.denoise_status()
    t_train = time.time() - t0
    del pairs
    if args.save:
        np.save(args.save, net.get_params())
    agg, rows = evaluate(net, range(100_000, 100_000 + args.eval), n_low=args.n_low, n_high=args.n_high)
    report = {"train_pairs": args.train, "first_seed": args.first_seed, "epochs": args.epochs, "n_low": args.n_low, "n_high": args.n_high, "generate_s": t_gen, "train_s": t_train,
              "train_step_ms": 1e3 * t_train / max(1, args.train * args.epochs), "losses": losses,
              "params": net.num_params(), "eval": agg, "rows": rows}
    print(json.dumps(report))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(report, f, indent=1)


if __name__ == "__main__":
    main()
