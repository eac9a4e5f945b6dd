"""Per-layer timing of the denoiser's tensor-core convolutions.

``python -m paper_2511_03115_gb300.conv_bench`` times the forward convolution (and the
weight gradient) of every layer shape of the 128 x 128 x 192 denoiser on random BF16
data, then a full inference and a training step, and prints one line per layer with
the achieved TFLOP/s (2 x voxels x 27 x Cin x Cout per forward; each call also packs its
weights for the tensor core, which the network does once per weight update).  ``--shape D H W Cin
Cout`` runs only that convolution ``--reps`` times (a small case for a profiler), or with
``--wgrad`` its weight gradient; ``--infer`` times only the whole-network inference.
"""
from __future__ import annotations

import argparse
import json

import paper_2511_03115_gb300 as S

# (D, H, W, Cin, Cout) of the forward layers, then the data-gradient shapes that differ
LAYER_SHAPES = [
    (192, 128, 128, 16, 32), (192, 128, 128, 32, 32), (96, 64, 64, 32, 64), (96, 64, 64, 64, 64),
    (48, 32, 32, 64, 128), (48, 32, 32, 128, 128), (96, 64, 64, 192, 64), (192, 128, 128, 96, 32),
    (192, 128, 128, 32, 16), (192, 128, 128, 32, 96), (96, 64, 64, 64, 192),
]


def _time(fn, reps, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    stream.synchronize()
    return a.elapsed_time(b) / reps


def _tensors(D, H, W, ci, co, seed=0):
    """Random input and weights, zeroed output; activations padded channel-group-major."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    x = S.to_pcg((0.5 * torch.randn(1, D, H, W, ci, device="cuda", generator=g)).to(torch.bfloat16))
    w = (0.05 * torch.randn(co, 27, ci, device="cuda", generator=g)).to(torch.bfloat16)
    b = torch.zeros(co, device="cuda")
    y = S.pcg_zeros(1, co, D, H, W)
    return x, w, b, y


def main():
    import torch
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--shape", type=int, nargs=5, default=None, metavar=("D", "H", "W", "CIN", "COUT"))
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--wgrad", action="store_true", help="with --shape: run the weight gradient")
    ap.add_argument("--infer", action="store_true",
                    help="only the whole-network inference: 4 warm-up calls, then --reps timed ones")
    args = ap.parse_args()
    torch.cuda.init()
    st = torch.cuda.current_stream()
    if args.infer:
        net = S.Denoiser(192, 128, 128, batch_max=1, seed=1)
        low = torch.rand(192, 128, 128, device="cuda")
        rho = torch.ones_like(low)
        for _ in range(4):
            net.infer(low, rho)
        ms = _time(lambda: net.infer(low, rho), args.reps, st)
        S.denoise_status()
        net.close()
        print(json.dumps({"infer_ms": ms, "reps": args.reps}))
        return
    if args.shape:
        D, H, W, ci, co = args.shape
        x, w, b, y = _tensors(D, H, W, ci, co)
        if args.wgrad:
            dw = torch.zeros(co, 27, ci, device="cuda")
            dy = S.to_pcg((0.5 * torch.randn(1, D, H, W, co, device="cuda")).to(torch.bfloat16))
        for _ in range(args.reps):
            if args.wgrad:
                S.conv3d_wgrad(x, dy, dw)
            else:
                S.conv3d(x, w, b, relu=True, y=y)
        torch.cuda.synchronize()
        S.denoise_status()
        print(json.dumps({"shape": args.shape, "reps": args.reps, "wgrad": args.wgrad, "ok": True}))
        return
    rows = []
    for D, H, W, ci, co in LAYER_SHAPES:
        x, w, b, y = _tensors(D, H, W, ci, co)
        flop = 2.0 * D * H * W * 27 * ci * co
        ms = _time(lambda: S.conv3d(x, w, b, relu=True, y=y), args.reps, st)
        S.denoise_status()
        row = {"shape": [D, H, W, ci, co], "fwd_ms": ms, "fwd_tflops": flop / ms / 1e9}
        if co <= 128:
            dw = torch.zeros(co, 27, ci, device="cuda")
            dy = S.to_pcg(torch.randn(1, D, H, W, co, device="cuda").to(torch.bfloat16))
            ms_w = _time(lambda: S.conv3d_wgrad(x, dy, dw), max(1, args.reps // 3), st)
            S.denoise_status()
            row.update({"wgrad_ms": ms_w, "wgrad_tflops": flop / ms_w / 1e9})
        rows.append(row)
        print(json.dumps(row), flush=True)
    net = S.Denoiser(192, 128, 128, batch_max=1, seed=1)
    low = torch.rand(192, 128, 128, device="cuda")
    rho = torch.ones_like(low)
    high = 1.01 * low
    infer = _time(lambda: net.infer(low, rho), 5, st)
    step = _time(lambda: net.train_step(low, rho, high, lr=1e-6, want_loss=False), 3, st)
    S.denoise_status()
    net.close()
    print(json.dumps({"infer_ms": infer, "train_step_ms": step}))


if __name__ == "__main__":
    main()
