"""Writes the FP64-oracle dose of held-out plans of the denoiser workload
(``denoise_reference_<seed>.npz`` beside this script): the reference against which the
benchmark reports the learned dose's gamma pass rate and maximum error.

Calls only the oracle (``oracle/``) on the seeded synthetic workload
``sde_workloads.denoise_case(seed)``; nothing from the CUDA path enters the file.  The dose
is stored relative to its maximum as float16 (3 significant digits, far below the dose's
statistical spread at these history counts), with the maximum dose per history (Gy) and
the history count.

    python tests/golden/make_denoise_reference.py [--seeds 100000] [--histories 10000000]
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from sde_workloads import denoise_case  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seeds", type=int, nargs="+", default=[100_000])
    ap.add_argument("--histories", type=int, default=10_000_000)
    ap.add_argument("--oracle-seed", type=int, default=424_242)
    args = ap.parse_args()
    oracle.build()
    for seed in args.seeds:
        wl = denoise_case(seed, n_hist=args.histories)
        t0 = time.time()
        dose, _, bal = oracle.run_workload(wl, seed=args.oracle_seed)
        assert bal["incident"] == bal["deposited"] + bal["escaped"] + bal["removed"]
        out = os.path.join(HERE, f"denoise_reference_{seed}.npz")
        dmax = float(dose.max())
        np.savez_compressed(out, dose_rel=(dose / dmax).astype(np.float16),
                            dmax_per_history=np.float64(dmax / wl.n_histories),
                            histories=np.int64(wl.n_histories), plan_seed=np.int64(seed),
                            oracle_seed=np.int64(args.oracle_seed))
        print(f"seed {seed}: {wl.n_histories} histories in {time.time() - t0:.0f} s -> {out} "
              f"({os.path.getsize(out) / 1e6:.1f} MB)", flush=True)


if __name__ == "__main__":
    main()
